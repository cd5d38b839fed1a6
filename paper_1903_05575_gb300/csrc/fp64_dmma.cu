// FP64 quaternion GEMM on the FP64 tensor cores (DMMA, mma.sync m16n8k4).
//
// The Hamilton product (Sec. 2.1, Eq. quaternion_prod) of a = op(A)_{i kappa}
// and b = op(B)_{kappa n} is linear in b:  (a b)^c = sum_j L(a)[c][j] b^j  with
// L(a)[c][j] = sign(c, j) a^(c xor j).  So the quaternion product C = op(A) op(B)
// is the real product  C_r (4m x n) = L(op(A)) (4m x 4k) * B_r (4k x n), where
// B_r and C_r put an element's four components on consecutive rows.  Every
// real multiply of this form is one of the 16 of a Hamilton product: nothing
// is redundant (16 m n k FMAs = the 32 m n k flops of the metric).
//
// One CTA computes a 32 x 32 quaternion tile (fp64_tile.cuh): tiles of op(A)
// and op(B) are staged by TMA in the stored layout, the A fragment of each
// DMMA is gathered with the sign of L(a) applied by an integer XOR
// (conjugation of A or B only changes those signs), and the epilogue applies
// C <- alpha P + beta C with left products in FP64.
#include <atomic>
#include <cstring>

#include "fp64_tile.cuh"

namespace qg {

__device__ int g_fp64_error;

namespace {

constexpr int kBMQ = 32;     // quaternion rows of C per CTA
constexpr int kBNQ = 32;     // quaternion columns of C per CTA
constexpr int kGroupM = 16;  // row-tiles per rasterisation group
using fp64::kBKQ;
using fp64::kSmemBytes;
using fp64::kStages;
using fp64::kThreads;

struct Fp64Args {
  fp64::Operands op;
  uint64_t limit_ns;
};

template <int LAYOUT, bool TA, bool TB, int BMQ = kBMQ, int BNQ = kBNQ>
__global__ void __launch_bounds__(kThreads)
    fp64_qgemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const Fp64Args p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *sA = reinterpret_cast<double *>(smem_raw);
  double *sB = sA + kStages * fp64::kMaxTileElems;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kStages * fp64::kMaxTileElems);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
    if (p.op.tmaA) tma_prefetch_desc(&tmA);
    if (p.op.tmaB) tma_prefetch_desc(&tmB);
  }
  __syncthreads();
  // grouped rasterisation: runs of kGroupM row-tiles share their B column
  // panels in L2 while they sweep the columns
  const int64_t tiles_m = (p.op.m + BMQ - 1) / BMQ, tiles_n = (p.op.n + BNQ - 1) / BNQ;
  const int64_t tid_lin = static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int64_t per_group = kGroupM * tiles_n;
  const int64_t first_m = (tid_lin / per_group) * kGroupM;
  const int64_t gsize = min(tiles_m - first_m, static_cast<int64_t>(kGroupM));
  const int64_t i0 = (first_m + (tid_lin % per_group) % gsize) * BMQ;
  const int64_t n0 = ((tid_lin % per_group) / gsize) * BNQ;
  if (fp64::tile_outside(p.op.tri, i0, n0, BMQ, BNQ)) return;
  uint32_t kb_run = 0;
  fp64::tile<LAYOUT, TA, TB, BMQ, BNQ>(p.op, &tmA, &tmB, sA, sB, full, kb_run, i0, n0,
                                       p.limit_ns, &g_fp64_error);
}

// K split: P = sum over z of the partial products (z ascending, so the result
// does not depend on the order the CTAs finished), then C <- alpha P + beta C
// with left products in FP64; beta == 0 does not read C.  tri: only the
// stored triangle (1 lower, 2 upper), its diagonal real (Hermitian update).
template <int LAYOUT>
__global__ void __launch_bounds__(256)
    splitk_reduce_kernel(const double *__restrict__ part, int ksplit, int64_t m, int64_t n,
                         double *C, int64_t ldc, int64_t psC, double a0, double a1, double a2,
                         double a3, double b0, double b1, double b2, double b3, int beta_zero,
                         int tri) {
  const double al[4] = {a0, a1, a2, a3}, be[4] = {b0, b1, b2, b3};
  const int64_t total = m * n, slab = total * 4;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    if ((tri == 1 && i < j) || (tri == 2 && i > j)) continue;
    double P[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int z = 0; z < ksplit; ++z) {
      const double2 *q = reinterpret_cast<const double2 *>(part + z * slab + 4 * e);
      const double2 lo = q[0], hi = q[1];
      P[0] += lo.x;
      P[1] += lo.y;
      P[2] += hi.x;
      P[3] += hi.y;
    }
    double *q[4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
      q[s] = LAYOUT == QGEMM_INTERLEAVED ? C + 4 * (i + j * ldc) + s : C + s * psC + i + j * ldc;
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    if (!beta_zero) {
#pragma unroll
      for (int s = 0; s < 4; ++s) c[s] = *q[s];
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      double v = 0.0;
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) {
        const int s = cc ^ j2;
        const double sg = basis_sign(s, j2) < 0 ? -1.0 : 1.0;
        v = fma(sg * al[s], P[j2], v);
        if (!beta_zero) v = fma(sg * be[s], c[j2], v);
      }
      *q[cc] = (tri && i == j && cc != 0) ? 0.0 : v;
    }
  }
}

// C <- beta C (k == 0 or alpha == 0), or C <- 0 when beta == 0.
template <typename T, int LAYOUT>
__global__ void scale_kernel(T *C, int64_t m, int64_t n, int64_t ldc, int64_t psC, double b0,
                             double b1, double b2, double b3, int beta_zero) {
  const double be[4] = {b0, b1, b2, b3};
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    T *q[4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
      q[s] = LAYOUT == QGEMM_INTERLEAVED ? C + 4 * (i + j * ldc) + s : C + s * psC + i + j * ldc;
    if (beta_zero) {
#pragma unroll
      for (int s = 0; s < 4; ++s) *q[s] = T(0);
      continue;
    }
    double c[4], o[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) c[s] = static_cast<double>(*q[s]);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      double v = 0.0;
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) v = fma(basis_sign(cc ^ j2, j2) * be[cc ^ j2], c[j2], v);
      o[cc] = v;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) *q[s] = static_cast<T>(o[s]);
  }
}

// Hermitian rank-k update with k == 0 or alpha == 0: C <- beta C on one
// triangle (beta real), the diagonal's vector parts set to zero.
template <typename T, int LAYOUT>
__global__ void herk_scale_kernel(T *C, int64_t n, int64_t ldc, int64_t psC, double beta, int tri) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    if ((tri == 1 && i < j) || (tri == 2 && i > j)) continue;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      T *q = LAYOUT == QGEMM_INTERLEAVED ? C + 4 * (i + j * ldc) + s : C + s * psC + i + j * ldc;
      *q = (beta == 0.0 || (i == j && s != 0)) ? T(0) : static_cast<T>(beta * static_cast<double>(*q));
    }
  }
}

template <int LAYOUT, bool TA, bool TB, int BMQ = kBMQ, int BNQ = kBNQ>
int launch_typed(const CUtensorMap &ta, const CUtensorMap &tb, const Fp64Args &args, dim3 grid,
                 cudaStream_t stream) {
  auto kern = fp64_qgemm_kernel<LAYOUT, TA, TB, BMQ, BNQ>;
  static bool attr_set[64];  // per instantiation and device; benign race (same value)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmemBytes)) != cudaSuccess) {
      cudaGetLastError();
      return QGEMM_ERR_CUDA;
    }
    attr_set[dev] = true;
  }
  kern<<<grid, kThreads, kSmemBytes, stream>>>(ta, tb, args);
  return launch_status();
}

}  // namespace

// Encodes the 3-D tensor map of a stored FP64 operand for a box of R x CC
// stored elements; returns false when TMA cannot address it.
bool encode_fp64_operand(CUtensorMap *map, const MatView &v, int layout, int R, int CC) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(v.ptr);
  if (base % 16 != 0 || v.rows <= 0 || v.cols <= 0) return false;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  if (layout == QGEMM_INTERLEAVED) {
    dims[0] = 4;
    dims[1] = static_cast<cuuint64_t>(v.rows);
    dims[2] = static_cast<cuuint64_t>(v.cols);
    strides[0] = 32;
    strides[1] = static_cast<cuuint64_t>(v.ld) * 32;
    box[0] = 4;
    box[1] = R;
    box[2] = CC;
  } else {
    if (v.ld % 2 != 0 || v.ps % 2 != 0) return false;
    dims[0] = static_cast<cuuint64_t>(v.rows);
    dims[1] = static_cast<cuuint64_t>(v.cols);
    dims[2] = 4;
    strides[0] = static_cast<cuuint64_t>(v.ld) * 8;
    strides[1] = static_cast<cuuint64_t>(v.ps) * 8;
    box[0] = R;
    box[1] = CC;
    box[2] = 4;
  }
  if (dims[1] >= (1ull << 32) || dims[2] >= (1ull << 32) || dims[0] >= (1ull << 32)) return false;
  if (strides[0] >= (1ull << 40) || strides[1] >= (1ull << 40)) return false;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void *>(v.ptr), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

fp64::Operands fp64_operands(const GemmDesc &d) {
  fp64::Operands a{};
  a.m = d.m;
  a.n = d.n;
  a.k = d.k;
  a.A = static_cast<const double *>(d.A.ptr);
  a.a_rows = d.A.rows;
  a.a_cols = d.A.cols;
  a.lda = d.A.ld;
  a.psA = d.A.ps;
  a.B = static_cast<const double *>(d.B.ptr);
  a.b_rows = d.B.rows;
  a.b_cols = d.B.cols;
  a.ldb = d.B.ld;
  a.psB = d.B.ps;
  a.C = static_cast<double *>(d.C);
  a.ldc = d.ldc;
  a.psC = d.psc;
  for (int s = 0; s < 4; ++s) {
    a.alpha[s] = d.alpha[s];
    a.beta[s] = d.beta[s];
  }
  a.negmask = block_neg_mask(op_conj(d.opA), op_conj(d.opB));
  a.beta_zero = d.beta_zero ? 1 : 0;
  a.tri = d.tri;
  a.krange = d.krange;
  a.swap = d.swap;
  return a;
}

int launch_keyed(int key, const CUtensorMap &tmA, const CUtensorMap &tmB, const Fp64Args &a,
                 dim3 grid, cudaStream_t stream);

// Number of K shares for the single-problem FP64 kernel.  With 16 x 16
// quaternion tiles and 2 CTAs per SM, a launch of w = tiles * s / (2 SMs)
// waves keeps the FP64 pipes busy for a fraction w / ceil(w) of its time.  For
// C of fewer than 8 waves of tiles, take the fewest shares s in [2, 256]
// whose fraction is within 2 % of the best, keeping at least 8 k-blocks (128
// quaternion k) per share, and split only when the best gains 5 % over s = 1.
// Plain products and the Hermitian update's triangle (whose tiles outside
// the triangle exit at once and do not count); no k-range (triangular
// operand) or turned-around problem.
int fp64_ksplit(const GemmDesc &d, int sms) {
  if (d.krange || d.swap || d.kwidth != 4 || d.m <= 0 || d.n <= 0) return 1;
  const int64_t tm = (d.m + 15) / 16, tn = (d.n + 15) / 16;
  // a square triangle keeps tm (tm + 1) / 2 of its tm^2 tiles
  const int64_t tiles = (d.tri && tm == tn) ? tm * (tm + 1) / 2 : tm * tn;
  const int64_t slots = 2LL * sms;
  if (tiles >= 8 * slots) return 1;
  const int64_t ktiles = (d.k + kBKQ - 1) / kBKQ;
  const int64_t smax = std::min<int64_t>(256, ktiles / 8);
  auto busy = [&](int64_t s) {
    const int64_t ctas = tiles * s;
    const int64_t waves = (ctas + slots - 1) / slots;
    return static_cast<double>(ctas) / static_cast<double>(waves * slots);
  };
  double top = busy(1);
  for (int64_t s = 2; s <= smax; ++s) top = std::max(top, busy(s));
  if (top < busy(1) + 0.05) return 1;
  for (int64_t s = 2; s <= smax; ++s)  // fewest shares within 2 % of the best
    if (busy(s) >= top - 0.02) return static_cast<int>(s);
  return 1;
}

size_t fp64_splitk_bytes(int64_t m, int64_t n, int ksplit) {
  return ksplit > 1 ? static_cast<size_t>(ksplit) * m * n * 4 * sizeof(double) : 0;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    return 152;  // GB300
  }
  return sms;
}

int launch_fp64_gemm(const GemmDesc &d, cudaStream_t stream) {
  return launch_fp64_gemm_ws(d, nullptr, 0, stream);
}

namespace {
// One-shot fault injection for the bounded-wait test (qgemm_debug_arm_fault).
std::atomic<int> g_fp64_debug_skip{0};
std::atomic<uint64_t> g_fp64_debug_limit{0};
}  // namespace

void fp64_arm_fault(int stage, uint64_t limit_ns) {
  g_fp64_debug_limit.store(limit_ns);
  g_fp64_debug_skip.store(stage + 1);
}

int launch_fp64_gemm_ws(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream) {
  const int debug_skip = g_fp64_debug_skip.exchange(0);
  // a plain product that fills the GPU many times over runs on the FP64 FMA
  // pipe, the faster of GB300's two FP64 pipes (fp64_dfma.cu); an armed fault
  // (a DMMA-kernel test hook) keeps the DMMA kernel
  if (!debug_skip && fp64_dfma_eligible(d, device_sms())) return launch_fp64_dfma(d, stream);
  Fp64Args a{};
  a.op = fp64_operands(d);
  a.op.debug_skip = debug_skip;
  a.limit_ns = a.op.debug_skip ? g_fp64_debug_limit.load() : wait_limit_ns();
  // K split when it pays and the caller's workspace holds the partials
  int ks = fp64_ksplit(d, device_sms());
  if (ks > 1) {
    const size_t per = static_cast<size_t>(d.m) * d.n * 4 * sizeof(double);  // one share
    const int64_t fit = (ws != nullptr && reinterpret_cast<uintptr_t>(ws) % 256 == 0)
                            ? static_cast<int64_t>(ws_bytes / per)
                            : 0;
    if (fit < ks) ks = static_cast<int>(fit);
    if (ks < 2) ks = 1;
  }
  if (ks > 1) {
    a.op.ksplit = ks;
    a.op.part = static_cast<double *>(ws);
  }
  const bool ta = op_trans(d.opA), tb = op_trans(d.opB);
  // 32 x 32 quaternion tiles, or 16 x 16 when 32 x 32 would give fewer than
  // about 32 waves of the 2 CTAs per SM that fit (the last, partial wave
  // idles the FP64 pipes of the SMs it leaves out: 16% at 1024^3)
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t big = ((d.m + kBMQ - 1) / kBMQ) * ((d.n + kBNQ - 1) / kBNQ);
  const bool small = big < 32LL * 2 * sms;
  const int bm = small ? 16 : kBMQ, bn = small ? 16 : kBNQ;
  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  a.op.tmaA = encode_fp64_operand(&tmA, d.A, d.layout, ta ? kBKQ : bm, ta ? bm : kBKQ) ? 1 : 0;
  a.op.tmaB = encode_fp64_operand(&tmB, d.B, d.layout, tb ? bn : kBKQ, tb ? kBKQ : bn) ? 1 : 0;
  const int64_t gx = (d.m + bm - 1) / bm, gy = (d.n + bn - 1) / bn;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy), static_cast<unsigned>(ks));
  const int key = (small ? 8 : 0) | (d.layout << 2) | (ta << 1) | tb;
  const int rc = launch_keyed(key, tmA, tmB, a, grid, stream);
  if (rc || ks == 1) return rc;
  return launch_splitk_reduce(d, a.op.part, ks, stream);
}

int launch_splitk_reduce(const GemmDesc &d, const double *part, int ks, cudaStream_t stream) {
  const int64_t total = d.m * d.n;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152LL * 16);
  double *C = static_cast<double *>(d.C);
  const double *al = d.alpha, *be = d.beta;
  if (d.layout == QGEMM_INTERLEAVED)
    splitk_reduce_kernel<QGEMM_INTERLEAVED><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        part, ks, d.m, d.n, C, d.ldc, d.psc, al[0], al[1], al[2], al[3], be[0], be[1], be[2],
        be[3], d.beta_zero ? 1 : 0, d.tri);
  else
    splitk_reduce_kernel<QGEMM_SPLIT_PLANES><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        part, ks, d.m, d.n, C, d.ldc, d.psc, al[0], al[1], al[2], al[3], be[0], be[1], be[2],
        be[3], d.beta_zero ? 1 : 0, d.tri);
  return launch_status();
}

int launch_keyed(int key, const CUtensorMap &tmA, const CUtensorMap &tmB, const Fp64Args &a,
                 dim3 grid, cudaStream_t stream) {
  switch (key) {
    case 0: return launch_typed<0, false, false>(tmA, tmB, a, grid, stream);
    case 1: return launch_typed<0, false, true>(tmA, tmB, a, grid, stream);
    case 2: return launch_typed<0, true, false>(tmA, tmB, a, grid, stream);
    case 3: return launch_typed<0, true, true>(tmA, tmB, a, grid, stream);
    case 4: return launch_typed<1, false, false>(tmA, tmB, a, grid, stream);
    case 5: return launch_typed<1, false, true>(tmA, tmB, a, grid, stream);
    case 6: return launch_typed<1, true, false>(tmA, tmB, a, grid, stream);
    case 7: return launch_typed<1, true, true>(tmA, tmB, a, grid, stream);
    case 8: return launch_typed<0, false, false, 16, 16>(tmA, tmB, a, grid, stream);
    case 9: return launch_typed<0, false, true, 16, 16>(tmA, tmB, a, grid, stream);
    case 10: return launch_typed<0, true, false, 16, 16>(tmA, tmB, a, grid, stream);
    case 11: return launch_typed<0, true, true, 16, 16>(tmA, tmB, a, grid, stream);
    case 12: return launch_typed<1, false, false, 16, 16>(tmA, tmB, a, grid, stream);
    case 13: return launch_typed<1, false, true, 16, 16>(tmA, tmB, a, grid, stream);
    case 14: return launch_typed<1, true, false, 16, 16>(tmA, tmB, a, grid, stream);
    default: return launch_typed<1, true, true, 16, 16>(tmA, tmB, a, grid, stream);
  }
}

int launch_scale(const GemmDesc &d, bool fp64, cudaStream_t stream) {
  const int64_t total = d.m * d.n;
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const int bz = d.beta_zero ? 1 : 0;
  const double *b = d.beta;
  if (fp64) {
    double *C = static_cast<double *>(d.C);
    if (d.layout == QGEMM_INTERLEAVED)
      scale_kernel<double, 0><<<blocks, threads, 0, stream>>>(C, d.m, d.n, d.ldc, d.psc, b[0], b[1],
                                                              b[2], b[3], bz);
    else
      scale_kernel<double, 1><<<blocks, threads, 0, stream>>>(C, d.m, d.n, d.ldc, d.psc, b[0], b[1],
                                                              b[2], b[3], bz);
  } else {
    float *C = static_cast<float *>(d.C);
    if (d.layout == QGEMM_INTERLEAVED)
      scale_kernel<float, 0><<<blocks, threads, 0, stream>>>(C, d.m, d.n, d.ldc, d.psc, b[0], b[1],
                                                             b[2], b[3], bz);
    else
      scale_kernel<float, 1><<<blocks, threads, 0, stream>>>(C, d.m, d.n, d.ldc, d.psc, b[0], b[1],
                                                             b[2], b[3], bz);
  }
  return launch_status();
}

int launch_herk_scale(const GemmDesc &d, bool fp64, cudaStream_t stream) {
  const int64_t total = d.m * d.m;
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) return QGEMM_SUCCESS;
  const double be = d.beta[0];
  if (fp64) {
    double *C = static_cast<double *>(d.C);
    if (d.layout == QGEMM_INTERLEAVED)
      herk_scale_kernel<double, 0><<<blocks, threads, 0, stream>>>(C, d.m, d.ldc, d.psc, be, d.tri);
    else
      herk_scale_kernel<double, 1><<<blocks, threads, 0, stream>>>(C, d.m, d.ldc, d.psc, be, d.tri);
  } else {
    float *C = static_cast<float *>(d.C);
    if (d.layout == QGEMM_INTERLEAVED)
      herk_scale_kernel<float, 0><<<blocks, threads, 0, stream>>>(C, d.m, d.ldc, d.psc, be, d.tri);
    else
      herk_scale_kernel<float, 1><<<blocks, threads, 0, stream>>>(C, d.m, d.ldc, d.psc, be, d.tri);
  }
  return launch_status();
}

int fp64_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_fp64_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_fp64_error, &z, sizeof(int));
  return v;
}

}  // namespace qg
