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
// Tiles of op(A) and op(B) are staged in shared memory by TMA (3-D boxes over
// component, row and column, zero-filled past the edges) in the stored layout
// (interleaved or split planes, transposed or not); the A fragment of each
// m16n8k4 DMMA is gathered from the A tile with the sign of L(a) applied by
// an integer XOR, and conjugation of A or B only changes those signs.  The
// epilogue applies C <- alpha P + beta C with left products in FP64, each lane
// gathering the four components of its element by warp shuffles.
#include <cstring>

#include "common.cuh"

namespace qg {

__device__ int g_fp64_error;

namespace {

constexpr int kBMQ = 32;      // quaternion rows of C per CTA
constexpr int kBNQ = 32;      // quaternion columns of C per CTA
constexpr int kBKQ = 16;      // quaternion k per pipeline stage
constexpr int kStages = 3;
constexpr int kThreads = 128; // 4 warps, warp w owns rows [8w, 8w+8) x all 32 columns
constexpr int kGroupM = 16;   // row-tiles per rasterisation group
constexpr int kTileElems = kBMQ * kBKQ * 4;  // = kBKQ * kBNQ * 4 (doubles)
constexpr uint32_t kTileBytes = kTileElems * sizeof(double);
static_assert(kBMQ * kBKQ == kBKQ * kBNQ, "A and B tiles have the same size");
constexpr size_t kSmemBytes = 2 * kStages * kTileBytes + kStages * sizeof(uint64_t);

struct Fp64Args {
  int64_t m, n, k;
  const double *A;
  int64_t a_rows, a_cols, lda, psA;
  const double *B;
  int64_t b_rows, b_cols, ldb, psB;
  double *C;
  int64_t ldc, psC;
  double alpha[4], beta[4];
  uint32_t negmask;
  int tmaA, tmaB, beta_zero;
  uint64_t limit_ns;
};

// Shared-memory index of component s of stored element (r, c) of a tile with
// R stored rows and CC stored columns (the TMA box order).
template <int LAYOUT, int R, int CC>
__device__ __forceinline__ int tile_idx(int r, int c, int s) {
  if (LAYOUT == QGEMM_INTERLEAVED) return s + 4 * (r + R * c);
  return r + R * (c + CC * s);
}

// op(A) tile: element (i, kk), i < kBMQ, kk < kBKQ.
template <int LAYOUT, bool TA>
__device__ __forceinline__ int a_idx(int i, int kk, int s) {
  if (!TA) return tile_idx<LAYOUT, kBMQ, kBKQ>(i, kk, s);
  return tile_idx<LAYOUT, kBKQ, kBMQ>(kk, i, s);
}
// op(B) tile: element (kk, j), kk < kBKQ, j < kBNQ.
template <int LAYOUT, bool TB>
__device__ __forceinline__ int b_idx(int kk, int j, int s) {
  if (!TB) return tile_idx<LAYOUT, kBKQ, kBNQ>(kk, j, s);
  return tile_idx<LAYOUT, kBNQ, kBKQ>(j, kk, s);
}

// Plain-load fallback with the same shared-memory layout as the TMA box
// (used when base or strides are not 16-byte aligned).
template <int LAYOUT, int R, int CC>
__device__ void load_tile_plain(double *dst, const double *base, int64_t rows, int64_t cols,
                                int64_t ld, int64_t ps, int64_t r0, int64_t c0) {
  constexpr int N = R * CC * 4;
  for (int e = threadIdx.x; e < N; e += kThreads) {
    int r, c, s;
    if (LAYOUT == QGEMM_INTERLEAVED) {
      s = e & 3;
      const int rest = e >> 2;
      r = rest % R;
      c = rest / R;
    } else {
      r = e % R;
      c = (e / R) % CC;
      s = e / (R * CC);
    }
    const int64_t gr = r0 + r, gc = c0 + c;
    double v = 0.0;
    if (gr < rows && gc < cols)
      v = LAYOUT == QGEMM_INTERLEAVED ? base[4 * (gr + gc * ld) + s] : base[s * ps + gr + gc * ld];
    dst[e] = v;
  }
}

__device__ __forceinline__ void dmma_16x8x4(double (&d)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

template <int LAYOUT, bool TA, bool TB>
__global__ void __launch_bounds__(kThreads)
    fp64_qgemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const Fp64Args p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *sA = reinterpret_cast<double *>(smem_raw);
  double *sB = sA + kStages * kTileElems;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kStages * kTileElems);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  // grouped rasterisation: runs of kGroupM row-tiles share their B column
  // panels in L2 while they sweep the columns
  const int64_t tiles_m = (p.m + kBMQ - 1) / kBMQ, tiles_n = (p.n + kBNQ - 1) / kBNQ;
  const int64_t tid_lin = static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int64_t per_group = kGroupM * tiles_n;
  const int64_t first_m = (tid_lin / per_group) * kGroupM;
  const int64_t gsize = min(tiles_m - first_m, static_cast<int64_t>(kGroupM));
  const int64_t i0 = (first_m + (tid_lin % per_group) % gsize) * kBMQ;
  const int64_t n0 = ((tid_lin % per_group) / gsize) * kBNQ;
  const int ktiles = static_cast<int>((p.k + kBKQ - 1) / kBKQ);
  const bool any_tma = p.tmaA || p.tmaB;
  const uint32_t tx_bytes = (p.tmaA ? kTileBytes : 0u) + (p.tmaB ? kTileBytes : 0u);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
    if (p.tmaA) tma_prefetch_desc(&tmA);
    if (p.tmaB) tma_prefetch_desc(&tmB);
  }
  __syncthreads();

  // stored coordinates of the k-tile kt
  auto a_rc = [&](int kt, int64_t &r0, int64_t &c0) {
    const int64_t kk0 = static_cast<int64_t>(kt) * kBKQ;
    r0 = TA ? kk0 : i0;
    c0 = TA ? i0 : kk0;
  };
  auto b_rc = [&](int kt, int64_t &r0, int64_t &c0) {
    const int64_t kk0 = static_cast<int64_t>(kt) * kBKQ;
    r0 = TB ? n0 : kk0;
    c0 = TB ? kk0 : n0;
  };
  auto issue = [&](int kt, int st) {
    mbar_arrive_expect_tx(&full[st], tx_bytes);
    int64_t r0, c0;
    if (p.tmaA) {
      a_rc(kt, r0, c0);
      if (LAYOUT == QGEMM_INTERLEAVED)
        tma_load_3d(sA + st * kTileElems, &tmA, &full[st], 0, (int)r0, (int)c0);
      else
        tma_load_3d(sA + st * kTileElems, &tmA, &full[st], (int)r0, (int)c0, 0);
    }
    if (p.tmaB) {
      b_rc(kt, r0, c0);
      if (LAYOUT == QGEMM_INTERLEAVED)
        tma_load_3d(sB + st * kTileElems, &tmB, &full[st], 0, (int)r0, (int)c0);
      else
        tma_load_3d(sB + st * kTileElems, &tmB, &full[st], (int)r0, (int)c0, 0);
    }
  };
  if (tid == 0 && any_tma)
    for (int s = 0; s < kStages && s < ktiles; ++s) issue(s, s);

  // per-lane A-fragment component and sign (integer XOR on the high word)
  const int c_lane = g & 3;
  const int compA = c_lane ^ t;
  const uint32_t negA = ((p.negmask >> (4 * c_lane + t)) & 1u) << 31;
  const int arow = warp * 8 + (g >> 2);  // + 4r (+2 for the second half)

  double acc[2][4][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[r][cc][e] = 0.0;

  int kt = 0;
  bool aborted = false;
  for (; kt < ktiles; ++kt) {
    const int st = kt % kStages;
    const uint32_t par = (kt / kStages) & 1;
    if (!p.tmaA) {
      int64_t r0, c0;
      a_rc(kt, r0, c0);
      if (TA)
        load_tile_plain<LAYOUT, kBKQ, kBMQ>(sA + st * kTileElems, p.A, p.a_rows, p.a_cols, p.lda,
                                            p.psA, r0, c0);
      else
        load_tile_plain<LAYOUT, kBMQ, kBKQ>(sA + st * kTileElems, p.A, p.a_rows, p.a_cols, p.lda,
                                            p.psA, r0, c0);
    }
    if (!p.tmaB) {
      int64_t r0, c0;
      b_rc(kt, r0, c0);
      if (TB)
        load_tile_plain<LAYOUT, kBNQ, kBKQ>(sB + st * kTileElems, p.B, p.b_rows, p.b_cols, p.ldb,
                                            p.psB, r0, c0);
      else
        load_tile_plain<LAYOUT, kBKQ, kBNQ>(sB + st * kTileElems, p.B, p.b_rows, p.b_cols, p.ldb,
                                            p.psB, r0, c0);
    }
    bool ok = true;
    if (any_tma) ok = mbar_wait_bounded(&full[st], par, p.limit_ns);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    const double *a_t = sA + st * kTileElems;
    const double *b_t = sB + st * kTileElems;
#pragma unroll 4
    for (int kk = 0; kk < kBKQ; ++kk) {
      double a[2][2], b[4];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        a[r][0] = flip_sign(a_t[a_idx<LAYOUT, TA>(arow + 4 * r, kk, compA)], negA);
        a[r][1] = flip_sign(a_t[a_idx<LAYOUT, TA>(arow + 4 * r + 2, kk, compA)], negA);
      }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) b[cc] = b_t[b_idx<LAYOUT, TB>(kk, 8 * cc + g, t)];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) dmma_16x8x4(acc[r][cc], a[r][0], a[r][1], b[cc]);
    }
    __syncthreads();
    if (tid == 0 && any_tma && kt + kStages < ktiles) issue(kt + kStages, st);
  }

  if (aborted) {
    if (tid == 0) {
      atomicCAS(&g_fp64_error, 0, QGEMM_ERR_TIMEOUT);
      // let copies still in flight land before the CTA retires
      for (int q = kt; q < ktiles && q < kt + kStages; ++q)
        mbar_wait_bounded(&full[q % kStages], (q / kStages) & 1, p.limit_ns);
    }
    return;
  }

  // ---- epilogue: C <- alpha P + beta C, left products, FP64 ----
  double la[4], lb[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int s = c_lane ^ j;
    la[j] = basis_sign(s, j) < 0 ? -p.alpha[s] : p.alpha[s];
    lb[j] = basis_sign(s, j) < 0 ? -p.beta[s] : p.beta[s];
  }
  const int src_base = lane & ~0xC;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t qi = i0 + warp * 8 + 4 * r + (g >> 2) + 2 * (e >> 1);
        const int64_t qn = n0 + 8 * cc + 2 * t + (e & 1);
        const bool inb = qi < p.m && qn < p.n;
        double P[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = __shfl_sync(0xffffffffu, acc[r][cc][e], src_base | (j << 2));
        double out = la[0] * P[0];
        out = fma(la[1], P[1], out);
        out = fma(la[2], P[2], out);
        out = fma(la[3], P[3], out);
        double *dst;
        if (LAYOUT == QGEMM_INTERLEAVED)
          dst = p.C + 4 * (qi + qn * p.ldc) + c_lane;
        else
          dst = p.C + c_lane * p.psC + qi + qn * p.ldc;
        if (!p.beta_zero) {
          const double cin = inb ? *dst : 0.0;
          double Cq[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) Cq[j] = __shfl_sync(0xffffffffu, cin, src_base | (j << 2));
#pragma unroll
          for (int j = 0; j < 4; ++j) out = fma(lb[j], Cq[j], out);
        }
        if (inb) *dst = out;
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

template <int LAYOUT, bool TA, bool TB>
int launch_typed(const CUtensorMap &ta, const CUtensorMap &tb, const Fp64Args &args, dim3 grid,
                 cudaStream_t stream) {
  auto kern = fp64_qgemm_kernel<LAYOUT, TA, TB>;
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
  if (cudaGetLastError() != cudaSuccess) return QGEMM_ERR_CUDA;
  return QGEMM_SUCCESS;
}

// Encodes the 3-D tensor map of a stored FP64 operand for a box of R x CC
// stored elements; returns false when TMA cannot address it.
bool encode_fp64(CUtensorMap *map, const MatView &v, int layout, int R, int CC) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(v.ptr);
  if (base % 16 != 0) return false;
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

}  // namespace

int launch_fp64_gemm(const GemmDesc &d, cudaStream_t stream) {
  Fp64Args a{};
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
  a.limit_ns = wait_limit_ns();
  const bool ta = op_trans(d.opA), tb = op_trans(d.opB);
  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  a.tmaA = encode_fp64(&tmA, d.A, d.layout, ta ? kBKQ : kBMQ, ta ? kBMQ : kBKQ) ? 1 : 0;
  a.tmaB = encode_fp64(&tmB, d.B, d.layout, tb ? kBNQ : kBKQ, tb ? kBKQ : kBNQ) ? 1 : 0;
  const int64_t gx = (d.m + kBMQ - 1) / kBMQ, gy = (d.n + kBNQ - 1) / kBNQ;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  const int key = (d.layout << 2) | (ta << 1) | tb;
  switch (key) {
    case 0: return launch_typed<0, false, false>(tmA, tmB, a, grid, stream);
    case 1: return launch_typed<0, false, true>(tmA, tmB, a, grid, stream);
    case 2: return launch_typed<0, true, false>(tmA, tmB, a, grid, stream);
    case 3: return launch_typed<0, true, true>(tmA, tmB, a, grid, stream);
    case 4: return launch_typed<1, false, false>(tmA, tmB, a, grid, stream);
    case 5: return launch_typed<1, false, true>(tmA, tmB, a, grid, stream);
    case 6: return launch_typed<1, true, false>(tmA, tmB, a, grid, stream);
    default: return launch_typed<1, true, true>(tmA, tmB, a, grid, stream);
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
  return cudaGetLastError() == cudaSuccess ? QGEMM_SUCCESS : QGEMM_ERR_CUDA;
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
