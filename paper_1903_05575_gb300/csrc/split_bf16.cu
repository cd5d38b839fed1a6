// Split-BF16 quaternion GEMM, single problem: host side of the path whose
// device code is in split_core.cuh (the real form C' = A' B' with the 4x4
// sign expansion of B, FP32 -> 3 x BF16 split, six term products on tcgen05,
// chunked TMEM drain, FP64 final combination), the tcgen05 throughput probe,
// and the fixed-scratch entry point's scratch array.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "split_core.cuh"

namespace qg {

__device__ int g_split_error;

namespace {

using namespace split;

struct SplitErr {
  static __device__ int *word() { return &g_split_error; }
};

template <bool IS_B>
__global__ void __launch_bounds__(256) split_prepass_kernel(const PrepArgs p) {
  __shared__ float4 tile[32][33];
  prep_tile<IS_B>(p, blockIdx.x, blockIdx.y, tile);
}

// ----------------------------------------------------- tcgen05 probe ---
// Back-to-back M=128, N=PN, K=16 BF16 MMAs on a fixed shared-memory tile,
// one CTA per SM: the tensor-pipe throughput of one instruction shape.  FILL
// puts integer values in [-127, 127] in the tile (as the GEMMs see), else
// zeros (lower power, so higher clocks).
template <int PN, bool FILL>
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(int iters, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *buf = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  constexpr uint32_t kBBytes = PN * BK * 2;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < static_cast<int>((kATermBytes + kBBytes) / 4); i += blockDim.x) {
    uint32_t w = 0;
    if (FILL) {
      const uint32_t h0 = (2u * i + 1u) * 2654435761u, h1 = (2u * i + 2u) * 2654435761u;
      const float f0 = static_cast<float>(static_cast<int>((h0 >> 16) % 255u) - 127);
      const float f1 = static_cast<float>(static_cast<int>((h1 >> 16) % 255u) - 127);
      w = (__float_as_uint(f0) >> 16) | (__float_as_uint(f1) & 0xffff0000u);
    }
    reinterpret_cast<uint32_t *>(buf)[i] = w;
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tbase, PN < 32 ? 32 : PN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0 && elect_one()) {
    constexpr uint32_t idesc = idesc_bf16(BM, PN);
    const uint32_t sa = smem_u32(buf), sb = sa + kATermBytes;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        umma_bf16(tbase, smem_desc_sw64(sa + ks * 32), smem_desc_sw64(sb + ks * 32), idesc,
                  (it | ks) ? 1u : 0u);
    }
    umma_commit(&bar);
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicCAS(&g_split_error, 0, QGEMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, PN < 32 ? 32 : PN);
  }
}

// ----------------------------------------------------------- host side ---
struct SplitPlan {
  int64_t kp;           // padded real K
  size_t a_bytes, b_bytes, b_offset, total;
};

SplitPlan plan_for(const GemmDesc &d) {
  SplitPlan s;
  s.kp = ((d.kwidth * d.k + BK - 1) / BK) * BK;
  s.a_bytes = static_cast<size_t>(TERMS) * d.m * s.kp * 2;
  s.b_bytes = static_cast<size_t>(TERMS) * 4 * d.n * s.kp * 2;
  s.b_offset = (s.a_bytes + 1023) & ~static_cast<size_t>(1023);
  s.total = s.b_offset + s.b_bytes;
  return s;
}

GemmParams gemm_params(const GemmDesc &d, int64_t kp) {
  GemmParams g{};
  g.m = d.m;
  g.n = d.n;
  g.num_kb = static_cast<int>(d.k > 0 ? kp / BK : 0);
  g.num_mt = static_cast<int>((d.m + BM - 1) / BM);
  g.num_nt = static_cast<int>((d.n + BNQ - 1) / BNQ);
  g.C = static_cast<float *>(d.C);
  g.ldc = d.ldc;
  g.psC = d.psc;
  g.layout = d.layout;
  g.beta_zero = d.beta_zero ? 1 : 0;
  g.tri = d.tri;
  g.krange = d.krange;
  g.swap = d.swap;
  g.c_vec4 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
  for (int s = 0; s < 4; ++s) {
    g.alpha[s] = static_cast<float>(d.alpha[s]);
    g.beta[s] = static_cast<float>(d.beta[s]);
  }
  return g;
}

bool encode_bf16_3d(CUtensorMap *map, const void *base, int64_t kp, int64_t rows, int box_rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows), TERMS};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(kp) * 2,
                           static_cast<cuuint64_t>(kp) * 2 * static_cast<cuuint64_t>(rows)};
  cuuint32_t box[3] = {BK, static_cast<cuuint32_t>(box_rows), TERMS};
  cuuint32_t estr[3] = {1, 1, 1};
  if (rows >= (1ll << 32) || kp >= (1ll << 32)) return false;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int chunk_for(int num_kb) {
  // The in-TMEM FP32 accumulation error grows linearly with the number of
  // MMAs summed before a drain (measured on GB300: relative error 6.7e-7 at
  // 2 k-blocks and 2.0e-6 at 9 k-blocks for m=n=k=8192, N(0,1)), so drain
  // every 2 k-blocks (24 MMAs) unless overridden.
  int ch = 2;
  if (const char *s = std::getenv("QGEMM_SPLIT_CHUNK")) {
    int v = std::atoi(s);
    if (v > 0) ch = v;
  }
  (void)num_kb;
  return ch;
}

template <typename K>
int set_smem(K kern, size_t bytes) {
  static bool done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(bytes)) != cudaSuccess) {
      cudaGetLastError();
      return QGEMM_ERR_CUDA;
    }
    done[dev] = true;
  }
  return QGEMM_SUCCESS;
}

int launch_prepass(bool is_b, const MatView &v, int op, int64_t rows, int64_t kq, int64_t kp,
                   int kw, int layout, __nv_bfloat16 *out, int64_t term_stride,
                   cudaStream_t stream) {
  PrepArgs a;
  a.X = static_cast<const float *>(v.ptr);
  a.ld = v.ld;
  a.ps = v.ps;
  a.rows = rows;
  a.kq = kq;
  a.kp = kp;
  a.term_stride = term_stride;
  a.out = out;
  a.layout = layout;
  // A: op row i is the stored row for N/C; B: op row n is the stored row for T/H
  a.row_contig = is_b ? (op_trans(op) ? 1 : 0) : (op_trans(op) ? 0 : 1);
  a.negmask = op_conj(op) ? 0xEu : 0u;
  a.width = v.width;
  a.kw = kw;
  const int64_t gx = (rows + 31) / 32, gy = (kp / kw + 31) / 32;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (is_b)
    split_prepass_kernel<true><<<grid, 256, 0, stream>>>(a);
  else
    split_prepass_kernel<false><<<grid, 256, 0, stream>>>(a);
  return launch_status();
}

}  // namespace

// 3-D FP32 tensor map of a stored operand (shared with the grouped path).
bool encode_fp32_operand(CUtensorMap *map, const MatView &v, int layout, int R, int CC);

namespace {

// The fused single-problem path (no workspace) is taken when the caller asks
// for it with QGEMM_SPLIT_FUSED=1 and every operand is TMA-addressable.
bool plain_quaternion(const GemmDesc &d) {
  return d.kwidth == 4 && d.A.width == 4 && d.B.width == 4 && !d.swap;
}

bool want_fused() {
  const char *e = std::getenv("QGEMM_SPLIT_FUSED");
  return e && e[0] == '1';
}

bool fused_maps(const GemmDesc &d, CUtensorMap *tmA, CUtensorMap *tmB) {
  const bool ta = op_trans(d.opA), tb = op_trans(d.opB);
  return encode_fp32_operand(tmA, d.A, d.layout, ta ? FKQ : BM, ta ? BM : FKQ) &&
         encode_fp32_operand(tmB, d.B, d.layout, tb ? BNQ : FKQ, tb ? FKQ : BNQ);
}

int launch_fused_single(const GemmDesc &d, const CUtensorMap &tmA, const CUtensorMap &tmB,
                        cudaStream_t stream) {
  GemmParams g = gemm_params(d, 4 * d.k);
  g.num_kb = static_cast<int>((d.k + FKQ - 1) / FKQ);
  FusedOps o{};
  o.layout = d.layout;
  o.ta = op_trans(d.opA) ? 1 : 0;
  o.tb = op_trans(d.opB) ? 1 : 0;
  o.conj_a = op_conj(d.opA) ? 0xEu : 0u;
  o.conj_b = op_conj(d.opB) ? 0xEu : 0u;
  const int64_t tiles = static_cast<int64_t>(g.num_mt) * g.num_nt;
  if (tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  int rc = set_smem(fused_kernel<SplitErr, false>, kFusedSmemBytes);
  if (rc) return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = static_cast<int>(std::min<int64_t>(tiles, sms));
  fused_kernel<SplitErr, false><<<grid, kFusedThreads, kFusedSmemBytes, stream>>>(
      tmA, tmB, g, o, nullptr, nullptr, static_cast<int>(tiles), chunk_for(g.num_kb),
      wait_limit_ns());
  return launch_status();
}

// K split: P = sum over z of the FP32 partial products (in FP64, z
// ascending), then C <- alpha P + beta C with left products in FP64 and one
// rounding to float; beta == 0 does not read C.
template <int LAYOUT>
__global__ void __launch_bounds__(256)
    split_reduce_kernel(const float *__restrict__ part, int ksplit, int64_t m, int64_t n,
                        float *C, int64_t ldc, int64_t psC, double a0, double a1, double a2,
                        double a3, double b0, double b1, double b2, double b3, int beta_zero) {
  const double al[4] = {a0, a1, a2, a3}, be[4] = {b0, b1, b2, b3};
  const int64_t total = m * n, slab = total * 4;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double P[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int z = 0; z < ksplit; ++z) {
      const float4 v = *reinterpret_cast<const float4 *>(part + z * slab + 4 * e);
      P[0] += v.x;
      P[1] += v.y;
      P[2] += v.z;
      P[3] += v.w;
    }
    const int64_t i = e % m, j = e / m;
    float *q[4];
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
      *q[cc] = static_cast<float>(v);
    }
  }
}

// K shares of a single problem (one CTA per SM, tiles of BM x BNQ
// quaternions): when C has fewer than 8 waves of tiles, the fewest shares s in
// [2, 256] whose tiles x s CTAs fill their waves to within 2 % of the best s,
// with at least 64 k-blocks (512 quaternion k) per share, if the best beats
// s = 1 by 5 % and s = 1 keeps at most half of the SMs busy.  Plain products only (no triangle, k-range or turned-around
// problem).  1: no split.
int split_ksplit(const GemmDesc &d, int sms) {
  if (d.tri || d.krange || d.swap || d.m <= 0 || d.n <= 0 || d.k <= 0) return 1;
  const int64_t tiles = ((d.m + BM - 1) / BM) * ((d.n + BNQ - 1) / BNQ);
  const int64_t slots = sms;
  if (tiles >= 8 * slots) return 1;
  const int64_t num_kb = (d.kwidth * d.k + BK - 1) / BK;
  const int64_t smax = std::min<int64_t>(256, num_kb / 64);
  auto busy = [&](int64_t s) {
    const int64_t ctas = tiles * s;
    const int64_t waves = (ctas + slots - 1) / slots;
    return static_cast<double>(ctas) / static_cast<double>(waves * slots);
  };
  // under the power cap the BF16 tensor cores gain little from more busy SMs
  // once half of them work, while the shares cost a write and a re-read
  if (busy(1) > 0.5) return 1;
  double top = busy(1);
  for (int64_t s = 2; s <= smax; ++s) top = std::max(top, busy(s));
  if (top < busy(1) + 0.05) return 1;
  for (int64_t s = 2; s <= smax; ++s)
    if (busy(s) >= top - 0.02) return static_cast<int>(s);
  return 1;
}

}  // namespace

size_t split_splitk_bytes(const GemmDesc &d) {
  if (d.k == 0 || d.m == 0 || d.n == 0) return 0;
  if (want_fused() && plain_quaternion(d)) return 0;  // the fused kernel never splits
  const int ks = split_ksplit(d, device_sms());
  return ks > 1 ? static_cast<size_t>(ks) * d.m * d.n * 16 : 0;
}

int split_workspace_bytes(const GemmDesc &d, size_t *bytes) {
  if (want_fused() && plain_quaternion(d) && d.k > 0 && d.m > 0 && d.n > 0) {
    CUtensorMap a, b;
    if (fused_maps(d, &a, &b)) {
      *bytes = 0;
      return QGEMM_SUCCESS;
    }
  }
  if (d.k == 0 || d.m == 0 || d.n == 0) {
    *bytes = 0;
    return QGEMM_SUCCESS;
  }
  *bytes = plan_for(d).total;
  return QGEMM_SUCCESS;
}

int launch_split_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (want_fused() && plain_quaternion(d)) {
    CUtensorMap fa, fb;
    std::memset(&fa, 0, sizeof(fa));
    std::memset(&fb, 0, sizeof(fb));
    if (fused_maps(d, &fa, &fb)) return launch_fused_single(d, fa, fb, stream);
  }
  const SplitPlan pl = plan_for(d);
  if (ws_bytes < pl.total || ws == nullptr) return QGEMM_ERR_WORKSPACE;
  auto *wa = static_cast<__nv_bfloat16 *>(ws);
  auto *wb = reinterpret_cast<__nv_bfloat16 *>(static_cast<unsigned char *>(ws) + pl.b_offset);
  int rc = launch_prepass(false, d.A, d.opA, d.m, d.k, pl.kp, d.kwidth, d.layout, wa,
                          d.m * pl.kp, stream);
  if (rc) return rc;
  rc = launch_prepass(true, d.B, d.opB, d.n, d.k, pl.kp, d.kwidth, d.layout, wb, 4 * d.n * pl.kp,
                      stream);
  if (rc) return rc;

  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  if (!encode_bf16_3d(&tmA, wa, pl.kp, d.m, BM) || !encode_bf16_3d(&tmB, wb, pl.kp, 4 * d.n, BN))
    return QGEMM_ERR_UNSUPPORTED;
  GemmParams g = gemm_params(d, pl.kp);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // K shares: as many as chosen for this device that fit after the plan
  int ks = split_ksplit(d, sms > 0 ? sms : 1);
  if (ks > 1) {
    const size_t per = static_cast<size_t>(d.m) * d.n * 16;
    const size_t off = (pl.total + 255) / 256 * 256;
    const int64_t fit = ws_bytes > off ? static_cast<int64_t>((ws_bytes - off) / per) : 0;
    if (fit < ks) ks = static_cast<int>(fit);
    if (ks > 1) {
      g.ksplit = ks;
      g.part = reinterpret_cast<float *>(static_cast<unsigned char *>(ws) + off);
    } else {
      ks = 1;
    }
  }
  const int64_t tiles = static_cast<int64_t>(g.num_mt) * g.num_nt * ks;
  if (tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  rc = set_smem(gemm_kernel<SplitErr, false>, kSmemBytes);
  if (rc) return rc;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, sms));
  gemm_kernel<SplitErr, false><<<grid, kThreads, kSmemBytes, stream>>>(
      tmA, tmB, g, nullptr, nullptr, static_cast<int>(tiles), chunk_for(g.num_kb),
      wait_limit_ns());
  rc = launch_status();
  if (rc || ks == 1) return rc;
  const int64_t total = d.m * d.n;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152LL * 16);
  const double *al = d.alpha, *be = d.beta;
  float *C = static_cast<float *>(d.C);
  if (d.layout == QGEMM_INTERLEAVED)
    split_reduce_kernel<QGEMM_INTERLEAVED><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        g.part, ks, d.m, d.n, C, d.ldc, d.psc, al[0], al[1], al[2], al[3], be[0], be[1], be[2],
        be[3], d.beta_zero ? 1 : 0);
  else
    split_reduce_kernel<QGEMM_SPLIT_PLANES><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        g.part, ks, d.m, d.n, C, d.ldc, d.psc, al[0], al[1], al[2], al[3], be[0], be[1], be[2],
        be[3], d.beta_zero ? 1 : 0);
  return launch_status();
}

template <int PN, bool FILL>
int probe_tcgen05_shape(double seconds, double *tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 1024 + kATermBytes + PN * BK * 2;
  int rc = set_smem(tc_probe_kernel<PN, FILL>, smem);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 1024;
  float ms = 0.f;
  rc = QGEMM_SUCCESS;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    tc_probe_kernel<PN, FILL><<<sms, 128, smem, stream>>>(iters, wait_limit_ns());
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = QGEMM_ERR_CUDA;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 0.5 * seconds * 1e3) break;
    double scale = (seconds * 1e3) / (ms > 0.01 ? ms : 0.01);
    if (scale > 64) scale = 64;
    iters = static_cast<int>(iters * scale);
    if (iters > (1 << 26)) iters = 1 << 26;
  }
  if (rc == QGEMM_SUCCESS && cudaGetLastError() != cudaSuccess) rc = QGEMM_ERR_CUDA;
  if (rc == QGEMM_SUCCESS)
    *tflops = 2.0 * BM * PN * 16 * 2.0 * iters * sms / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int probe_tcgen05_bf16(int which, double seconds, double *tflops, cudaStream_t stream) {
  switch (which) {
    case 3: return probe_tcgen05_shape<256, false>(seconds, tflops, stream);
    case 4: return probe_tcgen05_shape<256, true>(seconds, tflops, stream);
    case 5: return probe_tcgen05_shape<128, true>(seconds, tflops, stream);
    case 6: return probe_tcgen05_shape<64, true>(seconds, tflops, stream);
    default: return QGEMM_ERR_UNSUPPORTED;
  }
}

// ------------------------------------------------ fixed-scratch variant ---
// Scratch for qgemm_split_noalloc(): the split operands live in this array
// instead of a caller workspace.  Every device that loads this module holds
// it until the process exits.  Host code must not use the symbol's host-side
// stand-in as a device address; the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QGEMM_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];
}  // namespace

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this; make it before any capture).
int noalloc_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return QGEMM_ERR_NO_DEVICE;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return QGEMM_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return QGEMM_SUCCESS;
}

int split_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_split_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_split_error, &z, sizeof(int));
  return v;
}

}  // namespace qg
