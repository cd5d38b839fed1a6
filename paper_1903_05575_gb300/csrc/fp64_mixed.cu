// FP64 DMMA path of mixed-type products (qgemm_mixed): the quaternion tile
// code of fp64_tile.cuh with a complex or real right factor (WB = 2 or 1
// components per element).  b^j = 0 for j >= WB, so each DMMA m16n8k4 spans
// 4 / WB values of kappa instead of the 4 components of one: half (a
// quarter) of the DMMAs of the quaternion product.  A complex or real LEFT
// factor is handled by the caller through (AB)^H = B^H A^H (the tile stores
// C = conj(D)^T).
#include <cstring>

#include "fp64_tile.cuh"

namespace qg {

__device__ int g_fp64m_error;

bool encode_fp64_operand(CUtensorMap *map, const MatView &v, int layout, int R, int CC);
fp64::Operands fp64_operands(const GemmDesc &d);

namespace {

using fp64::kBKQ;
using fp64::kSmemBytes;
using fp64::kStages;
using fp64::kThreads;
constexpr int kGroupM = 16;

struct MixedArgs {
  fp64::Operands op;
  uint64_t limit_ns;
};

template <int LAYOUT, bool TA, bool TB, int BMQ, int BNQ, int WB>
__global__ void __launch_bounds__(kThreads)
    fp64_mixed_kernel(const __grid_constant__ CUtensorMap tmA, const MixedArgs p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *sA = reinterpret_cast<double *>(smem_raw);
  double *sB = sA + kStages * fp64::kMaxTileElems;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kStages * fp64::kMaxTileElems);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
    if (p.op.tmaA) tma_prefetch_desc(&tmA);
  }
  __syncthreads();
  const int64_t tiles_m = (p.op.m + BMQ - 1) / BMQ, tiles_n = (p.op.n + BNQ - 1) / BNQ;
  const int64_t tid_lin = static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int64_t per_group = kGroupM * tiles_n;
  const int64_t first_m = (tid_lin / per_group) * kGroupM;
  const int64_t gsize = min(tiles_m - first_m, static_cast<int64_t>(kGroupM));
  const int64_t i0 = (first_m + (tid_lin % per_group) % gsize) * BMQ;
  const int64_t n0 = ((tid_lin % per_group) / gsize) * BNQ;
  uint32_t kb_run = 0;
  fp64::tile<LAYOUT, TA, TB, BMQ, BNQ, WB>(p.op, &tmA, nullptr, sA, sB, full, kb_run, i0, n0,
                                           p.limit_ns, &g_fp64m_error);
}

template <int LAYOUT, bool TA, bool TB, int BMQ, int BNQ, int WB>
int launch_one(const CUtensorMap &ta, const MixedArgs &args, dim3 grid, cudaStream_t stream) {
  auto kern = fp64_mixed_kernel<LAYOUT, TA, TB, BMQ, BNQ, WB>;
  static bool attr_set[64];
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
  kern<<<grid, kThreads, kSmemBytes, stream>>>(ta, args);
  return launch_status();
}

template <int LAYOUT, int BMQ, int BNQ, int WB>
int launch_ops(bool ta, bool tb, const CUtensorMap &tm, const MixedArgs &a, dim3 g,
               cudaStream_t s) {
  if (!ta && !tb) return launch_one<LAYOUT, false, false, BMQ, BNQ, WB>(tm, a, g, s);
  if (!ta && tb) return launch_one<LAYOUT, false, true, BMQ, BNQ, WB>(tm, a, g, s);
  if (ta && !tb) return launch_one<LAYOUT, true, false, BMQ, BNQ, WB>(tm, a, g, s);
  return launch_one<LAYOUT, true, true, BMQ, BNQ, WB>(tm, a, g, s);
}

template <int BMQ, int BNQ, int WB>
int launch_layout(int layout, bool ta, bool tb, const CUtensorMap &tm, const MixedArgs &a,
                  dim3 g, cudaStream_t s) {
  return layout == QGEMM_INTERLEAVED ? launch_ops<0, BMQ, BNQ, WB>(ta, tb, tm, a, g, s)
                                     : launch_ops<1, BMQ, BNQ, WB>(ta, tb, tm, a, g, s);
}

}  // namespace

// d: op(A) quaternion (width 4), op(B) complex or real (width 2 or 1).
int launch_fp64_mixed(const GemmDesc &d, cudaStream_t stream) {
  if (d.A.width != 4 || (d.B.width != 2 && d.B.width != 1)) return QGEMM_ERR_UNSUPPORTED;
  MixedArgs a{};
  a.op = fp64_operands(d);
  a.limit_ns = wait_limit_ns();
  const bool ta = op_trans(d.opA), tb = op_trans(d.opB);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t big = ((d.m + 31) / 32) * ((d.n + 31) / 32);
  const bool small = big < 32LL * 2 * sms;
  const int bm = small ? 16 : 32, bn = small ? 16 : 32;
  CUtensorMap tmA;
  std::memset(&tmA, 0, sizeof(tmA));
  a.op.tmaA = encode_fp64_operand(&tmA, d.A, d.layout, ta ? kBKQ : bm, ta ? bm : kBKQ) ? 1 : 0;
  a.op.tmaB = 0;  // the narrow factor comes in by plain loads
  const int64_t gx = (d.m + bm - 1) / bm, gy = (d.n + bn - 1) / bn;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (small)
    return d.B.width == 2 ? launch_layout<16, 16, 2>(d.layout, ta, tb, tmA, a, grid, stream)
                          : launch_layout<16, 16, 1>(d.layout, ta, tb, tmA, a, grid, stream);
  return d.B.width == 2 ? launch_layout<32, 32, 2>(d.layout, ta, tb, tmA, a, grid, stream)
                        : launch_layout<32, 32, 1>(d.layout, ta, tb, tmA, a, grid, stream);
}

int fp64m_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_fp64m_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_fp64m_error, &z, sizeof(int));
  return v;
}

}  // namespace qg
