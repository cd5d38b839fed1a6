// Split-BF16 quaternion GEMM, single problem: host side of the path whose
// device code is in split_core.cuh (component planes of alpha op(A) and op(B)
// split into three BF16 terms each, six term products per plane pair on
// tcgen05, compensated TMEM drain, double-float epilogue), the tcgen05
// throughput probe, and the fixed-scratch entry point's scratch array.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

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
// Back-to-back M=128, N=PN, K=16 BF16 MMAs on fixed shared-memory tiles,
// one CTA per SM: the tensor-pipe throughput of one instruction shape.  Each
// k-step issues NB MMAs that share one A tile and read NB different B tiles
// (accumulator b % 4); with COLLECT the A tile is loaded into the tensor
// core's operand collector by the first of them and reused by the rest
// (.collector::a::fill / use / lastuse), so shared memory supplies A once per
// NB MMAs.  FILL puts integer values in [-127, 127] in the tiles (as the
// GEMMs see), else zeros (lower power, so higher clocks).
// Probe tiles: K-major rows of 32 BF16 (64-byte swizzle), two K = 16 steps.
constexpr int kProbeK = 32;
constexpr uint32_t kProbeABytes = BM * kProbeK * 2;  // 8 KB

template <int PN, bool FILL, int NB, bool COLLECT>
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(int iters, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *buf = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  constexpr int kTiles = NB < 4 ? NB : 4;  // distinct B tiles in shared memory
  constexpr uint32_t kBBytes = PN * kProbeK * 2;
  constexpr uint32_t kCols = (kTiles * PN) < 32 ? 32 : (kTiles * PN);
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < static_cast<int>((kProbeABytes + kTiles * kBBytes) / 4);
       i += blockDim.x) {
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
  if (warp == 0) tmem_alloc(&tbase, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0 && elect_one()) {
    constexpr uint32_t idesc = idesc_bf16(BM, PN);
    const uint32_t sa = smem_u32(buf), sb = sa + kProbeABytes;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ad = smem_desc_sw64(sa + ks * 32);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint32_t d = tbase + (b % kTiles) * PN;
          const uint64_t bd = smem_desc_sw64(sb + (b % kTiles) * kBBytes + ks * 32);
          const uint32_t acc = (it | ks) ? 1u : 0u;
          if (!COLLECT || NB == 1)
            umma_bf16(d, ad, bd, idesc, acc);
          else if (b == 0)
            umma_bf16_fill(d, ad, bd, idesc, acc);
          else if (b == NB - 1)
            umma_bf16_lastuse(d, ad, bd, idesc, acc);
          else
            umma_bf16_use(d, ad, bd, idesc, acc);
        }
      }
    }
    umma_commit(&bar);
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicCAS(&g_split_error, 0, QGEMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, kCols);
  }
}

// Plane-pattern probe: per iteration the 16 (p, j) products of one stage at
// N = 64, in sign groups of one A slice and two B slices sharing the
// collector (as the GEMM issues them).  RB: bytes per operand row.  RB = 32:
// four A and four B tiles of 32-byte rows (32-byte swizzle); RB = 128: one A
// and one B tile whose 128-byte rows hold the four planes side by side
// (128-byte swizzle), a plane selected by a 32-byte start offset.
template <int RB>
__global__ void __launch_bounds__(128, 1) tc_plane_probe_kernel(int iters, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *buf = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  constexpr uint32_t kABytes = 4 * BM * 32, kBBytes = 4 * 64 * 32;  // four planes each
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < static_cast<int>((kABytes + kBBytes) / 4); i += blockDim.x) {
    const uint32_t h0 = (2u * i + 1u) * 2654435761u, h1 = (2u * i + 2u) * 2654435761u;
    const float f0 = static_cast<float>(static_cast<int>((h0 >> 16) % 255u) - 127);
    const float f1 = static_cast<float>(static_cast<int>((h1 >> 16) % 255u) - 127);
    reinterpret_cast<uint32_t *>(buf)[i] = (__float_as_uint(f0) >> 16) | (__float_as_uint(f1) & 0xffff0000u);
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tbase, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0 && elect_one()) {
    constexpr uint32_t idesc = idesc_bf16(BM, 64);
    const uint32_t sa = smem_u32(buf), sb = sa + kABytes;
    auto desc = [&](uint32_t tile, int rows, int plane) -> uint64_t {
      uint64_t d = 0;
      const uint32_t addr = RB == 32 ? tile + plane * rows * 32 : tile + plane * 32;
      d |= static_cast<uint64_t>((addr >> 4) & 0x3FFF);
      d |= static_cast<uint64_t>(1) << 16;
      d |= static_cast<uint64_t>((8 * RB) >> 4) << 32;
      d |= static_cast<uint64_t>(1) << 46;
      d |= static_cast<uint64_t>(RB == 32 ? 6 : 2) << 61;
      return d;
    };
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint64_t ad = desc(sa, BM, p);
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
          const uint32_t grp = split::sign_group(p, sg);
          if (grp == 0) continue;
          const int j0 = split::low_bit(grp), j1 = split::high_bit(grp);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (!((grp >> j) & 1u)) continue;
            const uint64_t bd = desc(sb, 64, j);
            const uint32_t d = tbase + (p ^ j) * 64;
            const uint32_t acc = it ? 1u : 0u;
            const uint32_t id = idesc | (sg ? split::kNegB : 0u);
            if (j0 == j1) umma_bf16(d, ad, bd, id, acc);
            else if (j == j0) umma_bf16_fill(d, ad, bd, id, acc);
            else if (j == j1) umma_bf16_lastuse(d, ad, bd, id, acc);
            else umma_bf16_use(d, ad, bd, id, acc);
          }
        }
      }
    }
    umma_commit(&bar);
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicCAS(&g_split_error, 0, QGEMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 256);
  }
}

// Alternative MMA orders of one stage for the stage probe (4 x 4 planes):
// 1 the natural order (A term outer: hh hm hl, mh mm, lh) in (term, plane,
// sign) collector groups; 2 the GEMM's order without the collector; 3 the
// GEMM's passes with planes j outer and B terms inner in each group; 4 only
// the hh products, six times (the plane pattern within the stage layout).
template <int ORDER>
__device__ __forceinline__ void issue_stage_alt(uint32_t d0, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc_n) {
  constexpr int kPassTa[6] = {0, 1, 2, 0, 0, 0};
  constexpr int kPassTb0[6] = {0, 0, 0, 0, 0, 0};
  constexpr int kPassTb1[6] = {2, 1, 0, 0, 0, 0};
  constexpr int kGemmTa[4] = {2, 1, 0, 0};
  constexpr int kGemmTb0[4] = {0, 0, 1, 0};
  constexpr int kGemmTb1[4] = {0, 1, 2, 0};
  constexpr int npass = ORDER == 1 ? 3 : (ORDER == 4 ? 6 : 4);
#pragma unroll
  for (int pass = 0; pass < npass; ++pass) {
    const int ta = ORDER == 1 ? kPassTa[pass] : (ORDER == 4 ? 0 : kGemmTa[pass]);
    const int tb0 = ORDER == 1 ? kPassTb0[pass] : (ORDER == 4 ? 0 : kGemmTb0[pass]);
    const int tb1 = ORDER == 1 ? kPassTb1[pass] : (ORDER == 4 ? 0 : kGemmTb1[pass]);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint64_t ad = adesc + (((ta * 4 + p) * kAPlaneBytes) >> 4);
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const uint32_t grp = sign_group(p, sg);
        if (grp == 0) continue;
        const int jf = low_bit(grp), jl = high_bit(grp);
        const uint32_t id = idesc_n | (sg ? kNegB : 0u);
#pragma unroll
        for (int o = 0; o < 3 * 4; ++o) {
          const int tb = ORDER == 3 ? tb0 + o % 3 : tb0 + o / 4;
          const int j = ORDER == 3 ? o / 3 : o % 4;
          if (tb > tb1 || j > 3 || !((grp >> j) & 1u)) continue;
          const uint64_t bd = bdesc + (((tb * 4 + j) * kBPlaneBytes) >> 4);
          const uint32_t d = d0 + (p ^ j) * BNQ;
          const bool first = ORDER == 3 ? (j == jf && tb == tb0) : (tb == tb0 && j == jf);
          const bool last = ORDER == 3 ? (j == jl && tb == tb1) : (tb == tb1 && j == jl);
          if (ORDER == 2 || (first && last))
            umma_bf16(d, ad, bd, id, 1u);
          else if (first)
            umma_bf16_fill(d, ad, bd, id, 1u);
          else if (last)
            umma_bf16_lastuse(d, ad, bd, id, 1u);
          else
            umma_bf16_use(d, ad, bd, id, 1u);
        }
      }
    }
  }
}

// Stage probe: the GEMM's own MMA stream (issue_stage<4, 4>: 96 MMAs per
// 16-kappa stage) over three stage slots of the ring and the two TMEM
// accumulator sets, one commit per stage; with THROTTLE the issuer also waits
// for the commit two stages back before reusing an accumulator set, as the
// GEMM waits for the drain.  No TMA, no drain: the ceiling of the MMA issue.
template <bool THROTTLE, int ORDER>
__global__ void __launch_bounds__(128, 1) tc_stage_probe_kernel(int iters, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *buf = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  __shared__ uint64_t bar[2], done;
  __shared__ uint32_t tbase;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < static_cast<int>(STAGES * kStageBytes / 4); i += blockDim.x) {
    const uint32_t h0 = (2u * i + 1u) * 2654435761u, h1 = (2u * i + 2u) * 2654435761u;
    const float f0 = static_cast<float>(static_cast<int>((h0 >> 16) % 255u) - 127);
    const float f1 = static_cast<float>(static_cast<int>((h1 >> 16) % 255u) - 127);
    reinterpret_cast<uint32_t *>(buf)[i] = (__float_as_uint(f0) >> 16) | (__float_as_uint(f1) & 0xffff0000u);
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&done, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tbase, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0 && elect_one()) {
    const uint32_t idesc = idesc_bf16(BM, BNQ);
    const uint32_t ring = smem_u32(buf);
    bool ok = true;
    for (int it = 0; it < iters && ok; ++it) {
      const int b = it & 1;
      if (THROTTLE && it >= 2) {
        ok = mbar_wait_bounded(&bar[b], ((it - 2) >> 1) & 1, limit_ns);
        tc_fence_after();
      }
      const uint32_t sa = ring + (it % STAGES) * kStageBytes;
      if (ORDER == 0)
        issue_stage<4, 4>(tbase + b * kBufCols, smem_desc_sw32(sa), smem_desc_sw32(sa + kStageA),
                          idesc, it >= 2);
      else
        issue_stage_alt<ORDER>(tbase + b * kBufCols, smem_desc_sw32(sa),
                               smem_desc_sw32(sa + kStageA), idesc);
      umma_commit(&bar[b]);
    }
    // every MMA issued by this thread completes before TMEM is released
    umma_commit(&done);
    if (!mbar_wait_bounded(&done, 0, limit_ns) || !ok) atomicCAS(&g_split_error, 0, QGEMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, kTmemCols);
  }
}

// Pipeline probe: the GEMM's MMA stream inside the GEMM's warp roles, without
// data movement or drain work.  MODE 1: a producer warp and the MMA warp pass
// the three ring stages through full / empty barriers (the producer arrives
// instead of copying); MODE 2: also eight drain warps that take each chunk's
// accumulator set (accfull) and hand it back (accempty) without reading it.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) tc_pipe_probe_kernel(int iters, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *ring = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  SmemCtl *ctl = reinterpret_cast<SmemCtl *>(ring + STAGES * kStageBytes);
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < static_cast<int>(STAGES * kStageBytes / 4); i += blockDim.x) {
    const uint32_t h0 = (2u * i + 1u) * 2654435761u, h1 = (2u * i + 2u) * 2654435761u;
    const float f0 = static_cast<float>(static_cast<int>((h0 >> 16) % 255u) - 127);
    const float f1 = static_cast<float>(static_cast<int>((h1 >> 16) % 255u) - 127);
    reinterpret_cast<uint32_t *>(ring)[i] = (__float_as_uint(f0) >> 16) | (__float_as_uint(f1) & 0xffff0000u);
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < STAGES; ++s2) {
      mbar_init(&ctl->full[s2], 1);
      mbar_init(&ctl->empty[s2], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->accfull[b], 1);
      mbar_init(&ctl->accempty[b], kEpiWarps);
    }
    mbar_init(&ctl->done, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem_base, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  if (warp == 0) {
    if (elect_one()) {
      for (int s_run = 0; s_run < iters; ++s_run) {
        const int st = s_run % STAGES;
        if (!wait_phase(&ctl->empty[st], ((s_run / STAGES) & 1) ^ 1, limit_ns, ctl)) {
          set_abort<SplitErr>(ctl);
          break;
        }
        mbar_arrive(&ctl->full[st]);
      }
    }
  } else if (warp == 1) {
    if (elect_one()) {
      const uint32_t idesc = idesc_bf16(BM, BNQ);
      const uint32_t ring_addr = smem_u32(ring);
      for (int s_run = 0; s_run < iters; ++s_run) {
        const int st = s_run % STAGES, b = s_run & 1;
        if (MODE == 2) {
          if (!wait_phase(&ctl->accempty[b], ((s_run >> 1) & 1) ^ 1, limit_ns, ctl)) {
            set_abort<SplitErr>(ctl);
            break;
          }
          tc_fence_after();
        }
        if (!wait_phase(&ctl->full[st], (s_run / STAGES) & 1, limit_ns, ctl)) {
          set_abort<SplitErr>(ctl);
          break;
        }
        tc_fence_after();
        const uint32_t sa = ring_addr + st * kStageBytes;
        issue_stage<4, 4>(tmem + b * kBufCols, smem_desc_sw32(sa), smem_desc_sw32(sa + kStageA),
                          idesc, s_run >= 2);
        umma_commit(&ctl->empty[st]);
        if (MODE == 2) umma_commit(&ctl->accfull[b]);
      }
      umma_commit(&ctl->done);
      mbar_wait_bounded(&ctl->done, 0, limit_ns);
    }
  } else if (warp >= 4 && MODE == 2) {
    const int lane = threadIdx.x & 31;
    for (int c_run = 0; c_run < iters; ++c_run) {
      const int b = c_run & 1;
      if (!wait_phase(&ctl->accfull[b], (c_run >> 1) & 1, limit_ns, ctl)) {
        set_abort<SplitErr>(ctl);
        break;
      }
      tc_fence_after();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->accempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------- host side ---
struct SplitPlan {
  int64_t kp;           // kappa pitch of the split operands (multiple of 8)
  int pa, pb;           // planes of A' (after alpha) and B'
  int smode;            // how the A pre-pass applies alpha
  size_t a_bytes, b_bytes, b_offset, total;
};

// Planes of alpha op(A) and the pre-pass mode: alpha = 1 is not applied, a
// real alpha keeps op(A)'s planes, a complex alpha keeps a complex op(A)
// complex; otherwise the product is a full quaternion.
int a_planes(const GemmDesc &d, int *smode) {
  const double *al = d.alpha;
  const bool real = al[1] == 0.0 && al[2] == 0.0 && al[3] == 0.0;
  const bool cplx = al[2] == 0.0 && al[3] == 0.0;
  *smode = (real && al[0] == 1.0) ? kScaleNone : (real ? kScaleReal : kScaleLeft);
  if (real) return d.A.width;
  if (cplx && d.A.width <= 2) return 2;
  return 4;
}

SplitPlan plan_for(const GemmDesc &d) {
  SplitPlan s;
  s.kp = (d.k + 7) / 8 * 8;
  s.pa = a_planes(d, &s.smode);
  s.pb = d.B.width;
  s.a_bytes = static_cast<size_t>(TERMS) * s.pa * d.m * s.kp * 2;
  s.b_bytes = static_cast<size_t>(TERMS) * s.pb * d.n * s.kp * 2;
  s.b_offset = (s.a_bytes + 1023) & ~static_cast<size_t>(1023);
  s.total = s.b_offset + s.b_bytes;
  return s;
}

void to_double_float(const double *x, float *hi, float *lo) {
  for (int s = 0; s < 4; ++s) {
    hi[s] = static_cast<float>(x[s]);
    lo[s] = static_cast<float>(x[s] - static_cast<double>(hi[s]));
  }
}

GemmParams gemm_params(const GemmDesc &d, const SplitPlan &pl) {
  GemmParams g{};
  g.m = d.m;
  g.n = d.n;
  g.num_kb = static_cast<int>(d.k > 0 ? (d.k + KQ - 1) / KQ : 0);
  g.num_mt = static_cast<int>((d.m + BM - 1) / BM);
  g.num_nt = static_cast<int>((d.n + BNQ - 1) / BNQ);
  g.pa = pl.pa;
  g.pb = pl.pb;
  g.C = static_cast<float *>(d.C);
  g.ldc = d.ldc;
  g.psC = d.psc;
  g.layout = d.layout;
  g.beta_zero = d.beta_zero ? 1 : 0;
  g.beta_real = (d.beta[1] == 0.0 && d.beta[2] == 0.0 && d.beta[3] == 0.0) ? 1 : 0;
  g.tri = d.tri;
  g.krange = d.krange;
  g.swap = d.swap;
  g.c_vec4 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
  set_beta(g, d.beta);
  return g;
}

}  // namespace

// 4-D tensor map of split operand planes: (kappa < kq, rows, planes, 3 terms),
// kappa pitch kp, boxes of KQ kappa x box_rows rows x all planes x all terms,
// 32-byte swizzle (the layout the MMA descriptors address).  Shared with the
// grouped path.
bool encode_split_planes(CUtensorMap *map, const void *base, int64_t kq, int64_t kp,
                         int64_t rows, int planes, int box_rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc || rows <= 0 || kq <= 0) return false;
  if (rows >= (1ll << 32) || kq >= (1ll << 32)) return false;
  cuuint64_t dims[4] = {static_cast<cuuint64_t>(kq), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(planes), TERMS};
  const cuuint64_t row = static_cast<cuuint64_t>(kp) * 2;
  cuuint64_t strides[3] = {row, row * static_cast<cuuint64_t>(rows),
                           row * static_cast<cuuint64_t>(rows) * static_cast<cuuint64_t>(planes)};
  if (strides[2] >= (1ull << 40)) return false;
  cuuint32_t box[4] = {KQ, static_cast<cuuint32_t>(box_rows), static_cast<cuuint32_t>(planes),
                       TERMS};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// Raises the dynamic shared-memory limit of one kernel, once per (kernel,
// device).  Keyed by the kernel's address: kernels of one signature share a
// type, so a per-type flag would skip all but the first of them.
template <typename K>
int set_smem(K kern, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::pair<const void *, int> key(reinterpret_cast<const void *>(kern), dev);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(key)) return QGEMM_SUCCESS;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(bytes)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  done.insert(key);
  return QGEMM_SUCCESS;
}

int launch_prepass(bool is_b, const MatView &v, int op, int64_t rows, int64_t kq, int64_t kp,
                   int planes, int smode, const double *scalar, int layout, __nv_bfloat16 *out,
                   cudaStream_t stream) {
  PrepArgs a{};
  a.X = static_cast<const float *>(v.ptr);
  a.ld = v.ld;
  a.ps = v.ps;
  a.rows = rows;
  a.kq = kq;
  a.kp = kp;
  a.out = out;
  a.layout = layout;
  // A: op row i is the stored row for N/C; B: op row n is the stored row for T/H
  a.row_contig = is_b ? (op_trans(op) ? 1 : 0) : (op_trans(op) ? 0 : 1);
  a.conj = op_conj(op) ? 1 : 0;
  a.width = v.width;
  a.planes = planes;
  a.smode = smode;
  if (scalar) to_double_float(scalar, a.s_hi, a.s_lo);
  const int64_t gx = (rows + 31) / 32, gy = (kq + 31) / 32;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (is_b)
    split_prepass_kernel<true><<<grid, 256, 0, stream>>>(a);
  else
    split_prepass_kernel<false><<<grid, 256, 0, stream>>>(a);
  return launch_status();
}

// K split: P = sum over z of the FP32 partial products (in FP64, z
// ascending), then C <- P + beta C with the left product in FP64 and one
// rounding to float (alpha was applied to op(A) by the pre-pass); beta == 0
// does not read C.
template <int LAYOUT>
__global__ void __launch_bounds__(256)
    split_reduce_kernel(const float *__restrict__ part, int ksplit, int64_t m, int64_t n,
                        float *C, int64_t ldc, int64_t psC, double b0, double b1, double b2,
                        double b3, int beta_zero) {
  const double be[4] = {b0, b1, b2, b3};
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
      double v = P[cc];
      if (!beta_zero) {
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
          const int s = cc ^ j2;
          const double sg = basis_sign(s, j2) < 0 ? -1.0 : 1.0;
          v = fma(sg * be[s], c[j2], v);
        }
      }
      *q[cc] = static_cast<float>(v);
    }
  }
}

// K shares of a single problem (one CTA per SM, tiles of BM x BNQ
// quaternions): when C has fewer than 8 waves of tiles, the fewest shares s in
// [2, 256] whose tiles x s CTAs fill their waves to within 2 % of the best s,
// with at least 32 stages (512 quaternion k) per share, if the best beats s = 1
// by 5 % and s = 1 keeps at most half of the SMs busy.  Plain products only
// (no triangle, k-range or turned-around problem).  1: no split.
int split_ksplit(const GemmDesc &d, int sms) {
  if (d.tri || d.krange || d.swap || d.m <= 0 || d.n <= 0 || d.k <= 0) return 1;
  const int64_t tiles = ((d.m + BM - 1) / BM) * ((d.n + BNQ - 1) / BNQ);
  const int64_t slots = sms;
  if (tiles >= 8 * slots) return 1;
  const int64_t stages = (d.k + KQ - 1) / KQ;
  const int64_t smax = std::min<int64_t>(256, stages / 32);
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

// One-shot fault injection for the bounded-wait test (qgemm_debug_arm_fault).
std::atomic<int> g_debug_skip{0};
std::atomic<uint64_t> g_debug_limit{0};

}  // namespace

void split_arm_fault(int stage, uint64_t limit_ns) {
  g_debug_limit.store(limit_ns);
  g_debug_skip.store(stage + 1);
}

size_t split_splitk_bytes(const GemmDesc &d) {
  if (d.k == 0 || d.m == 0 || d.n == 0) return 0;
  const int ks = split_ksplit(d, device_sms());
  return ks > 1 ? static_cast<size_t>(ks) * d.m * d.n * 16 : 0;
}

int split_workspace_bytes(const GemmDesc &d, size_t *bytes) {
  if (d.k == 0 || d.m == 0 || d.n == 0) {
    *bytes = 0;
    return QGEMM_SUCCESS;
  }
  if (d.k > kMaxK) return QGEMM_ERR_UNSUPPORTED;
  *bytes = plan_for(d).total;
  return QGEMM_SUCCESS;
}

int launch_split_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (d.k > kMaxK) return QGEMM_ERR_UNSUPPORTED;
  const SplitPlan pl = plan_for(d);
  if (ws_bytes < pl.total || ws == nullptr) return QGEMM_ERR_WORKSPACE;
  auto *wa = static_cast<__nv_bfloat16 *>(ws);
  auto *wb = reinterpret_cast<__nv_bfloat16 *>(static_cast<unsigned char *>(ws) + pl.b_offset);
  int rc = launch_prepass(false, d.A, d.opA, d.m, d.k, pl.kp, pl.pa, pl.smode, d.alpha, d.layout,
                          wa, stream);
  if (rc) return rc;
  rc = launch_prepass(true, d.B, d.opB, d.n, d.k, pl.kp, pl.pb, kScaleNone, nullptr, d.layout, wb,
                      stream);
  if (rc) return rc;

  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  if (!encode_split_planes(&tmA, wa, d.k, pl.kp, d.m, pl.pa, BM) ||
      !encode_split_planes(&tmB, wb, d.k, pl.kp, d.n, pl.pb, BNQ))
    return QGEMM_ERR_UNSUPPORTED;
  GemmParams g = gemm_params(d, pl);
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
  const int skip = g_debug_skip.exchange(0);
  const uint64_t limit = skip ? g_debug_limit.load() : wait_limit_ns();
  gemm_kernel<SplitErr, false><<<grid, kThreads, kSmemBytes, stream>>>(
      tmA, tmB, g, nullptr, nullptr, static_cast<int>(tiles), limit, skip);
  rc = launch_status();
  if (rc || ks == 1) return rc;
  const int64_t total = d.m * d.n;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152LL * 16);
  const double *be = d.beta;
  float *C = static_cast<float *>(d.C);
  if (d.layout == QGEMM_INTERLEAVED)
    split_reduce_kernel<QGEMM_INTERLEAVED><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        g.part, ks, d.m, d.n, C, d.ldc, d.psc, be[0], be[1], be[2], be[3], d.beta_zero ? 1 : 0);
  else
    split_reduce_kernel<QGEMM_SPLIT_PLANES><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        g.part, ks, d.m, d.n, C, d.ldc, d.psc, be[0], be[1], be[2], be[3], d.beta_zero ? 1 : 0);
  return launch_status();
}

template <int PN, bool FILL, int NB, bool COLLECT>
int probe_tcgen05_shape(double seconds, double *tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  constexpr int kTiles = NB < 4 ? NB : 4;
  const size_t smem = 1024 + kProbeABytes + kTiles * PN * kProbeK * 2;
  int rc = set_smem(tc_probe_kernel<PN, FILL, NB, COLLECT>, smem);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 1024 / NB;
  float ms = 0.f;
  rc = QGEMM_SUCCESS;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    tc_probe_kernel<PN, FILL, NB, COLLECT><<<sms, 128, smem, stream>>>(iters, wait_limit_ns());
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
    *tflops = 2.0 * BM * PN * 16 * 2.0 * NB * iters * sms / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// which: 3 N=256 zero tiles; 4 N=256, 5 N=128, 6 N=64 (one B tile, integer
// data); 8 N=64 with 4 B tiles per A tile and the A collector; 9 the same
// without the collector; 10 N=32, 4 B tiles, collector; 11 N=128, 2 B tiles,
// collector; 12 N=64, 12 MMAs per A tile (4 B tiles, 3 passes), collector.
template <int RB>
int probe_plane_pattern(double seconds, double *tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 1024 + 4 * BM * 32 + 4 * 64 * 32;
  int rc = set_smem(tc_plane_probe_kernel<RB>, smem);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 64;
  float ms = 0.f;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    tc_plane_probe_kernel<RB><<<sms, 128, smem, stream>>>(iters, wait_limit_ns());
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
    if (iters > (1 << 24)) iters = 1 << 24;
  }
  if (rc == QGEMM_SUCCESS && cudaGetLastError() != cudaSuccess) rc = QGEMM_ERR_CUDA;
  if (rc == QGEMM_SUCCESS) *tflops = 2.0 * BM * 64 * 16 * 16.0 * iters * sms / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

template <bool THROTTLE, int ORDER>
int probe_stage_pattern(double seconds, double *tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 1024 + STAGES * kStageBytes;
  int rc = set_smem(tc_stage_probe_kernel<THROTTLE, ORDER>, smem);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 64;
  float ms = 0.f;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    tc_stage_probe_kernel<THROTTLE, ORDER><<<sms, 128, smem, stream>>>(iters, wait_limit_ns());
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
    if (iters > (1 << 22)) iters = 1 << 22;
  }
  if (rc == QGEMM_SUCCESS && cudaGetLastError() != cudaSuccess) rc = QGEMM_ERR_CUDA;
  if (rc == QGEMM_SUCCESS) *tflops = 2.0 * BM * BNQ * KQ * 96.0 * iters * sms / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

template <int MODE>
int probe_pipe_pattern(double seconds, double *tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int rc = set_smem(tc_pipe_probe_kernel<MODE>, kSmemBytes);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 64;
  float ms = 0.f;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    tc_pipe_probe_kernel<MODE><<<sms, kThreads, kSmemBytes, stream>>>(iters, wait_limit_ns());
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
    if (iters > (1 << 22)) iters = 1 << 22;
  }
  if (rc == QGEMM_SUCCESS && cudaGetLastError() != cudaSuccess) rc = QGEMM_ERR_CUDA;
  if (rc == QGEMM_SUCCESS) *tflops = 2.0 * BM * BNQ * KQ * 96.0 * iters * sms / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int probe_tcgen05_bf16(int which, double seconds, double *tflops, cudaStream_t stream) {
  switch (which) {
    case 21: return probe_pipe_pattern<1>(seconds, tflops, stream);
    case 22: return probe_pipe_pattern<2>(seconds, tflops, stream);
    case 15: return probe_stage_pattern<false, 0>(seconds, tflops, stream);
    case 16: return probe_stage_pattern<true, 0>(seconds, tflops, stream);
    case 17: return probe_stage_pattern<false, 1>(seconds, tflops, stream);
    case 18: return probe_stage_pattern<false, 2>(seconds, tflops, stream);
    case 19: return probe_stage_pattern<false, 3>(seconds, tflops, stream);
    case 20: return probe_stage_pattern<false, 4>(seconds, tflops, stream);
    case 13: return probe_plane_pattern<32>(seconds, tflops, stream);
    case 14: return probe_plane_pattern<128>(seconds, tflops, stream);
    case 3: return probe_tcgen05_shape<256, false, 1, false>(seconds, tflops, stream);
    case 4: return probe_tcgen05_shape<256, true, 1, false>(seconds, tflops, stream);
    case 5: return probe_tcgen05_shape<128, true, 1, false>(seconds, tflops, stream);
    case 6: return probe_tcgen05_shape<64, true, 1, false>(seconds, tflops, stream);
    case 8: return probe_tcgen05_shape<64, true, 4, true>(seconds, tflops, stream);
    case 9: return probe_tcgen05_shape<64, true, 4, false>(seconds, tflops, stream);
    case 10: return probe_tcgen05_shape<32, true, 4, true>(seconds, tflops, stream);
    case 11: return probe_tcgen05_shape<128, true, 2, true>(seconds, tflops, stream);
    case 12: return probe_tcgen05_shape<64, true, 12, true>(seconds, tflops, stream);
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
