// FP64 quaternion GEMM on the BF16 tensor cores by exact digit slicing.
//
// Splitting.  After the error-free splitting of matrix products of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), with integer digits:
// every component of quaternion row i of op(A) is written as
//     a = 2^(e_i - 7) * sum_{t=0..5} d_t 2^(-8 t),   |d_t| <= 128 integers,
// where max_row |a| < 2^(e_i) (the digits are the balanced base-256 digits of
// round(a 2^(47 - e_i)), so the representation error is <= 2^(e_i - 48)).
// Quaternion column n of op(B) is split the same way with its own e_n.  Every
// digit is exact in BF16.
//
// Products.  In the real form of the quaternion product (split_core.cuh),
// C' = A' B', slice i of A' times slice j of B' is a matrix of integer sums of
// products |d d'| <= 2^14.  All pairs with the same level l = i + j share the
// scale 2^(-8 l), so level l accumulates in its own TMEM region (64 columns
// each, regions 0..5 side by side); one MMA of A slice i against B slices
// j..j+3 (N up to 256) feeds regions i+j..i+j+3 at once.  Levels 0..5 are kept
// (21 of the 36 slice pairs); the dropped levels are below 2^-48 of
// 2^(e_i + e_n) per real product.
//
// Exactness.  Level l sums (l + 1) pairs; over 256 real k its integer sum is
// at most 4 * 256 * 2^14 = 2^24 for l <= 3, exact in the FP32 accumulator.
// So levels 0..3 are drained every 256 real k (8 k-blocks) into a 64-bit
// integer per output, T = sum 2^(8 (3 - l)) S_l, and levels 4 and 5 (scale
// <= 2^-32, where FP32 rounding is far below the FP64 target) accumulate in
// TMEM over the whole K and are read once per tile.  The epilogue forms
// P = 2^(e_i + e_n - 38) (T + tail) and C <- alpha P + beta C in FP64.
//
// Kernel.  Persistent, warp-specialised as the split-BF16 kernel: a TMA warp
// (6 A slices 128 x 32 and 6 B slices 64 x 32 per stage, 64-byte swizzle),
// an MMA warp (8 MMAs of M = 128, N = 64..256, K = 16 per k-step), eight
// drain/epilogue warps.  One TMEM accumulator set (384 of 512 columns): the
// MMAs of the next 256-k chunk wait for the drain of levels 0..3; the
// epilogue of a tile overlaps the next tile's MMAs.  Every wait is bounded.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "split_core.cuh"

namespace qg {

__device__ int g_sliced_error;

namespace {

using split::elect_one;
using split::idesc_bf16;
using split::smem_desc_sw64;
using split::tc_fence_after;
using split::tc_fence_before;
using split::tmem_alloc;
using split::tmem_dealloc;
using split::umma_bf16;
using split::umma_commit;

constexpr int SBM = 128;        // rows of C per tile
constexpr int SBN = 64;         // real columns of C' per tile (16 quaternions)
constexpr int SBNQ = SBN / 4;
constexpr int SBK = 32;         // real k per stage
constexpr int SST = 3;          // stages
constexpr int NSL = 6;          // digit slices per operand
constexpr int kChunkKb = 8;     // k-blocks per exact chunk (256 real k)
constexpr int kDrainWarps = 8;
constexpr int kSThreads = 64 + 32 * kDrainWarps;
constexpr uint32_t kSliceA = SBM * SBK * 2;          // 8 KB
constexpr uint32_t kSliceB = SBN * SBK * 2;          // 4 KB
constexpr uint32_t kStageA = NSL * kSliceA;          // 48 KB
constexpr uint32_t kStageBytes = kStageA + NSL * kSliceB;  // 72 KB
constexpr uint32_t kTmemCols = 512;                  // 6 regions x 64 used
constexpr size_t kSmem = 1024 + SST * kStageBytes + 256;
constexpr int kGroupM = 8;
constexpr int kNonFinite = -0x40000000;              // exponent slot of a non-finite row

struct SlicedParams {
  int64_t m, n;
  int num_kb, num_mt, num_nt;
  int layout, beta_zero, tri, c_vec2;
  double *C;
  int64_t ldc, psC;
  double alpha[4], beta[4];
  const int *eA;  // per quaternion row of op(A)
  const int *eB;  // per quaternion column of op(B)
};

struct Ctl {
  uint64_t full[SST];
  uint64_t empty[SST];
  uint64_t accfull;
  uint64_t accempty;
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ void set_abort(Ctl *ctl) {
  atomicCAS(&g_sliced_error, 0, QGEMM_ERR_TIMEOUT);
  *reinterpret_cast<volatile int *>(&ctl->abort) = 1;
}
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                           Ctl *ctl) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*reinterpret_cast<volatile int *>(&ctl->abort) != 0 || globaltimer_ns() - t0 > limit_ns)
      return false;
  }
}

__device__ __forceinline__ void tile_coords(const SlicedParams &g, int t, int &mt, int &nt) {
  const int per_group = kGroupM * g.num_nt;
  const int first_m = (t / per_group) * kGroupM;
  const int gsize = min(g.num_mt - first_m, kGroupM);
  mt = first_m + (t % per_group) % gsize;
  nt = (t % per_group) / gsize;
}

__device__ __forceinline__ bool tile_skip(const SlicedParams &g, int mt, int nt) {
  if (g.tri == 1) return static_cast<int64_t>(mt) * SBM + SBM - 1 < static_cast<int64_t>(nt) * SBNQ;
  if (g.tri == 2) return static_cast<int64_t>(nt) * SBNQ + SBNQ - 1 < static_cast<int64_t>(mt) * SBM;
  return false;
}

// The 21 slice products of one k-step (16 real k) as 8 MMAs: A slice i
// against B slices j0.. (adjacent in shared memory), into level regions
// i + j0 .. (adjacent in TMEM, 64 columns each).
__device__ __forceinline__ void mma_kstep(uint32_t d, uint32_t sa, uint32_t sb, int ks,
                                          uint32_t acc03, uint32_t acc45) {
  const uint32_t ka = sa + ks * 32, kb = sb + ks * 32;
  umma_bf16(d + 0 * SBN, smem_desc_sw64(ka + 0 * kSliceA), smem_desc_sw64(kb + 0 * kSliceB),
            idesc_bf16(SBM, 4 * SBN), acc03);                                    // 00 01 02 03
  umma_bf16(d + 4 * SBN, smem_desc_sw64(ka + 0 * kSliceA), smem_desc_sw64(kb + 4 * kSliceB),
            idesc_bf16(SBM, 2 * SBN), acc45);                                    // 04 05
  umma_bf16(d + 1 * SBN, smem_desc_sw64(ka + 1 * kSliceA), smem_desc_sw64(kb + 0 * kSliceB),
            idesc_bf16(SBM, 4 * SBN), 1u);                                       // 10 11 12 13
  umma_bf16(d + 5 * SBN, smem_desc_sw64(ka + 1 * kSliceA), smem_desc_sw64(kb + 4 * kSliceB),
            idesc_bf16(SBM, 1 * SBN), 1u);                                       // 14
  umma_bf16(d + 2 * SBN, smem_desc_sw64(ka + 2 * kSliceA), smem_desc_sw64(kb + 0 * kSliceB),
            idesc_bf16(SBM, 4 * SBN), 1u);                                       // 20 21 22 23
  umma_bf16(d + 3 * SBN, smem_desc_sw64(ka + 3 * kSliceA), smem_desc_sw64(kb + 0 * kSliceB),
            idesc_bf16(SBM, 3 * SBN), 1u);                                       // 30 31 32
  umma_bf16(d + 4 * SBN, smem_desc_sw64(ka + 4 * kSliceA), smem_desc_sw64(kb + 0 * kSliceB),
            idesc_bf16(SBM, 2 * SBN), 1u);                                       // 40 41
  umma_bf16(d + 5 * SBN, smem_desc_sw64(ka + 5 * kSliceA), smem_desc_sw64(kb + 0 * kSliceB),
            idesc_bf16(SBM, 1 * SBN), 1u);                                       // 50
}

// One drain thread's epilogue: row i, quaternion columns nq0 .. nq0 + 7,
// S = T + tail (in units of 2^-24 of the level-0 digit products) for the 32
// real columns 4 (n - nq0) + c.
__device__ __forceinline__ void epilogue(const SlicedParams &g, int64_t i, int64_t nq0,
                                         const double (&S)[32]) {
  if (i >= g.m) return;
  if (g.tri == 2 && nq0 + 7 < i) return;
  const int ea = g.eA[i];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t nn = nq0 + q;
    if (nn >= g.n) continue;
    if ((g.tri == 1 && i < nn) || (g.tri == 2 && i > nn)) continue;
    const int eb = g.eB[nn];
    double P[4];
    if (ea == kNonFinite || eb == kNonFinite) {
#pragma unroll
      for (int c = 0; c < 4; ++c) P[c] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) P[c] = ldexp(S[4 * q + c], ea + eb - 38);
    }
    double cin[4] = {0.0, 0.0, 0.0, 0.0};
    double *dst0;
    if (g.layout == QGEMM_INTERLEAVED) {
      dst0 = g.C + 4 * (i + nn * g.ldc);
      if (!g.beta_zero) {
        if (g.c_vec2) {
          const double2 lo = *reinterpret_cast<const double2 *>(dst0);
          const double2 hi = *reinterpret_cast<const double2 *>(dst0 + 2);
          cin[0] = lo.x; cin[1] = lo.y; cin[2] = hi.x; cin[3] = hi.y;
        } else {
#pragma unroll
          for (int s = 0; s < 4; ++s) cin[s] = dst0[s];
        }
      }
    } else {
      dst0 = g.C + i + nn * g.ldc;
      if (!g.beta_zero) {
#pragma unroll
        for (int s = 0; s < 4; ++s) cin[s] = dst0[s * g.psC];
      }
    }
    // out = alpha P + beta C (left products): (x y)^c = sum_j sign(c^j, j) x^(c^j) y^j
    double out[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = c ^ j;
        const double a = basis_sign(s, j) < 0 ? -g.alpha[s] : g.alpha[s];
        acc = fma(a, P[j], acc);
      }
      if (!g.beta_zero) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int s = c ^ j;
          const double b = basis_sign(s, j) < 0 ? -g.beta[s] : g.beta[s];
          acc = fma(b, cin[j], acc);
        }
      }
      out[c] = acc;
    }
    if (g.tri && i == nn) out[1] = out[2] = out[3] = 0.0;  // Hermitian diagonal is real
    if (g.layout == QGEMM_INTERLEAVED) {
      if (g.c_vec2) {
        *reinterpret_cast<double2 *>(dst0) = make_double2(out[0], out[1]);
        *reinterpret_cast<double2 *>(dst0 + 2) = make_double2(out[2], out[3]);
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) dst0[s] = out[s];
      }
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) dst0[s * g.psC] = out[s];
    }
  }
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// T[off + q] += 2^SHIFT * v[q] for exact integers v[q].
template <int SHIFT>
__device__ __forceinline__ void add_level(long long (&T)[32], int off, const float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q)
    T[off + q] += static_cast<long long>(__float2int_rn(v[q])) * (1ll << SHIFT);
}

// Adds this thread's 32 columns of levels 0..3 (exact integers) to T.
__device__ __forceinline__ void drain_levels03(uint32_t base, long long (&T)[32]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float v[16];
    tmem_ld16(base + 0 * SBN + 16 * h, v);
    add_level<24>(T, 16 * h, v);
    tmem_ld16(base + 1 * SBN + 16 * h, v);
    add_level<16>(T, 16 * h, v);
    tmem_ld16(base + 2 * SBN + 16 * h, v);
    add_level<8>(T, 16 * h, v);
    tmem_ld16(base + 3 * SBN + 16 * h, v);
    add_level<0>(T, 16 * h, v);
  }
}

__global__ void __launch_bounds__(kSThreads, 1)
    sliced_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB, const SlicedParams g, int ntiles,
                       uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *ring = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  Ctl *ctl = reinterpret_cast<Ctl *>(ring + SST * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SST; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    mbar_init(&ctl->accfull, 1);
    mbar_init(&ctl->accempty, kDrainWarps);
    mbar_init(&ctl->done, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem_base, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  const int nkb = g.num_kb;
  const int nch = (nkb + kChunkKb - 1) / kChunkKb;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (elect_one()) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      uint32_t s_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int mt, nt;
        tile_coords(g, t, mt, nt);
        if (tile_skip(g, mt, nt)) continue;
        for (int kb = 0; kb < nkb; ++kb, ++s_run) {
          const int st = s_run % SST;
          if (!wait_phase(&ctl->empty[st], ((s_run / SST) & 1) ^ 1, limit_ns, ctl)) {
            set_abort(ctl);
            ok = false;
            break;
          }
          unsigned char *sa = ring + st * kStageBytes;
          mbar_arrive_expect_tx(&ctl->full[st], kStageBytes);
          tma_load_3d(sa, &tmA, &ctl->full[st], kb * SBK, mt * SBM, 0);
          tma_load_3d(sa + kStageA, &tmB, &ctl->full[st], kb * SBK, nt * SBN, 0);
        }
      }
      if (!ok) {  // let this CTA's copies in flight land before it retires
        for (uint32_t q = s_run > SST ? s_run - SST : 0; q < s_run; ++q)
          mbar_wait_bounded(&ctl->full[q % SST], (q / SST) & 1, limit_ns);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (elect_one()) {
      const uint32_t ring_addr = smem_u32(ring);
      uint32_t s_run = 0, c_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int mt, nt;
        tile_coords(g, t, mt, nt);
        if (tile_skip(g, mt, nt)) continue;
        for (int ch = 0; ch < nch && ok; ++ch, ++c_run) {
          // levels 0..3 of the previous chunk (all levels after a tile) drained
          if (!wait_phase(&ctl->accempty, (c_run & 1) ^ 1, limit_ns, ctl)) {
            set_abort(ctl);
            ok = false;
            break;
          }
          tc_fence_after();
          const int kb0 = ch * kChunkKb, kb1 = min(nkb, kb0 + kChunkKb);
          for (int kb = kb0; kb < kb1; ++kb, ++s_run) {
            const int st = s_run % SST;
            if (!wait_phase(&ctl->full[st], (s_run / SST) & 1, limit_ns, ctl)) {
              set_abort(ctl);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = ring_addr + st * kStageBytes;
            const uint32_t sb = sa + kStageA;
#pragma unroll
            for (int ks = 0; ks < SBK / 16; ++ks) {
              const bool first = kb == kb0 && ks == 0;
              mma_kstep(tmem, sa, sb, ks, first ? 0u : 1u, (first && ch == 0) ? 0u : 1u);
            }
            umma_commit(&ctl->empty[st]);  // frees the stage when these MMAs finish
          }
          if (!ok) break;
          umma_commit(&ctl->accfull);
        }
      }
      umma_commit(&ctl->done);
      mbar_wait_bounded(&ctl->done, 0, limit_ns);
    }
  } else {
    // ---------------- drain + epilogue (8 warps) ----------------
    const int ew = warp - 2;
    const int quad = warp & 3;  // TMEM lanes 32*quad .. +31 (hardware rule: warp % 4)
    const int half = ew >> 2;   // columns [32*half, 32*half + 32) of each level region
    const uint32_t base = tmem + (static_cast<uint32_t>(32 * quad) << 16) + 32 * half;
    uint32_t c_run = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int mt, nt;
      tile_coords(g, t, mt, nt);
      if (tile_skip(g, mt, nt)) continue;
      long long T[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) T[q] = 0;
      // chunks 0 .. nch-2: levels 0..3; the last chunk also levels 4 and 5
      for (int ch = 0; ch < nch - 1; ++ch, ++c_run) {
        if (!wait_phase(&ctl->accfull, c_run & 1, limit_ns, ctl)) {
          set_abort(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        drain_levels03(base, T);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->accempty);
      }
      if (!ok) break;
      if (!wait_phase(&ctl->accfull, c_run & 1, limit_ns, ctl)) {
        set_abort(ctl);
        break;
      }
      ++c_run;
      tc_fence_after();
      drain_levels03(base, T);
      double S[32];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v4[16], v5[16];
        tmem_ld16(base + 4 * SBN + 16 * h, v4);
        tmem_ld16(base + 5 * SBN + 16 * h, v5);
#pragma unroll
        for (int q = 0; q < 16; ++q)
          S[16 * h + q] = static_cast<double>(T[16 * h + q]) +
                          static_cast<double>(fmaf(v5[q], 0.00390625f, v4[q]) * 0.00390625f);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->accempty);
      epilogue(g, static_cast<int64_t>(mt) * SBM + 32 * quad + lane,
               static_cast<int64_t>(nt) * SBNQ + 8 * half, S);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------ pre-pass ---
// Largest |component| of each quaternion row (by_col = 0) or column
// (by_col = 1) of a stored matrix, as the bits of a non-negative double
// (ordered like the values; NaN above Inf), max-reduced into out[].
__global__ void __launch_bounds__(256)
    slice_max_kernel(const double *__restrict__ X, int64_t ld, int64_t ps, int64_t srows,
                     int64_t scols, int layout, int by_col, unsigned long long *out) {
  __shared__ unsigned long long red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r = static_cast<int64_t>(blockIdx.x) * 32 + tx;
  const int64_t c0 = static_cast<int64_t>(blockIdx.y) * 32;
  unsigned long long rowm = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t c = c0 + ty + 8 * s;
    unsigned long long mx = 0;
    if (r < srows && c < scols) {
#pragma unroll
      for (int comp = 0; comp < 4; ++comp) {
        const double x = layout == QGEMM_INTERLEAVED ? X[4 * (r + c * ld) + comp]
                                                     : X[r + c * ld + comp * ps];
        const unsigned long long b =
            static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
        mx = b > mx ? b : mx;
      }
    }
    if (by_col) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
      }
      if (tx == 0 && c < scols && mx != 0) atomicMax(out + c, mx);
    } else {
      rowm = mx > rowm ? mx : rowm;
    }
  }
  if (!by_col) {
    red[ty][tx] = rowm;
    __syncthreads();
    if (ty == 0) {
      unsigned long long v = red[0][tx];
#pragma unroll
      for (int w = 1; w < 8; ++w) v = red[w][tx] > v ? red[w][tx] : v;
      if (r < srows && v != 0) atomicMax(out + r, v);
    }
  }
}

// Exponent e with max < 2^e (0 for a zero row, kNonFinite for Inf or NaN).
__device__ __forceinline__ int exponent_of(unsigned long long maxbits) {
  if (maxbits >= 0x7ff0000000000000ull) return kNonFinite;
  if (maxbits == 0) return 0;
  int e = 0;
  frexp(__longlong_as_double(static_cast<long long>(maxbits)), &e);
  return e;
}

struct SliceArgs {
  const double *X;
  int64_t ld, ps;        // stored leading dimension, plane stride
  int64_t rows;          // rows of the op-matrix (m for A, n for B)
  int64_t kq;            // quaternion K
  int64_t kp;            // padded real K (multiple of SBK)
  int64_t slice_stride;  // elements between slices in the output
  __nv_bfloat16 *out;
  const unsigned long long *maxbits;  // per op row
  int *eout;                          // per op row: the exponent used
  int layout;
  int row_contig;        // stored row index == op row
  uint32_t negmask;      // bit j: negate component j (conjugation)
};

// Balanced base-256 digits of round(x) for |x| <= 2^47: x ~ sum d_t 2^(8 (5 - t)).
__device__ __forceinline__ void digits6(double x, int (&d)[NSL]) {
  long long X = __double2ll_rn(x);
#pragma unroll
  for (int t = NSL - 1; t >= 1; --t) {
    const long long lo = ((X + 128) & 255) - 128;
    d[t] = static_cast<int>(lo);
    X = (X - lo) >> 8;
  }
  d[0] = static_cast<int>(X);
}

// One 32 x 32 tile of the op-matrix (rows r, columns kappa), read coalesced
// through shared memory and written as digit slices, K-major:
//   A: A'_t[r][4 kappa + j] = d_t(a^j)
//   B: B'_t[4 r + c][4 kappa + j] = sign(j, j^c) d_t(b^(j^c))
// Columns kappa >= kq up to kp/4 are zeros (K padding).
template <bool IS_B>
__global__ void __launch_bounds__(256) slice_kernel(const SliceArgs p) {
  __shared__ double4 tile[32][33];
  __shared__ double scale1[32], scale2[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * 32;
  if (threadIdx.x < 32) {
    const int64_t r = r0 + threadIdx.x;
    int e = 0;
    if (r < p.rows) {
      e = exponent_of(p.maxbits[r]);
      if (blockIdx.y == 0) p.eout[r] = e;
    }
    // x = a 2^(47 - e) as two exact power-of-two factors (each in range)
    const int s = e == kNonFinite ? 0 : 47 - e;
    const int s1 = s > 1000 ? 1000 : (s < -1000 ? -1000 : s);
    scale1[threadIdx.x] = ldexp(1.0, s1);
    scale2[threadIdx.x] = ldexp(1.0, s - s1);
    if (e == kNonFinite) scale1[threadIdx.x] = 0.0;
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int a = tx, b = ty + 8 * s;
    const int rr = p.row_contig ? a : b;
    const int kk = p.row_contig ? b : a;
    const int64_t r = r0 + rr, kq = k0 + kk;
    double4 v = make_double4(0.0, 0.0, 0.0, 0.0);
    if (r < p.rows && kq < p.kq) {
      const int64_t sr = p.row_contig ? r : kq, sc = p.row_contig ? kq : r;
      if (p.layout == QGEMM_INTERLEAVED) {
        const double *e = p.X + 4 * (sr + sc * p.ld);
        v = make_double4(e[0], e[1], e[2], e[3]);
      } else {
        const double *e = p.X + sr + sc * p.ld;
        v = make_double4(e[0], e[p.ps], e[2 * p.ps], e[3 * p.ps]);
      }
      if (p.negmask & 2u) v.y = -v.y;
      if (p.negmask & 4u) v.z = -v.z;
      if (p.negmask & 8u) v.w = -v.w;
    }
    tile[kk][rr] = v;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int kk = tx, rr = ty + 8 * s;
    const int64_t r = r0 + rr, kq = k0 + kk;
    if (r >= p.rows || 4 * kq >= p.kp) continue;
    const double4 v = tile[kk][rr];
    const double f1 = scale1[rr], f2 = scale2[rr];
    const double comp[4] = {v.x, v.y, v.z, v.w};
    int d[4][NSL];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double x = comp[j] * f1;
      x *= f2;
      if (!(fabs(x) <= 140737488355328.0)) x = 0.0;  // non-finite row: digits 0, C gets NaN
      digits6(x, d[j]);
    }
    if (!IS_B) {
#pragma unroll
      for (int t = 0; t < NSL; ++t) {
        __nv_bfloat16 *dst = p.out + t * p.slice_stride + r * p.kp + 4 * kq;
        __align__(8) __nv_bfloat16 w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = __float2bfloat16_rn(static_cast<float>(d[j][t]));
        *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(w);
      }
    } else {
#pragma unroll
      for (int t = 0; t < NSL; ++t)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          __align__(8) __nv_bfloat16 w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int q = j ^ c;
            const int x = basis_sign(j, q) < 0 ? -d[q][t] : d[q][t];
            w[j] = __float2bfloat16_rn(static_cast<float>(x));
          }
          __nv_bfloat16 *dst = p.out + t * p.slice_stride + (4 * r + c) * p.kp + 4 * kq;
          *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(w);
        }
    }
  }
}

// ----------------------------------------------------------- host side ---
struct SlicedPlan {
  int64_t kp;
  size_t a_off, b_off, maxa_off, maxb_off, ea_off, eb_off, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

SlicedPlan plan_for(const GemmDesc &d) {
  SlicedPlan s;
  s.kp = ((4 * d.k + SBK - 1) / SBK) * SBK;
  s.a_off = 0;
  const size_t a_bytes = static_cast<size_t>(NSL) * d.m * s.kp * 2;
  s.b_off = align_up(a_bytes, 1024);
  const size_t b_bytes = static_cast<size_t>(NSL) * 4 * d.n * s.kp * 2;
  s.maxa_off = align_up(s.b_off + b_bytes, 256);
  s.maxb_off = align_up(s.maxa_off + 8 * d.m, 256);
  s.ea_off = align_up(s.maxb_off + 8 * d.n, 256);
  s.eb_off = align_up(s.ea_off + 4 * d.m, 256);
  s.total = align_up(s.eb_off + 4 * d.n, 256);
  return s;
}

bool encode_slices(CUtensorMap *map, const void *base, int64_t kp, int64_t rows, int box_rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  if (rows >= (1ll << 32) || kp >= (1ll << 32)) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows), NSL};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(kp) * 2,
                           static_cast<cuuint64_t>(kp) * 2 * static_cast<cuuint64_t>(rows)};
  cuuint32_t box[3] = {SBK, static_cast<cuuint32_t>(box_rows), NSL};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int launch_max(const MatView &v, bool by_col, int layout, unsigned long long *out,
               cudaStream_t stream) {
  const int64_t gx = (v.rows + 31) / 32, gy = (v.cols + 31) / 32;
  if (gx == 0 || gy == 0) return QGEMM_SUCCESS;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  slice_max_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), 256, 0,
                     stream>>>(static_cast<const double *>(v.ptr), v.ld, v.ps, v.rows, v.cols,
                               layout, by_col ? 1 : 0, out);
  return launch_status();
}

int launch_slices(bool is_b, const MatView &v, int op, int64_t rows, int64_t kq, int64_t kp,
                  int layout, __nv_bfloat16 *out, int64_t slice_stride,
                  const unsigned long long *maxbits, int *eout, cudaStream_t stream) {
  SliceArgs a;
  a.X = static_cast<const double *>(v.ptr);
  a.ld = v.ld;
  a.ps = v.ps;
  a.rows = rows;
  a.kq = kq;
  a.kp = kp;
  a.slice_stride = slice_stride;
  a.out = out;
  a.maxbits = maxbits;
  a.eout = eout;
  a.layout = layout;
  a.row_contig = is_b ? (op_trans(op) ? 1 : 0) : (op_trans(op) ? 0 : 1);
  a.negmask = op_conj(op) ? 0xEu : 0u;
  const int64_t gx = (rows + 31) / 32, gy = (kp / 4 + 31) / 32;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (is_b)
    slice_kernel<true><<<grid, 256, 0, stream>>>(a);
  else
    slice_kernel<false><<<grid, 256, 0, stream>>>(a);
  return launch_status();
}

}  // namespace

int sliced_workspace_bytes(const GemmDesc &d, size_t *bytes) {
  *bytes = (d.k == 0 || d.m == 0 || d.n == 0) ? 0 : plan_for(d).total;
  return QGEMM_SUCCESS;
}

int launch_sliced_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream) {
  const SlicedPlan pl = plan_for(d);
  if (ws == nullptr || ws_bytes < pl.total) return QGEMM_ERR_WORKSPACE;
  unsigned char *w = static_cast<unsigned char *>(ws);
  auto *wa = reinterpret_cast<__nv_bfloat16 *>(w + pl.a_off);
  auto *wb = reinterpret_cast<__nv_bfloat16 *>(w + pl.b_off);
  auto *maxa = reinterpret_cast<unsigned long long *>(w + pl.maxa_off);
  auto *maxb = reinterpret_cast<unsigned long long *>(w + pl.maxb_off);
  int *ea = reinterpret_cast<int *>(w + pl.ea_off);
  int *eb = reinterpret_cast<int *>(w + pl.eb_off);

  if (cudaMemsetAsync(w + pl.maxa_off, 0, pl.ea_off - pl.maxa_off, stream) != cudaSuccess)
    return launch_status();
  // row maxima of op(A): stored rows for N/C, stored columns for T/H;
  // column maxima of op(B): stored columns for N/C, stored rows for T/H
  int rc = launch_max(d.A, op_trans(d.opA), d.layout, maxa, stream);
  if (rc) return rc;
  rc = launch_max(d.B, !op_trans(d.opB), d.layout, maxb, stream);
  if (rc) return rc;
  rc = launch_slices(false, d.A, d.opA, d.m, d.k, pl.kp, d.layout, wa, d.m * pl.kp, maxa, ea,
                     stream);
  if (rc) return rc;
  rc = launch_slices(true, d.B, d.opB, d.n, d.k, pl.kp, d.layout, wb, 4 * d.n * pl.kp, maxb, eb,
                     stream);
  if (rc) return rc;

  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  if (!encode_slices(&tmA, wa, pl.kp, d.m, SBM) || !encode_slices(&tmB, wb, pl.kp, 4 * d.n, SBN))
    return QGEMM_ERR_UNSUPPORTED;
  SlicedParams g{};
  g.m = d.m;
  g.n = d.n;
  g.num_kb = static_cast<int>(pl.kp / SBK);
  g.num_mt = static_cast<int>((d.m + SBM - 1) / SBM);
  g.num_nt = static_cast<int>((d.n + SBNQ - 1) / SBNQ);
  g.layout = d.layout;
  g.beta_zero = d.beta_zero ? 1 : 0;
  g.tri = d.tri;
  g.c_vec2 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
  g.C = static_cast<double *>(d.C);
  g.ldc = d.ldc;
  g.psC = d.psc;
  for (int s = 0; s < 4; ++s) {
    g.alpha[s] = d.alpha[s];
    g.beta[s] = d.beta[s];
  }
  g.eA = ea;
  g.eB = eb;
  const int64_t tiles = static_cast<int64_t>(g.num_mt) * g.num_nt;
  if (tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  static bool smem_set[64];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!smem_set[dev]) {
    if (cudaFuncSetAttribute(sliced_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmem)) != cudaSuccess)
      return launch_status();
    smem_set[dev] = true;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = static_cast<int>(std::min<int64_t>(tiles, sms));
  sliced_gemm_kernel<<<grid, kSThreads, kSmem, stream>>>(tmA, tmB, g, static_cast<int>(tiles),
                                                         wait_limit_ns());
  return launch_status();
}

int sliced_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_sliced_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_sliced_error, &z, sizeof(int));
  return v;
}

}  // namespace qg
