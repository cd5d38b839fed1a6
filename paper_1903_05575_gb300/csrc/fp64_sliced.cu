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
#include <vector>

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
using split::tmem_ld32;
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
// Largest quaternion k: the slicing grid (k/8 blocks <= 65535) and the 64-bit
// level sums (2^46 per 256-k chunk) both stay in range.
constexpr int64_t kMaxSlicedK = int64_t(1) << 21;

struct SlicedParams {
  int64_t m, n;
  int num_kb, num_mt, num_nt;
  int layout, beta_zero, tri, c_vec2;
  int swap;       // 1: the kernel computes D = (op(A) op(B))^H; store C = conj(D)^T
  int alpha_real, beta_real;  // scalars with zero vector part: 4 FP64 products, not 16
  int krange;     // k-range of a tile when op(A) or op(B) is triangular (GemmDesc)
  double *C;
  int64_t ldc, psC;
  double alpha[4], beta[4];
  const int *eA;  // per quaternion row of op(A)
  const int *eB;  // per quaternion column of op(B)
  // K split (single problems): tile t of the launch is share z = t / (num_mt
  // num_nt) of its tile's k-blocks, whose product P goes to part + z m n 4
  // (dense, interleaved, leading dimension m) for a second kernel to sum.
  int ksplit;     // 0 or 1: no split
  double *part;
};

// Pre-pass arguments of one operand.  The maxima are kept as exponents: the
// largest e(x) over a row, column or kappa, where e(x) is the exponent with
// 2^(e - 1) <= |x| < 2^e (integer, from the bits of x); kExpEmpty (the memset
// byte 0x80) when every element is zero, kExpInf when one is Inf or NaN.
// Kappa balancing: with per-kappa exponents ka, kb of op(A) and op(B), kappa
// gets t = floor((ka - kb) / 2), and the products use the exact rescaling
// (A diag(2^-t)) (diag(2^t) B) = A B, so a row of op(A) and a column of
// op(B) that span many binades along kappa share their largest scales.
constexpr int kExpInf = 0x40000000;
constexpr int kExpEmpty = static_cast<int>(0x80808080u);
struct MaxArgs {
  const double *X;
  int64_t ld, ps;        // stored leading dimension, plane stride
  int64_t srows, scols;  // stored extent
  int layout;
  int by_col;            // 0: maxima per stored row, 1: per stored column
  int width;             // components stored per element (4, 2 or 1)
  int *out;              // exponent maxima (atomicMax)
  // balancing: 0 none; -1 this is op(A) (exponents e - t); +1 op(B) (e + t).
  // The kappa of a stored element is its column when by_col = 0, else its row.
  int tsign;
  const int *ka, *kb;    // per-kappa exponents of op(A) and op(B)
};

struct SliceArgs {
  const double *X;
  int64_t ld, ps;        // stored leading dimension, plane stride
  int64_t rows;          // rows of the op-matrix (m for A, n for B)
  int64_t kq;            // quaternion K
  int64_t kp;            // padded real K (multiple of SBK)
  int64_t slice_stride;  // elements between slices in the output
  __nv_bfloat16 *out;
  const int *emax;       // per op row: exponent maxima (balanced when tsign != 0)
  int *eout;             // per op row: the exponent used
  int tsign;             // balancing as in MaxArgs (-1 for A, +1 for B, 0 none)
  const int *ka, *kb;    // per-kappa exponents of op(A) and op(B)
  int layout;
  int row_contig;        // stored row index == op row
  uint32_t negmask;      // bit j: negate component j (conjugation)
  int width;             // components stored per element (4, 2 or 1; the rest are 0)
  int kw;                // components per kappa in the output (4; 2 or 1 for a
                         // complex or real left operand)
};

// One problem of a grouped batch (device descriptor in the workspace).
struct alignas(128) SlicedProb {
  CUtensorMap tmA;  // A' slices: (kp, m, 6) bf16
  CUtensorMap tmB;  // B' slices: (kp, 4n, 6) bf16
  SlicedParams g;
  MaxArgs ma, mb;
  SliceArgs sa, sb;
};

struct Ctl {
  uint64_t full[SST];
  uint64_t empty[SST];
  uint64_t accfull;  // the MMAs of a chunk completed
  uint64_t free23;   // drain has read levels 2, 3 of a chunk
  uint64_t free01;   // drain has read levels 0, 1 of a chunk
  uint64_t free45;   // drain has read levels 4, 5 of a tile
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
  // a triangular operand: the tiles with the longest k-range first, so the
  // CTAs' round-robin shares stay balanced
  if (g.krange == 1) mt = g.num_mt - 1 - mt;
  if (g.krange == 4) nt = g.num_nt - 1 - nt;
}

// k-blocks [lo, hi) of tile (mt, nt): all of K, or the part where a
// triangular operand can be nonzero for the tile's rows or columns.
__device__ __forceinline__ void kb_range(const SlicedParams &g, int mt, int nt, int z, int &lo,
                                         int &hi) {
  lo = 0;
  hi = g.num_kb;
  const int64_t rq0 = static_cast<int64_t>(mt) * SBM, cq0 = static_cast<int64_t>(nt) * SBNQ;
  if (g.krange == 1) {
    const int64_t e = (4 * (rq0 + SBM) + SBK - 1) / SBK;
    if (e < hi) hi = static_cast<int>(e);
  }
  if (g.krange == 2) lo = static_cast<int>(4 * rq0 / SBK);
  if (g.krange == 3) lo = static_cast<int>(4 * cq0 / SBK);
  if (g.krange == 4) {
    const int64_t e = (4 * (cq0 + SBNQ) + SBK - 1) / SBK;
    if (e < hi) hi = static_cast<int>(e);
  }
  if (lo > hi) lo = hi;
  if (g.ksplit > 1) {  // share z of the k-blocks
    const int64_t span = hi - lo;
    const int l2 = lo + static_cast<int>(span * z / g.ksplit);
    hi = lo + static_cast<int>(span * (z + 1) / g.ksplit);
    lo = l2;
  }
}

__device__ __forceinline__ bool tile_skip(const SlicedParams &g, int mt, int nt) {
  if (g.tri == 1) return static_cast<int64_t>(mt) * SBM + SBM - 1 < static_cast<int64_t>(nt) * SBNQ;
  if (g.tri == 2) return static_cast<int64_t>(nt) * SBNQ + SBNQ - 1 < static_cast<int64_t>(mt) * SBM;
  return false;
}

__device__ __forceinline__ void mma(uint32_t d, uint32_t a, uint32_t b, int n, uint32_t acc) {
  umma_bf16(d, smem_desc_sw64(a), smem_desc_sw64(b), idesc_bf16(SBM, n), acc);
}

// One k-step (16 real k) of the 21 slice products, in two groups: A slice i
// against the adjacent B slices j0.., into the adjacent level regions
// i + j0.. (64 TMEM columns each).
// Levels 2..5: 18 products, 6 MMAs.  Levels 2, 3 restart at a chunk's first
// k-step, levels 4, 5 at a tile's first k-step.
__device__ __forceinline__ void mma_levels25(uint32_t d, uint32_t ka, uint32_t kb,
                                             bool chunk_start, bool tile_start) {
  if (chunk_start && !tile_start) {
    mma(d + 2 * SBN, ka, kb + 2 * kSliceB, 2 * SBN, 0u);                  // 02 03
    mma(d + 4 * SBN, ka, kb + 4 * kSliceB, 2 * SBN, 1u);                  // 04 05
  } else {
    mma(d + 2 * SBN, ka, kb + 2 * kSliceB, 4 * SBN, tile_start ? 0u : 1u);  // 02 03 04 05
  }
  mma(d + 2 * SBN, ka + 1 * kSliceA, kb + 1 * kSliceB, 4 * SBN, 1u);      // 11 12 13 14
  mma(d + 2 * SBN, ka + 2 * kSliceA, kb, 4 * SBN, 1u);                    // 20 21 22 23
  mma(d + 3 * SBN, ka + 3 * kSliceA, kb, 3 * SBN, 1u);                    // 30 31 32
  mma(d + 4 * SBN, ka + 4 * kSliceA, kb, 2 * SBN, 1u);                    // 40 41
  mma(d + 5 * SBN, ka + 5 * kSliceA, kb, 1 * SBN, 1u);                    // 50
}
// Levels 0, 1: 3 products, 2 MMAs; both restart at a chunk's first k-step.
__device__ __forceinline__ void mma_levels01(uint32_t d, uint32_t ka, uint32_t kb,
                                             bool chunk_start) {
  mma(d, ka, kb, 2 * SBN, chunk_start ? 0u : 1u);                         // 00 01
  mma(d + SBN, ka + kSliceA, kb, 1 * SBN, 1u);                            // 10
}

// The same 21 products in three groups by level, for the first stage of a
// chunk: levels 4, 5 (11 products, 6 MMAs) do not wait for the drain of the
// previous chunk, levels 2, 3 (7 products, 4 MMAs) and 0, 1 (3 products, 2
// MMAs) wait for their regions to be read.
__device__ __forceinline__ void mma_levels45(uint32_t d, uint32_t ka, uint32_t kb,
                                             bool tile_start) {
  mma(d + 4 * SBN, ka, kb + 4 * kSliceB, 2 * SBN, tile_start ? 0u : 1u);  // 04 05
  mma(d + 4 * SBN, ka + 1 * kSliceA, kb + 3 * kSliceB, 2 * SBN, 1u);      // 13 14
  mma(d + 4 * SBN, ka + 2 * kSliceA, kb + 2 * kSliceB, 2 * SBN, 1u);      // 22 23
  mma(d + 4 * SBN, ka + 3 * kSliceA, kb + 1 * kSliceB, 2 * SBN, 1u);      // 31 32
  mma(d + 4 * SBN, ka + 4 * kSliceA, kb, 2 * SBN, 1u);                    // 40 41
  mma(d + 5 * SBN, ka + 5 * kSliceA, kb, 1 * SBN, 1u);                    // 50
}
__device__ __forceinline__ void mma_levels23(uint32_t d, uint32_t ka, uint32_t kb,
                                             bool chunk_start) {
  mma(d + 2 * SBN, ka, kb + 2 * kSliceB, 2 * SBN, chunk_start ? 0u : 1u);  // 02 03
  mma(d + 2 * SBN, ka + 1 * kSliceA, kb + 1 * kSliceB, 2 * SBN, 1u);       // 11 12
  mma(d + 2 * SBN, ka + 2 * kSliceA, kb, 2 * SBN, 1u);                     // 20 21
  mma(d + 3 * SBN, ka + 3 * kSliceA, kb, 1 * SBN, 1u);                     // 30
}

// TMEM <-> registers, 32x32b shapes (lane = row of this thread).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
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
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

// T[q] += 2^SHIFT * v[q] for exact integers v[q].
template <int SHIFT>
__device__ __forceinline__ void add_level(long long (&T)[32], const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 32; ++q)
    T[q] += static_cast<long long>(__float2int_rn(v[q])) * (1ll << SHIFT);
}

// Keeps the compiler from sinking the adds into T below the next TMEM load
// (which would hold two sets of loaded levels live at once).
__device__ __forceinline__ void pin(long long (&T)[32]) {
#pragma unroll
  for (int q = 0; q < 32; ++q) asm volatile("" : "+l"(T[q]));
}

// x * 2^e without rounding unless the result is subnormal.
__device__ __forceinline__ double scale2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __hiloint2double((e + 1023) << 20, 0);
  return ldexp(x, e);
}

// The epilogue of quaternion column nq0 + q of row i of a finished tile:
// S (4 doubles, units of 2^-24 of a level-0 digit product) from the spare
// TMEM columns, P = 2^(e_i + e_n - 38) S, C <- alpha P + beta C in FP64.
// All lanes execute the TMEM load; the rest is per lane.
__device__ __forceinline__ void epilogue_piece(const SlicedParams &g, uint32_t spare, int64_t i,
                                               int ea, int64_t nq0, int q, int z) {
  uint32_t r[8];
  tmem_ld8(spare + 8 * q, r);
  const int64_t nn = nq0 + q;
  if (i >= g.m || nn >= g.n) return;
  if ((g.tri == 1 && i < nn) || (g.tri == 2 && i > nn)) return;
  double P[4] = {0.0, 0.0, 0.0, 0.0};
  if (g.num_kb > 0) {  // k = 0 (or alpha = 0) in a grouped batch: C <- beta C
    const int eb = g.eB[nn];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double Sc =
          __hiloint2double(static_cast<int>(r[2 * c + 1]), static_cast<int>(r[2 * c]));
      P[c] = (ea == kNonFinite || eb == kNonFinite) ? __longlong_as_double(0x7ff8000000000000ll)
                                                    : scale2(Sc, ea + eb - 38);
    }
  }
  if (g.ksplit > 1) {  // this K share's product, for the summing kernel
    double *dst = g.part + (static_cast<int64_t>(z) * g.m * g.n + i + nn * g.m) * 4;
    *reinterpret_cast<double2 *>(dst) = make_double2(P[0], P[1]);
    *reinterpret_cast<double2 *>(dst + 2) = make_double2(P[2], P[3]);
    return;
  }
  // element (ci, cj) of C; a transposed problem holds (AB)^H: take conj(D)^T
  int64_t ci = i, cj = nn;
  if (g.swap) {
    ci = nn;
    cj = i;
    P[1] = -P[1];
    P[2] = -P[2];
    P[3] = -P[3];
  }
  double cin[4] = {0.0, 0.0, 0.0, 0.0};
  double *dst0;
  if (g.layout == QGEMM_INTERLEAVED) {
    dst0 = g.C + 4 * (ci + cj * g.ldc);
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
    dst0 = g.C + ci + cj * g.ldc;
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
    if (g.alpha_real) {
      acc = g.alpha[0] * P[c];
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = c ^ j;
        const double a = basis_sign(s, j) < 0 ? -g.alpha[s] : g.alpha[s];
        acc = fma(a, P[j], acc);
      }
    }
    if (!g.beta_zero) {
      if (g.beta_real) {
        acc = fma(g.beta[0], cin[c], acc);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int s = c ^ j;
          const double b = basis_sign(s, j) < 0 ? -g.beta[s] : g.beta[s];
          acc = fma(b, cin[j], acc);
        }
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

// A finished tile whose epilogue is still (partly) pending, for one drain
// thread: its row, first quaternion column, row exponent and progress.
struct Pending {
  const SlicedParams *g;
  int64_t i, nq0;
  int ea;
  int z;     // K share (split problems)
  int done;  // quaternions 0 .. done-1 written; 8 when nothing is pending
};

__device__ __forceinline__ void run_pending(uint32_t spare, Pending &pd, int upto) {
  while (pd.done < upto) {
    epilogue_piece(*pd.g, spare, pd.i, pd.ea, pd.nq0, pd.done, pd.z);
    ++pd.done;
  }
}

// Tile t -> problem parameters, tensor maps and tile coordinates.  Single
// problem: rasterised in groups of kGroupM row tiles; grouped: tiles[t] =
// (problem, row tile, column tile).
template <bool GROUPED>
__device__ __forceinline__ void tile_of(int t, const SlicedParams &single, const CUtensorMap *smA,
                                        const CUtensorMap *smB, const SlicedProb *probs,
                                        const int4 *tiles, const SlicedParams *&g,
                                        const CUtensorMap *&mA, const CUtensorMap *&mB, int &mt,
                                        int &nt, int &z) {
  if (GROUPED) {
    const int4 e = tiles[t];
    const SlicedProb *pr = probs + e.x;
    g = &pr->g;
    mA = &pr->tmA;
    mB = &pr->tmB;
    mt = e.y;
    nt = e.z;
    z = 0;
  } else {
    g = &single;
    mA = smA;
    mB = smB;
    const int per = single.num_mt * single.num_nt;
    z = single.ksplit > 1 ? t / per : 0;
    tile_coords(single, single.ksplit > 1 ? t % per : t, mt, nt);
  }
}

template <bool GROUPED>
__global__ void __launch_bounds__(kSThreads, 1)
    sliced_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB, const SlicedParams single,
                       const SlicedProb *__restrict__ probs, const int4 *__restrict__ tiles,
                       int ntiles, uint64_t limit_ns) {
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
    mbar_init(&ctl->free23, kDrainWarps);
    mbar_init(&ctl->free01, kDrainWarps);
    mbar_init(&ctl->free45, kDrainWarps);
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
    // ---------------- TMA producer ----------------
    if (elect_one()) {
      if (!GROUPED) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
      }
      uint32_t s_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const SlicedParams *g;
        const CUtensorMap *mA, *mB;
        int mt, nt, z;
        tile_of<GROUPED>(t, single, &tmA, &tmB, probs, tiles, g, mA, mB, mt, nt, z);
        if (tile_skip(*g, mt, nt)) continue;
        int kb_lo, kb_hi;
        kb_range(*g, mt, nt, z, kb_lo, kb_hi);
        for (int kb = kb_lo; kb < kb_hi; ++kb, ++s_run) {
          const int st = s_run % SST;
          if (!wait_phase(&ctl->empty[st], ((s_run / SST) & 1) ^ 1, limit_ns, ctl)) {
            set_abort(ctl);
            ok = false;
            break;
          }
          unsigned char *sa = ring + st * kStageBytes;
          mbar_arrive_expect_tx(&ctl->full[st], kStageBytes);
          tma_load_3d(sa, mA, &ctl->full[st], kb * SBK, mt * SBM, 0);
          tma_load_3d(sa + kStageA, mB, &ctl->full[st], kb * SBK, nt * SBN, 0);
        }
      }
      if (!ok) {  // let this CTA's copies in flight land before it retires
        for (uint32_t q = s_run > SST ? s_run - SST : 0; q < s_run; ++q)
          mbar_wait_bounded(&ctl->full[q % SST], (q / SST) & 1, limit_ns);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // The first stage of a chunk issues the level 4, 5 products of both
    // k-steps at once (those regions are read only at a tile's end: a tile's
    // first chunk waits for that), then the level 2, 3 products once the
    // drain has read those regions of the previous chunk, then levels 0, 1.
    // The other stages issue all 21 products as 8 MMAs.
    if (elect_one()) {
      const uint32_t ring_addr = smem_u32(ring);
      uint32_t s_run = 0, c_run = 0, t_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const SlicedParams *g;
        const CUtensorMap *mA, *mB;
        int mt, nt, z;
        tile_of<GROUPED>(t, single, &tmA, &tmB, probs, tiles, g, mA, mB, mt, nt, z);
        if (tile_skip(*g, mt, nt)) continue;
        int kb_lo, kb_hi;
        kb_range(*g, mt, nt, z, kb_lo, kb_hi);
        const int nch = (kb_hi - kb_lo + kChunkKb - 1) / kChunkKb;
        if (nch > 0) {
          // levels 4, 5 of the previous tile read
          if (!wait_phase(&ctl->free45, (t_run & 1) ^ 1, limit_ns, ctl)) {
            set_abort(ctl);
            ok = false;
            break;
          }
          ++t_run;
          tc_fence_after();
        }
        for (int ch = 0; ch < nch && ok; ++ch, ++c_run) {
          const uint32_t par = (c_run & 1) ^ 1;
          const int kb0 = kb_lo + ch * kChunkKb, kb1 = min(kb_hi, kb0 + kChunkKb);
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
            if (kb == kb0) {
#pragma unroll
              for (int ks = 0; ks < SBK / 16; ++ks)
                mma_levels45(tmem, sa + ks * 32, sb + ks * 32, ks == 0 && ch == 0);
              if (!wait_phase(&ctl->free23, par, limit_ns, ctl)) {
                set_abort(ctl);
                ok = false;
                break;
              }
              tc_fence_after();
#pragma unroll
              for (int ks = 0; ks < SBK / 16; ++ks)
                mma_levels23(tmem, sa + ks * 32, sb + ks * 32, ks == 0);
              if (!wait_phase(&ctl->free01, par, limit_ns, ctl)) {
                set_abort(ctl);
                ok = false;
                break;
              }
              tc_fence_after();
#pragma unroll
              for (int ks = 0; ks < SBK / 16; ++ks)
                mma_levels01(tmem, sa + ks * 32, sb + ks * 32, ks == 0);
            } else {
#pragma unroll
              for (int ks = 0; ks < SBK / 16; ++ks) {
                mma_levels25(tmem, sa + ks * 32, sb + ks * 32, false, false);
                mma_levels01(tmem, sa + ks * 32, sb + ks * 32, false);
              }
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
    // Per chunk: read levels 2, 3 -> release them -> add; read levels 0, 1 ->
    // release -> add; then a share of the previous tile's epilogue, whose S
    // waits in the spare TMEM columns 384..511.
    const int ew = warp - 2;
    const int quad = warp & 3;  // TMEM lanes 32*quad .. +31 (hardware rule: warp % 4)
    const int half = ew >> 2;   // columns [32*half, 32*half + 32) of each level region
    const uint32_t lanes = static_cast<uint32_t>(32 * quad) << 16;
    const uint32_t base = tmem + lanes + 32 * half;
    const uint32_t spare = tmem + lanes + 6 * SBN + 64 * half;
    uint32_t c_run = 0;
    bool ok = true;
    Pending pd{nullptr, 0, 0, 0, 0, 8};
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const SlicedParams *g;
      const CUtensorMap *mA, *mB;
      int mt, nt, z;
      tile_of<GROUPED>(t, single, &tmA, &tmB, probs, tiles, g, mA, mB, mt, nt, z);
      if (tile_skip(*g, mt, nt)) continue;
      int kb_lo, kb_hi;
      kb_range(*g, mt, nt, z, kb_lo, kb_hi);
      const int nch = (kb_hi - kb_lo + kChunkKb - 1) / kChunkKb;
      const int nbound = nch - 1;  // chunk ends before the tile's last
      long long T[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) T[q] = 0;
      for (int ch = 0; ch < nbound; ++ch, ++c_run) {
        if (!wait_phase(&ctl->accfull, c_run & 1, limit_ns, ctl)) {
          set_abort(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        {
          float v2[32], v3[32];
          tmem_ld32(base + 2 * SBN, v2);
          tmem_ld32(base + 3 * SBN, v3);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->free23);
          add_level<8>(T, v2);
          add_level<0>(T, v3);
          pin(T);
        }
        {
          float v0[32], v1[32];
          tmem_ld32(base + 0 * SBN, v0);
          tmem_ld32(base + 1 * SBN, v1);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->free01);
          add_level<24>(T, v0);
          add_level<16>(T, v1);
          pin(T);
        }
        run_pending(spare, pd, ((ch + 1) * 8 + nbound - 1) / nbound);
      }
      if (!ok) break;
      // last chunk: levels 4, 5 as well; then this tile's S goes to TMEM
      // (no chunk at all for k = 0 in a grouped batch)
      float tail[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) tail[q] = 0.f;
      if (nch > 0) {
        if (!wait_phase(&ctl->accfull, c_run & 1, limit_ns, ctl)) {
          set_abort(ctl);
          break;
        }
        ++c_run;
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v4[16], v5[16];
          tmem_ld16(base + 4 * SBN + 16 * h, v4);
          tmem_ld16(base + 5 * SBN + 16 * h, v5);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            tail[16 * h + q] = fmaf(v5[q], 0.00390625f, v4[q]) * 0.00390625f;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->free45);
        float v[32];
        tmem_ld32(base + 2 * SBN, v);
        add_level<8>(T, v);
        tmem_ld32(base + 3 * SBN, v);
        add_level<0>(T, v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->free23);
        tmem_ld32(base + 0 * SBN, v);
        add_level<24>(T, v);
        tmem_ld32(base + 1 * SBN, v);
        add_level<16>(T, v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->free01);
      }
      run_pending(spare, pd, 8);  // the previous tile's S leaves TMEM first
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t w[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const double S = static_cast<double>(T[8 * h + q]) + static_cast<double>(tail[8 * h + q]);
          w[2 * q] = static_cast<uint32_t>(__double2loint(S));
          w[2 * q + 1] = static_cast<uint32_t>(__double2hiint(S));
        }
        tmem_st16(spare + 16 * h, w);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      pd.g = g;
      pd.i = static_cast<int64_t>(mt) * SBM + 32 * quad + lane;
      pd.nq0 = static_cast<int64_t>(nt) * SBNQ + 8 * half;
      pd.ea = pd.i < g->m ? g->eA[pd.i] : 0;
      pd.z = z;
      pd.done = 0;
    }
    run_pending(spare, pd, 8);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------ pre-pass ---
// e(x): 2^(e - 1) <= |x| < 2^e for finite nonzero x, from the bits of x
// (integer operations only); kExpEmpty for zero, kExpInf for Inf or NaN.
__device__ __forceinline__ int elem_exp(double x) {
  const unsigned long long b =
      static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
  if (b >= 0x7ff0000000000000ull) return kExpInf;
  if (b == 0) return kExpEmpty;
  const int E = static_cast<int>(b >> 52);
  if (E > 0) return E - 1022;
  return (63 - __clzll(static_cast<long long>(b))) - 1073;  // subnormal
}

// The balancing exponent t of one kappa (0 when a kappa maximum is zero or
// not finite): op(A)'s kappa column scaled by 2^-t and op(B)'s kappa row by
// 2^t then have the same largest exponent, up to one.
__device__ __forceinline__ int kappa_balance(const int *ka, const int *kb, int64_t kappa) {
  const int x = ka[kappa], y = kb[kappa];
  if (x <= kExpEmpty / 2 || y <= kExpEmpty / 2 || x >= kExpInf || y >= kExpInf) return 0;
  return (x - y) >> 1;  // floor
}

// Largest exponent of the components of each quaternion row (by_col = 0) or
// column (by_col = 1) of a stored matrix, with the kappa balancing of the
// element when tsign != 0, max-reduced into out[]: one 32 x 32 tile (rt, ct)
// of the stored matrix per call, 256 threads.
__device__ __forceinline__ void max_tile(const MaxArgs &a, int64_t rt, int64_t ct,
                                         int (*red)[32]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r = rt * 32 + tx;
  const int64_t c0 = ct * 32;
  int rowm = kExpEmpty;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t c = c0 + ty + 8 * s;
    int mx = kExpEmpty;
    if (r < a.srows && c < a.scols) {
      for (int comp = 0; comp < a.width; ++comp) {
        const double x = a.layout == QGEMM_INTERLEAVED ? a.X[a.width * (r + c * a.ld) + comp]
                                                       : a.X[r + c * a.ld + comp * a.ps];
        const int e = elem_exp(x);
        mx = e > mx ? e : mx;
      }
      if (a.tsign != 0 && mx > kExpEmpty && mx < kExpInf)
        mx += a.tsign * kappa_balance(a.ka, a.kb, a.by_col ? r : c);
    }
    if (a.by_col) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
      }
      if (tx == 0 && c < a.scols && mx != kExpEmpty) atomicMax(a.out + c, mx);
    } else {
      rowm = mx > rowm ? mx : rowm;
    }
  }
  if (!a.by_col) {
    red[ty][tx] = rowm;
    __syncthreads();
    if (ty == 0) {
      int v = red[0][tx];
#pragma unroll
      for (int w = 1; w < 8; ++w) v = red[w][tx] > v ? red[w][tx] : v;
      if (r < a.srows && v != kExpEmpty) atomicMax(a.out + r, v);
    }
  }
}

__global__ void __launch_bounds__(256) slice_max_kernel(const MaxArgs a) {
  __shared__ int red[8][32];
  max_tile(a, blockIdx.x, blockIdx.y, red);
}

// Grouped: mtiles[t] = (problem, operand 0 A / 1 B, row tile, column tile).
__global__ void __launch_bounds__(256)
    grouped_slice_max_kernel(const SlicedProb *__restrict__ probs,
                             const int4 *__restrict__ mtiles, int n) {
  __shared__ int red[8][32];
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int4 e = mtiles[t];
    const SlicedProb &pr = probs[e.x];
    max_tile(e.y ? pr.mb : pr.ma, e.z, e.w, red);
    __syncthreads();
  }
}

// Exponent e with max < 2^e of a row from its maximum: 0 for a zero row,
// kNonFinite for a row with Inf or NaN.
__device__ __forceinline__ int row_exponent(int emax) {
  if (emax >= kExpInf) return kNonFinite;
  if (emax <= kExpEmpty / 2) return 0;
  return emax;
}

// round(a 2^s) to the nearest integer (ties to even) for |a| 2^s <= 2^47,
// from the bits of a: integer operations only (GB300's FP64 pipe is narrow).
__device__ __forceinline__ long long round_scaled(double a, int s) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(a));
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int e2;  // |a| = m 2^e2
  if (E == 0) {
    e2 = -1074;
  } else {
    m |= 1ull << 52;
    e2 = E - 1075;
  }
  const int sh = -(e2 + s);  // |a| 2^s = m 2^-sh
  long long q;
  if (sh <= 0) {
    q = static_cast<long long>(m << (-sh));
  } else if (sh >= 64) {
    q = 0;  // m < 2^53 <= 2^(sh-1): below one half
  } else {
    const unsigned long long qq = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1);
    const unsigned long long half = 1ull << (sh - 1);
    q = static_cast<long long>(qq + ((rem > half || (rem == half && (qq & 1))) ? 1 : 0));
  }
  return (b >> 63) ? -q : q;
}

// Balanced base-256 digits of X, |X| <= 2^47: X = sum d_t 2^(8 (5 - t)).
__device__ __forceinline__ void digits6(long long X, int (&d)[NSL]) {
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
// The first kw of four BF16 values (bits lo = v0 | v1 << 16, hi = v2 | v3 << 16)
// at dst (aligned to kw values).
__device__ __forceinline__ void store_bits(__nv_bfloat16 *dst, uint32_t lo, uint32_t hi, int kw) {
  if (kw == 4)
    *reinterpret_cast<uint2 *>(dst) = make_uint2(lo, hi);
  else if (kw == 2)
    *reinterpret_cast<uint32_t *>(dst) = lo;
  else
    *reinterpret_cast<unsigned short *>(dst) = static_cast<unsigned short>(lo & 0xffffu);
}

struct SliceSmem {
  double4 tile[32][33];
  int shift[32];  // 47 - e of each row; kNonFinite for a row with Inf or NaN
};

template <bool IS_B>
__device__ __forceinline__ void slice_tile(const SliceArgs &p, int64_t rt, int64_t kt,
                                           SliceSmem &sm) {
  double4 (*tile)[33] = sm.tile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = rt * 32;
  const int64_t k0 = kt * 32;
  if (threadIdx.x < 32) {
    const int64_t r = r0 + threadIdx.x;
    int e = 0;
    if (r < p.rows) {
      e = row_exponent(p.emax[r]);
      if (kt == 0) p.eout[r] = e;
    }
    sm.shift[threadIdx.x] = e == kNonFinite ? kNonFinite : 47 - e;
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
      double e4[4] = {0.0, 0.0, 0.0, 0.0};
      if (p.layout == QGEMM_INTERLEAVED) {
        const double *e = p.X + p.width * (sr + sc * p.ld);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < p.width) e4[q] = e[q];
      } else {
        const double *e = p.X + sr + sc * p.ld;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < p.width) e4[q] = e[q * p.ps];
      }
      v = make_double4(e4[0], e4[1], e4[2], e4[3]);
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
    if (r >= p.rows || p.kw * kq >= p.kp) continue;
    const double4 v = tile[kk][rr];
    // kappa balancing: op(A) scaled by 2^-t, op(B) by 2^t (exact)
    const int tk = (p.tsign != 0 && kq < p.kq) ? p.tsign * kappa_balance(p.ka, p.kb, kq) : 0;
    const int sft = sm.shift[rr] == kNonFinite ? kNonFinite : sm.shift[rr] + tk;
    const double comp[4] = {v.x, v.y, v.z, v.w};
    long long X[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)  // a non-finite row gets digits 0 (its C entries NaN)
      X[j] = sft == kNonFinite ? 0ll : round_scaled(comp[j], sft);
    // Balanced base-256 digits as in digits6, least significant (t = 5) first,
    // so only the four remainders stay live; each digit's BF16 bits are exact
    // (|d| <= 256) and a sign flip is an XOR.
#pragma unroll
    for (int t = NSL - 1; t >= 0; --t) {
      uint32_t hb[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        long long dj = X[j];
        if (t > 0) {
          dj = ((X[j] + 128) & 255) - 128;
          X[j] = (X[j] - dj) >> 8;
        }
        hb[j] = __float_as_uint(static_cast<float>(static_cast<int>(dj))) >> 16;
      }
      if (!IS_B) {
        store_bits(p.out + t * p.slice_stride + r * p.kp + p.kw * kq, hb[0] | (hb[1] << 16),
                   hb[2] | (hb[3] << 16), p.kw);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int q = j ^ c;
            w[j] = hb[q] ^ (basis_sign(j, q) < 0 ? 0x8000u : 0u);
          }
          store_bits(p.out + t * p.slice_stride + (4 * r + c) * p.kp + p.kw * kq,
                     w[0] | (w[1] << 16), w[2] | (w[3] << 16), p.kw);
        }
      }
    }
  }
}

template <bool IS_B>
__global__ void __launch_bounds__(256) slice_kernel(const SliceArgs p) {
  __shared__ SliceSmem sm;
  slice_tile<IS_B>(p, blockIdx.x, blockIdx.y, sm);
}

// Grouped: stiles[0].x = the number of A tiles nA, then nA entries (problem,
// 0, row tile, k tile) of A operands and the B entries (problem, 1, ...).
// One launch per operand kind, so each compiles to the registers of its own
// path rather than the maximum of both (A: 40, six CTAs per SM; B: 48, five).
template <bool IS_B>
__global__ void __launch_bounds__(256, IS_B ? 5 : 6)
    grouped_slice_kernel(const SlicedProb *__restrict__ probs, const int4 *__restrict__ stiles,
                         int n) {
  __shared__ SliceSmem sm;
  const int na = stiles[0].x;
  const int lo = IS_B ? 1 + na : 1, hi = IS_B ? n : 1 + na;
  for (int t = lo + static_cast<int>(blockIdx.x); t < hi; t += gridDim.x) {
    const int4 e = stiles[t];
    slice_tile<IS_B>(IS_B ? probs[e.x].sb : probs[e.x].sa, e.z, e.w, sm);
    __syncthreads();
  }
}

// ----------------------------------------------------------- host side ---
struct SlicedPlan {
  int64_t kp;
  size_t a_off, b_off, maxa_off, maxb_off, ka_off, kb_off, ea_off, eb_off, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

SlicedPlan plan_for(const GemmDesc &d) {
  SlicedPlan s;
  s.kp = ((d.kwidth * d.k + SBK - 1) / SBK) * SBK;
  s.a_off = 0;
  const size_t a_bytes = static_cast<size_t>(NSL) * d.m * s.kp * 2;
  s.b_off = align_up(a_bytes, 1024);
  const size_t b_bytes = static_cast<size_t>(NSL) * 4 * d.n * s.kp * 2;
  s.maxa_off = align_up(s.b_off + b_bytes, 256);
  s.maxb_off = align_up(s.maxa_off + 4 * d.m, 256);
  s.ka_off = align_up(s.maxb_off + 4 * d.n, 256);
  s.kb_off = align_up(s.ka_off + 4 * d.k, 256);
  s.ea_off = align_up(s.kb_off + 4 * d.k, 256);
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

MaxArgs max_args(const MatView &v, bool by_col, int layout, int *out, int tsign = 0,
                 const int *ka = nullptr, const int *kb = nullptr) {
  MaxArgs a;
  a.tsign = tsign;
  a.ka = ka;
  a.kb = kb;
  a.X = static_cast<const double *>(v.ptr);
  a.ld = v.ld;
  a.ps = v.ps;
  a.srows = v.rows;
  a.scols = v.cols;
  a.layout = layout;
  a.by_col = by_col ? 1 : 0;
  a.width = v.width;
  a.out = out;
  return a;
}

SliceArgs slice_args(bool is_b, const MatView &v, int op, int64_t rows, int64_t kq, int64_t kp,
                     int kw, int layout, __nv_bfloat16 *out, const int *emax, int *eout,
                     int tsign = 0, const int *ka = nullptr, const int *kb = nullptr) {
  SliceArgs a;
  a.tsign = tsign;
  a.ka = ka;
  a.kb = kb;
  a.X = static_cast<const double *>(v.ptr);
  a.ld = v.ld;
  a.ps = v.ps;
  a.rows = rows;
  a.kq = kq;
  a.kp = kp;
  a.slice_stride = (is_b ? 4 * rows : rows) * kp;
  a.out = out;
  a.emax = emax;
  a.eout = eout;
  a.layout = layout;
  a.row_contig = is_b ? (op_trans(op) ? 1 : 0) : (op_trans(op) ? 0 : 1);
  a.negmask = op_conj(op) ? 0xEu : 0u;
  a.width = v.width;
  a.kw = kw;
  return a;
}

// Row maxima of op(A): stored rows for N/C, stored columns for T/H; column
// maxima of op(B): stored columns for N/C, stored rows for T/H.
bool max_by_col(bool is_b, int op) { return is_b ? !op_trans(op) : op_trans(op); }

int launch_max(const MaxArgs &a, cudaStream_t stream) {
  const int64_t gx = (a.srows + 31) / 32, gy = (a.scols + 31) / 32;
  if (gx == 0 || gy == 0) return QGEMM_SUCCESS;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  slice_max_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), 256, 0,
                     stream>>>(a);
  return launch_status();
}

int launch_slices(bool is_b, const SliceArgs &a, cudaStream_t stream) {
  const int64_t gx = (a.rows + 31) / 32, gy = (a.kp / a.kw + 31) / 32;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (is_b)
    slice_kernel<true><<<grid, 256, 0, stream>>>(a);
  else
    slice_kernel<false><<<grid, 256, 0, stream>>>(a);
  return launch_status();
}

SlicedParams params_for(const GemmDesc &d, int64_t kp, const int *ea, const int *eb) {
  SlicedParams g{};
  g.m = d.m;
  g.n = d.n;
  g.num_kb = static_cast<int>(d.k > 0 ? kp / SBK : 0);
  g.num_mt = static_cast<int>((d.m + SBM - 1) / SBM);
  g.num_nt = static_cast<int>((d.n + SBNQ - 1) / SBNQ);
  g.layout = d.layout;
  g.beta_zero = d.beta_zero ? 1 : 0;
  g.tri = d.tri;
  g.swap = 0;
  g.alpha_real = (d.alpha[1] == 0.0 && d.alpha[2] == 0.0 && d.alpha[3] == 0.0) ? 1 : 0;
  g.beta_real = (d.beta[1] == 0.0 && d.beta[2] == 0.0 && d.beta[3] == 0.0) ? 1 : 0;
  g.krange = d.krange;
  g.swap = d.swap;
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
  return g;
}

template <bool GROUPED>
int set_gemm_smem() {
  static bool done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(sliced_gemm_kernel<GROUPED>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmem)) != cudaSuccess)
      return launch_status();
    done[dev] = true;
  }
  return QGEMM_SUCCESS;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// K shares of a single problem (one CTA per SM, tiles of SBM x SBNQ
// quaternions): when C has fewer than 8 waves of tiles, the fewest shares s in
// [2, 256] whose tiles x s CTAs fill their waves to within 2 % of the best s,
// with at least 32 k-blocks (256 quaternion k, 4 chunks) per share, if the
// best beats s = 1 by 5 % and s = 1 keeps at most half of the SMs busy.  Plain products only (no triangle, k-range or
// turned-around problem).  1: no split.
int sliced_ksplit(const GemmDesc &d, int sms) {
  if (d.tri || d.krange || d.swap || d.m <= 0 || d.n <= 0 || d.k <= 0) return 1;
  const int64_t tiles = ((d.m + SBM - 1) / SBM) * ((d.n + SBNQ - 1) / SBNQ);
  const int64_t slots = sms;
  if (tiles >= 8 * slots) return 1;
  const int64_t num_kb = ((d.kwidth * d.k + SBK - 1) / SBK * SBK) / SBK;
  const int64_t smax = std::min<int64_t>(256, num_kb / 32);
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

// Required: the slices, maxima and exponents (plan_for).
int sliced_workspace_bytes(const GemmDesc &d, size_t *bytes) {
  *bytes = (d.k == 0 || d.m == 0 || d.n == 0) ? 0 : plan_for(d).total;
  return QGEMM_SUCCESS;
}

// Optional, after the required part: the K shares' partial products of a
// product that splits K (0 when it does not).
size_t sliced_splitk_bytes(const GemmDesc &d) {
  if (d.k == 0 || d.m == 0 || d.n == 0) return 0;
  const int ks = sliced_ksplit(d, device_sms());
  return ks > 1 ? static_cast<size_t>(ks) * d.m * d.n * 32 : 0;
}

int launch_sliced_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (d.k > kMaxSlicedK) return QGEMM_ERR_UNSUPPORTED;
  const SlicedPlan pl = plan_for(d);
  if (ws == nullptr || ws_bytes < pl.total) return QGEMM_ERR_WORKSPACE;
  unsigned char *w = static_cast<unsigned char *>(ws);
  auto *wa = reinterpret_cast<__nv_bfloat16 *>(w + pl.a_off);
  auto *wb = reinterpret_cast<__nv_bfloat16 *>(w + pl.b_off);
  int *maxa = reinterpret_cast<int *>(w + pl.maxa_off);
  int *maxb = reinterpret_cast<int *>(w + pl.maxb_off);
  int *ka = reinterpret_cast<int *>(w + pl.ka_off);
  int *kb = reinterpret_cast<int *>(w + pl.kb_off);
  int *ea = reinterpret_cast<int *>(w + pl.ea_off);
  int *eb = reinterpret_cast<int *>(w + pl.eb_off);

  // every maximum starts at kExpEmpty (bytes 0x80)
  if (cudaMemsetAsync(w + pl.maxa_off, 0x80, pl.ea_off - pl.maxa_off, stream) != cudaSuccess)
    return launch_status();
  // per-kappa exponents of op(A) and op(B), then the balanced row / column
  // exponents, then the balanced slices
  int rc = launch_max(max_args(d.A, !max_by_col(false, d.opA), d.layout, ka), stream);
  if (rc) return rc;
  rc = launch_max(max_args(d.B, !max_by_col(true, d.opB), d.layout, kb), stream);
  if (rc) return rc;
  rc = launch_max(max_args(d.A, max_by_col(false, d.opA), d.layout, maxa, -1, ka, kb), stream);
  if (rc) return rc;
  rc = launch_max(max_args(d.B, max_by_col(true, d.opB), d.layout, maxb, 1, ka, kb), stream);
  if (rc) return rc;
  rc = launch_slices(false, slice_args(false, d.A, d.opA, d.m, d.k, pl.kp, d.kwidth, d.layout, wa,
                                      maxa, ea, -1, ka, kb),
                     stream);
  if (rc) return rc;
  rc = launch_slices(true, slice_args(true, d.B, d.opB, d.n, d.k, pl.kp, d.kwidth, d.layout, wb,
                                      maxb, eb, 1, ka, kb),
                     stream);
  if (rc) return rc;

  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  if (!encode_slices(&tmA, wa, pl.kp, d.m, SBM) || !encode_slices(&tmB, wb, pl.kp, 4 * d.n, SBN))
    return QGEMM_ERR_UNSUPPORTED;
  SlicedParams g = params_for(d, pl.kp, ea, eb);
  // K shares: as many as chosen for this device that fit after the plan
  int ks = sliced_ksplit(d, sm_count());
  if (ks > 1) {
    const size_t per = static_cast<size_t>(d.m) * d.n * 32;
    const int64_t fit = static_cast<int64_t>((ws_bytes - pl.total) / per);
    if (fit < ks) ks = static_cast<int>(fit);
    if (ks > 1) {
      g.ksplit = ks;
      g.part = reinterpret_cast<double *>(w + pl.total);
    } else {
      ks = 1;
    }
  }
  const int64_t tiles = static_cast<int64_t>(g.num_mt) * g.num_nt * ks;
  if (tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  rc = set_gemm_smem<false>();
  if (rc) return rc;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, sm_count()));
  sliced_gemm_kernel<false><<<grid, kSThreads, kSmem, stream>>>(
      tmA, tmB, g, nullptr, nullptr, static_cast<int>(tiles), wait_limit_ns());
  rc = launch_status();
  if (rc || ks == 1) return rc;
  return launch_splitk_reduce(d, g.part, ks, stream);
}

// ---------------------------------------------------- grouped batches ---
namespace {

// (op(X))^H = op'(X).
int op_conjtrans(int op) {
  switch (op) {
    case QGEMM_OP_N: return QGEMM_OP_H;
    case QGEMM_OP_H: return QGEMM_OP_N;
    case QGEMM_OP_T: return QGEMM_OP_C;
    default: return QGEMM_OP_T;
  }
}

// (AB)^H = B^H A^H (Sec. 2.2): a problem is computed as D = op(B)^H op(A)^H
// and stored as C = conj(D)^T when that pads less (tile rows are padded to
// 128, columns to 16).
GemmDesc oriented(const GemmDesc &d, bool *swapped) {
  auto padded = [](int64_t r, int64_t c) {
    return ((r + SBM - 1) / SBM) * SBM * (((c + SBNQ - 1) / SBNQ) * SBNQ);
  };
  *swapped = d.k > 0 && padded(d.n, d.m) < padded(d.m, d.n);
  if (!*swapped) return d;
  GemmDesc t = d;
  t.m = d.n;
  t.n = d.m;
  t.opA = op_conjtrans(d.opB);
  t.opB = op_conjtrans(d.opA);
  t.A = d.B;
  t.B = d.A;
  return t;
}

constexpr size_t kGroupedHeader = 256;

struct GroupedLayout {
  size_t desc_off, tile_off, mtile_off, stile_off, max_off, exp_off, data_off, total;
  int64_t tiles, mtiles, stiles;
  std::vector<size_t> maxa, maxb, ea, eb, a_off, b_off;  // per problem, from the workspace
  std::vector<int64_t> kp;
  std::vector<GemmDesc> ds;
  std::vector<int> swapped;
};

GroupedLayout grouped_layout(const std::vector<GemmDesc> &in) {
  GroupedLayout L{};
  const size_t P = in.size();
  L.ds.resize(P);
  L.swapped.assign(P, 0);
  L.maxa.assign(P, 0);
  L.maxb.assign(P, 0);
  L.ea.assign(P, 0);
  L.eb.assign(P, 0);
  L.a_off.assign(P, 0);
  L.b_off.assign(P, 0);
  L.kp.assign(P, 0);
  L.stiles = 1;  // the slicing list's header entry (number of A tiles)
  size_t maxb_total = 0, exp_total = 0, data = 0;
  for (size_t p = 0; p < P; ++p) {
    bool sw = false;
    L.ds[p] = oriented(in[p], &sw);
    L.swapped[p] = sw ? 1 : 0;
    const GemmDesc &d = L.ds[p];
    L.kp[p] = ((4 * d.k + SBK - 1) / SBK) * SBK;
    if (d.m == 0 || d.n == 0) continue;
    L.tiles += ((d.m + SBM - 1) / SBM) * ((d.n + SBNQ - 1) / SBNQ);
    L.ea[p] = exp_total;
    L.eb[p] = exp_total + 4 * d.m;
    exp_total += 4 * (d.m + d.n);
    if (d.k == 0) continue;
    L.maxa[p] = maxb_total;
    L.maxb[p] = maxb_total + 8 * d.m;
    maxb_total += 8 * (d.m + d.n);
    L.mtiles += ((d.A.rows + 31) / 32) * ((d.A.cols + 31) / 32) +
                ((d.B.rows + 31) / 32) * ((d.B.cols + 31) / 32);
    const int64_t kt = (L.kp[p] / 4 + 31) / 32;
    L.stiles += ((d.m + 31) / 32) * kt + ((d.n + 31) / 32) * kt;
    L.a_off[p] = data;
    data = align_up(data + static_cast<size_t>(NSL) * d.m * L.kp[p] * 2, 1024);
    L.b_off[p] = data;
    data = align_up(data + static_cast<size_t>(NSL) * 4 * d.n * L.kp[p] * 2, 1024);
  }
  L.desc_off = kGroupedHeader;
  L.tile_off = align_up(L.desc_off + P * sizeof(SlicedProb), 256);
  L.mtile_off = align_up(L.tile_off + static_cast<size_t>(L.tiles) * sizeof(int4), 256);
  L.stile_off = align_up(L.mtile_off + static_cast<size_t>(L.mtiles) * sizeof(int4), 256);
  L.max_off = align_up(L.stile_off + static_cast<size_t>(L.stiles) * sizeof(int4), 256);
  L.exp_off = align_up(L.max_off + maxb_total, 256);
  L.data_off = align_up(L.exp_off + exp_total, 1024);
  L.total = L.data_off + data;
  for (size_t p = 0; p < P; ++p) {
    L.maxa[p] += L.max_off;
    L.maxb[p] += L.max_off;
    L.ea[p] += L.exp_off;
    L.eb[p] += L.exp_off;
    L.a_off[p] += L.data_off;
    L.b_off[p] += L.data_off;
  }
  return L;
}

}  // namespace

size_t sliced_grouped_workspace_bytes(const std::vector<GemmDesc> &ds) {
  return grouped_layout(ds).total;
}

int prepare_sliced_grouped(const std::vector<GemmDesc> &in, int layout, unsigned char *ws,
                           size_t ws_bytes, cudaStream_t s, qgemm_grouped_plan *plan) {
  const GroupedLayout L = grouped_layout(in);
  if (ws_bytes < L.total) return -6;
  for (const GemmDesc &d : in)
    if (d.k > kMaxSlicedK) return QGEMM_ERR_UNSUPPORTED;
  if (L.tiles > 0x7fffffff || L.mtiles > 0x7fffffff || L.stiles > 0x7fffffff)
    return QGEMM_ERR_UNSUPPORTED;
  int rc = set_gemm_smem<true>();
  if (rc) return rc;
  std::vector<unsigned char> host(L.max_off - L.desc_off, 0);
  auto *hd = reinterpret_cast<SlicedProb *>(host.data());
  std::vector<int4> tiles, mtiles, stiles, stiles_b;
  std::vector<int> tile_kb;
  stiles.push_back(make_int4(0, 0, 0, 0));  // header: the number of A tiles
  for (size_t p = 0; p < L.ds.size(); ++p) {
    const GemmDesc &d = L.ds[p];
    if (d.m == 0 || d.n == 0) continue;
    SlicedProb &q = hd[p];
    const int64_t kp = L.kp[p];
    auto *wa = reinterpret_cast<__nv_bfloat16 *>(ws + L.a_off[p]);
    auto *wb = reinterpret_cast<__nv_bfloat16 *>(ws + L.b_off[p]);
    auto *maxa = reinterpret_cast<int *>(ws + L.maxa[p]);
    auto *maxb = reinterpret_cast<int *>(ws + L.maxb[p]);
    int *ea = reinterpret_cast<int *>(ws + L.ea[p]);
    int *eb = reinterpret_cast<int *>(ws + L.eb[p]);
    GemmDesc dl = d;
    dl.layout = layout;
    q.g = params_for(dl, kp, ea, eb);
    q.g.swap = L.swapped[p];
    if (d.k > 0) {
      const bool bca = max_by_col(false, d.opA), bcb = max_by_col(true, d.opB);
      q.ma = max_args(d.A, bca, layout, maxa);
      q.mb = max_args(d.B, bcb, layout, maxb);
      q.sa = slice_args(false, d.A, d.opA, d.m, d.k, kp, 4, layout, wa, maxa, ea);
      q.sb = slice_args(true, d.B, d.opB, d.n, d.k, kp, 4, layout, wb, maxb, eb);
      if (!encode_slices(&q.tmA, wa, kp, d.m, SBM) || !encode_slices(&q.tmB, wb, kp, 4 * d.n, SBN))
        return QGEMM_ERR_UNSUPPORTED;
      const MatView *v[2] = {&d.A, &d.B};
      for (int o = 0; o < 2; ++o)
        for (int64_t r = 0; r < (v[o]->rows + 31) / 32; ++r)
          for (int64_t c = 0; c < (v[o]->cols + 31) / 32; ++c)
            mtiles.push_back(make_int4(static_cast<int>(p), o, static_cast<int>(r),
                                       static_cast<int>(c)));
      const int64_t kt = (kp / 4 + 31) / 32;
      for (int64_t r = 0; r < (d.m + 31) / 32; ++r)
        for (int64_t c = 0; c < kt; ++c)
          stiles.push_back(make_int4(static_cast<int>(p), 0, static_cast<int>(r),
                                     static_cast<int>(c)));
      for (int64_t r = 0; r < (d.n + 31) / 32; ++r)
        for (int64_t c = 0; c < kt; ++c)
          stiles_b.push_back(make_int4(static_cast<int>(p), 1, static_cast<int>(r),
                                       static_cast<int>(c)));
    }
    for (int a = 0; a < q.g.num_mt; ++a)
      for (int b = 0; b < q.g.num_nt; ++b) {
        tiles.push_back(make_int4(static_cast<int>(p), a, b, 0));
        tile_kb.push_back(q.g.num_kb);
      }
  }
  // longest tiles first; CTAs take tiles t, t + grid, ...
  std::vector<int32_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int32_t>(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return tile_kb[a] > tile_kb[b]; });
  int4 *ht = reinterpret_cast<int4 *>(host.data() + (L.tile_off - L.desc_off));
  for (size_t i = 0; i < order.size(); ++i) ht[i] = tiles[order[i]];
  std::memcpy(host.data() + (L.mtile_off - L.desc_off), mtiles.data(),
              mtiles.size() * sizeof(int4));
  stiles[0].x = static_cast<int>(stiles.size() - 1);
  stiles.insert(stiles.end(), stiles_b.begin(), stiles_b.end());
  if (static_cast<int64_t>(stiles.size()) != L.stiles) return QGEMM_ERR_UNSUPPORTED;
  std::memcpy(host.data() + (L.stile_off - L.desc_off), stiles.data(),
              stiles.size() * sizeof(int4));
  if (!host.empty() && cudaMemcpyAsync(ws + L.desc_off, host.data(), host.size(),
                                       cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  const int sms = sm_count();
  plan->workspace_bytes = L.total;
  plan->tiles = L.tiles;
  plan->grid = static_cast<int32_t>(std::min<int64_t>(std::max<int64_t>(L.tiles, 1), sms));
  // pre-pass CTAs (grid-stride over the tile lists): many small tiles, so up
  // to 64 CTAs per SM keep more of them in flight than 8 do
  plan->reserved0 = 64 * sms;
  plan->desc_offset = static_cast<int64_t>(L.desc_off);
  plan->tile_offset = static_cast<int64_t>(L.tile_off);
  plan->data_offset = static_cast<int64_t>(L.max_off);
  plan->reserved[0] = static_cast<int64_t>(L.mtile_off);
  plan->reserved[1] = L.mtiles | (L.stiles << 32);
  plan->reserved[2] = static_cast<int64_t>(L.stile_off);
  plan->reserved[3] = static_cast<int64_t>(L.exp_off - L.max_off);
  return QGEMM_SUCCESS;
}

int launch_sliced_grouped(const qgemm_grouped_plan *plan, cudaStream_t s) {
  int rc = set_gemm_smem<true>();
  if (rc) return rc;
  unsigned char *ws = static_cast<unsigned char *>(plan->workspace);
  const auto *probs = reinterpret_cast<const SlicedProb *>(ws + plan->desc_offset);
  const auto *tiles = reinterpret_cast<const int4 *>(ws + plan->tile_offset);
  const auto *mtiles = reinterpret_cast<const int4 *>(ws + plan->reserved[0]);
  const auto *stiles = reinterpret_cast<const int4 *>(ws + plan->reserved[2]);
  const int nm = static_cast<int>(plan->reserved[1] & 0xffffffff);
  const int ns = static_cast<int>(plan->reserved[1] >> 32);
  if (plan->reserved[3] > 0 &&
      cudaMemsetAsync(ws + plan->data_offset, 0x80, static_cast<size_t>(plan->reserved[3]), s) !=
          cudaSuccess)
    return launch_status();
  const int pgrid = plan->reserved0 > 0 ? plan->reserved0 : 1;
  if (nm > 0) grouped_slice_max_kernel<<<std::min(nm, pgrid), 256, 0, s>>>(probs, mtiles, nm);
  if (ns > 1) {  // entry 0 is the header
    grouped_slice_kernel<false><<<std::min(ns - 1, pgrid), 256, 0, s>>>(probs, stiles, ns);
    grouped_slice_kernel<true><<<std::min(ns - 1, pgrid), 256, 0, s>>>(probs, stiles, ns);
  }
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  const SlicedParams unused{};
  sliced_gemm_kernel<true><<<plan->grid, kSThreads, kSmem, s>>>(
      none, none, unused, probs, tiles, static_cast<int>(plan->tiles), wait_limit_ns());
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
