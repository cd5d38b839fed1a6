// One output tile of the FP64 quaternion GEMM on DMMA tensor cores, shared by
// the single-problem kernel and the persistent grouped kernel.
//
// Real form: (a b)^c = sum_j L(a)[c][j] b^j with L(a)[c][j] =
// sign(c xor j, j) a^(c xor j) (Sec. 2.1, Eq. quaternion_prod), so the tile
// is C_r = L(op(A)) B_r over the real K = 4k.  An m16n8k4 DMMA covers 4
// quaternion rows (16 real rows: row 4i + c), 8 quaternion columns and one
// quaternion k element (4 real k: column j); its A fragment is gathered from
// the staged op(A) tile with the sign of L(a) applied as an integer XOR.
//
// The CTA has 4 warps arranged WARPS_M x WARPS_N over a BMQ x BNQ tile; each
// warp owns 8 quaternion rows and BNQ / WARPS_N columns.  Tiles of 16
// quaternion k pass through a STAGES-deep shared-memory ring filled by TMA
// (3-D boxes: component x row x column for interleaved data, row x column x
// plane for split planes; zero fill past the edges) or by plain loads when a
// base or stride is not 16-byte aligned.  Ring slots and barrier phases are
// counted by a running k-block index so a persistent CTA can continue across
// tiles.
#pragma once
#include "common.cuh"

namespace qg {
namespace fp64 {

constexpr int kBKQ = 16;
constexpr int kStages = 3;
constexpr int kThreads = 128;
constexpr int kMaxTileElems = 32 * kBKQ * 4;  // largest A or B tile (doubles)
constexpr uint32_t kMaxTileBytes = kMaxTileElems * sizeof(double);
constexpr size_t kSmemBytes = 2 * kStages * kMaxTileBytes + kStages * sizeof(uint64_t) + 16;

// Operands of one problem as the tile code reads them.
struct Operands {
  const double *A;
  int64_t a_rows, a_cols, lda, psA;
  const double *B;
  int64_t b_rows, b_cols, ldb, psB;
  double *C;
  int64_t ldc, psC;
  int64_t m, n, k;
  double alpha[4], beta[4];
  uint32_t negmask;
  int tmaA, tmaB, beta_zero;
  int tri;  // 0 full; 1 lower (row >= col) only; 2 upper; diagonal written real
  int krange;  // k-range of a tile when op(A) or op(B) is triangular (see GemmDesc)
  int swap;    // 1: the tile holds D = (op(A) op(B))^H; store C = conj(D)^T
  // K split across blockIdx.z (single-problem kernel only): CTA z sums its
  // share of the k-blocks and stores that partial product, four doubles per
  // quaternion, to part + z m n 4 (dense, interleaved, leading dimension m);
  // a second kernel sums the ksplit partials and applies alpha and beta.
  int ksplit;  // 0 or 1: no split
  double *part;
  // Fault injection (tests of the bounded waits): > 0 makes the first CTA of
  // the launch leave out the copies of its ring stage debug_skip - 1.
  int debug_skip;
};

// True when the tile at quaternion offset (i0, n0) of size BMQ x BNQ has no
// element in the stored triangle.
__device__ __forceinline__ bool tile_outside(int tri, int64_t i0, int64_t n0, int bm, int bn) {
  if (tri == 1) return i0 + bm - 1 < n0;
  if (tri == 2) return n0 + bn - 1 < i0;
  return false;
}

// Shared-memory index of component s of stored element (r, c) of a tile with
// R stored rows and CC stored columns (the TMA box order); W components per
// element (4 quaternion, 2 complex, 1 real).
template <int LAYOUT, int R, int CC, int W = 4>
__device__ __forceinline__ int tile_idx(int r, int c, int s) {
  if (LAYOUT == QGEMM_INTERLEAVED) return s + W * (r + R * c);
  return r + R * (c + CC * s);
}

template <int LAYOUT, int R, int CC, int W = 4>
__device__ void load_tile_plain(double *dst, const double *base, int64_t rows, int64_t cols,
                                int64_t ld, int64_t ps, int64_t r0, int64_t c0) {
  constexpr int N = R * CC * W;
  for (int e = threadIdx.x; e < N; e += kThreads) {
    int r, c, s;
    if (LAYOUT == QGEMM_INTERLEAVED) {
      s = e % W;
      const int rest = e / W;
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
      v = LAYOUT == QGEMM_INTERLEAVED ? base[W * (gr + gc * ld) + s] : base[s * ps + gr + gc * ld];
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

__device__ __forceinline__ void tma_box(double *dst, const CUtensorMap *map, uint64_t *bar,
                                        int layout, int64_t r0, int64_t c0) {
  if (layout == QGEMM_INTERLEAVED)
    tma_load_3d(dst, map, bar, 0, static_cast<int>(r0), static_cast<int>(c0));
  else
    tma_load_3d(dst, map, bar, static_cast<int>(r0), static_cast<int>(c0), 0);
}

// Computes and stores one BMQ x BNQ tile at quaternion offset (i0, n0).
// kb_run counts k-blocks consumed by this CTA so far (ring slot and barrier
// phase).  Returns false if a bounded wait gave up (after draining its own
// copies); the caller then stops.
// WB: components of op(B)'s elements (4; 2 or 1 for a complex or real right
// factor, loaded with plain loads).  Then b^j = 0 for j >= WB, and one DMMA's
// k = 4 spans 4 / WB values of kappa: lane k-index t is kappa offset t / WB,
// component j = t % WB, and L(a)[c][j] is gathered for that (kappa, j).
template <int LAYOUT, bool TA, bool TB, int BMQ, int BNQ, int WB = 4>
__device__ bool tile(const Operands &p, const CUtensorMap *tmA, const CUtensorMap *tmB,
                     double *sA, double *sB, uint64_t *full, uint32_t &kb_run, int64_t i0,
                     int64_t n0, uint64_t limit_ns, int *err_word) {
  constexpr int WARPS_M = BMQ / 8;
  constexpr int WARPS_N = 4 / WARPS_M;
  constexpr int WN = BNQ / WARPS_N;  // quaternion columns per warp
  constexpr int NC = WN / 8;         // m16n8k4 column blocks per warp
  static_assert(WARPS_M * WARPS_N == 4 && NC >= 1 && WN % 8 == 0, "tile shape");
  constexpr int A_R = TA ? kBKQ : BMQ, A_C = TA ? BMQ : kBKQ;
  constexpr int B_R = TB ? BNQ : kBKQ, B_C = TB ? kBKQ : BNQ;
  constexpr uint32_t kABytes = BMQ * kBKQ * 4 * sizeof(double);
  constexpr uint32_t kBBytes = BNQ * kBKQ * 4 * sizeof(double);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp % WARPS_M, wn = warp / WARPS_M;
  // k-blocks [kt_lo, kt_lo + ktiles): all of K, or the part where a
  // triangular operand can be nonzero for this tile's rows or columns
  int kt_lo = 0, kt_hi = static_cast<int>((p.k + kBKQ - 1) / kBKQ);
  if (p.krange == 1) kt_hi = min(kt_hi, static_cast<int>((i0 + BMQ + kBKQ - 1) / kBKQ));
  if (p.krange == 2) kt_lo = static_cast<int>(i0 / kBKQ);
  if (p.krange == 3) kt_lo = static_cast<int>(n0 / kBKQ);
  if (p.krange == 4) kt_hi = min(kt_hi, static_cast<int>((n0 + BNQ + kBKQ - 1) / kBKQ));
  if (p.ksplit > 1) {  // this CTA's share of the k-blocks
    const int64_t span = kt_hi > kt_lo ? kt_hi - kt_lo : 0, z = blockIdx.z;
    const int lo = kt_lo + static_cast<int>(span * z / p.ksplit);
    kt_hi = kt_lo + static_cast<int>(span * (z + 1) / p.ksplit);
    kt_lo = lo;
  }
  const int ktiles = kt_hi > kt_lo ? kt_hi - kt_lo : 0;
  const uint32_t tx_bytes = (p.tmaA ? kABytes : 0u) + (p.tmaB ? kBBytes : 0u);

  // Every k-block arrives on its ring slot's barrier, with the TMA byte count
  // (0 when both operands use plain loads): barrier phases then follow the
  // running k-block count even when a persistent CTA mixes TMA and
  // plain-load problems.
  auto issue = [&](int kt) {
    const uint32_t q = kb_run + kt;
    const int st = q % kStages;
    if (p.debug_skip > 0 && q == static_cast<uint32_t>(p.debug_skip - 1) && blockIdx.x == 0 &&
        blockIdx.y == 0 && blockIdx.z == 0)
      return;
    mbar_arrive_expect_tx(&full[st], tx_bytes);
    const int64_t kk0 = static_cast<int64_t>(kt_lo + kt) * kBKQ;
    if (p.tmaA) tma_box(sA + st * kMaxTileElems, tmA, &full[st], LAYOUT, TA ? kk0 : i0, TA ? i0 : kk0);
    if (p.tmaB) tma_box(sB + st * kMaxTileElems, tmB, &full[st], LAYOUT, TB ? n0 : kk0, TB ? kk0 : n0);
  };
  if (tid == 0)
    for (int s = 0; s < kStages && s < ktiles; ++s) issue(s);

  const int c_lane = g & 3;
  const int compA = c_lane ^ t;
  const uint32_t negA = ((p.negmask >> (4 * c_lane + t)) & 1u) << 31;
  const int arow = wm * 8 + (g >> 2);
  const int bcol = wn * WN + g;

  // DMMA blocks (4 quaternion rows x 8 columns) entirely past the edge of C
  // are skipped, and so are k steps past k: ragged problems pay only for the
  // DMMA granularity, not for the whole tile (warp-uniform conditions)
  bool row_live[2], col_live[NC];
#pragma unroll
  for (int r = 0; r < 2; ++r) row_live[r] = i0 + wm * 8 + 4 * r < p.m;
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) col_live[cc] = n0 + wn * WN + 8 * cc < p.n;

  double acc[2][NC][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[r][cc][e] = 0.0;

  for (int kt = 0; kt < ktiles; ++kt) {
    const uint32_t q = kb_run + kt;
    const int st = q % kStages;
    const uint32_t par = (q / kStages) & 1;
    const int64_t kk0 = static_cast<int64_t>(kt_lo + kt) * kBKQ;
    double *a_t = sA + st * kMaxTileElems;
    double *b_t = sB + st * kMaxTileElems;
    if (!p.tmaA)
      load_tile_plain<LAYOUT, A_R, A_C>(a_t, p.A, p.a_rows, p.a_cols, p.lda, p.psA,
                                        TA ? kk0 : i0, TA ? i0 : kk0);
    if (!p.tmaB)
      load_tile_plain<LAYOUT, B_R, B_C, WB>(b_t, p.B, p.b_rows, p.b_cols, p.ldb, p.psB,
                                            TB ? n0 : kk0, TB ? kk0 : n0);
    const bool ok = mbar_wait_bounded(&full[st], par, limit_ns);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicCAS(err_word, 0, QGEMM_ERR_TIMEOUT);
        for (int r = kt; r < ktiles && r < kt + kStages; ++r) {
          const uint32_t qq = kb_run + r;
          mbar_wait_bounded(&full[qq % kStages], (qq / kStages) & 1, limit_ns);
        }
      }
      return false;
    }
    const int kk_end = static_cast<int>(min(static_cast<int64_t>(kBKQ), p.k - kk0));
    if (WB == 4) {
#pragma unroll 4
      for (int kk = 0; kk < kk_end; ++kk) {
        double a[2][2], b[NC];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int i = arow + 4 * r;
          a[r][0] = flip_sign(a_t[TA ? tile_idx<LAYOUT, A_R, A_C>(kk, i, compA)
                                     : tile_idx<LAYOUT, A_R, A_C>(i, kk, compA)], negA);
          a[r][1] = flip_sign(a_t[TA ? tile_idx<LAYOUT, A_R, A_C>(kk, i + 2, compA)
                                     : tile_idx<LAYOUT, A_R, A_C>(i + 2, kk, compA)], negA);
        }
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
          const int j = bcol + 8 * cc;
          b[cc] = b_t[TB ? tile_idx<LAYOUT, B_R, B_C>(j, kk, t) : tile_idx<LAYOUT, B_R, B_C>(kk, j, t)];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (!row_live[r]) continue;
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) {
            if (!col_live[cc]) continue;
            dmma_16x8x4(acc[r][cc], a[r][0], a[r][1], b[cc]);
          }
        }
      }
    } else {
      // narrow right factor: this lane's (kappa offset, component j) per step;
      // steps past k read the zero fill of the tiles
      constexpr int KPS = 4 / WB;
      const int jw = t % WB, kofs = t / WB;
      const int compW = c_lane ^ jw;
      const uint32_t negW = ((p.negmask >> (4 * c_lane + jw)) & 1u) << 31;
      const int nsteps = (kk_end + KPS - 1) / KPS;
#pragma unroll 2
      for (int stp = 0; stp < nsteps; ++stp) {
        const int kk = stp * KPS + kofs;
        double a[2][2], b[NC];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int i = arow + 4 * r;
          a[r][0] = flip_sign(a_t[TA ? tile_idx<LAYOUT, A_R, A_C>(kk, i, compW)
                                     : tile_idx<LAYOUT, A_R, A_C>(i, kk, compW)], negW);
          a[r][1] = flip_sign(a_t[TA ? tile_idx<LAYOUT, A_R, A_C>(kk, i + 2, compW)
                                     : tile_idx<LAYOUT, A_R, A_C>(i + 2, kk, compW)], negW);
        }
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
          const int j = bcol + 8 * cc;
          b[cc] = b_t[TB ? tile_idx<LAYOUT, B_R, B_C, WB>(j, kk, jw)
                         : tile_idx<LAYOUT, B_R, B_C, WB>(kk, j, jw)];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (!row_live[r]) continue;
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) {
            if (!col_live[cc]) continue;
            dmma_16x8x4(acc[r][cc], a[r][0], a[r][1], b[cc]);
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && kt + kStages < ktiles) issue(kt + kStages);
  }
  kb_run += ktiles;

  if (p.ksplit > 1) {  // partial product of this K share: each lane its component
    double *slab = p.part + static_cast<int64_t>(blockIdx.z) * p.m * p.n * 4;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t qi = i0 + arow + 4 * r + 2 * (e >> 1);
          const int64_t qn = n0 + wn * WN + 8 * cc + 2 * t + (e & 1);
          if (qi < p.m && qn < p.n) slab[4 * (qi + qn * p.m) + c_lane] = acc[r][cc][e];
        }
    return true;
  }

  // epilogue: C <- alpha P + beta C, left products, FP64
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
    for (int cc = 0; cc < NC; ++cc)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t qi = i0 + arow + 4 * r + 2 * (e >> 1);
        const int64_t qn = n0 + wn * WN + 8 * cc + 2 * t + (e & 1);
        bool inb = qi < p.m && qn < p.n;
        if (p.tri == 1) inb = inb && qi >= qn;
        if (p.tri == 2) inb = inb && qi <= qn;
        double P[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = __shfl_sync(0xffffffffu, acc[r][cc][e], src_base | (j << 2));
        // a turned-around problem holds D = (op(A) op(B))^H: C = conj(D)^T
        int64_t ci = qi, cj = qn;
        if (p.swap) {
          ci = qn;
          cj = qi;
          P[1] = -P[1];
          P[2] = -P[2];
          P[3] = -P[3];
        }
        double out = la[0] * P[0];
        out = fma(la[1], P[1], out);
        out = fma(la[2], P[2], out);
        out = fma(la[3], P[3], out);
        double *dst = LAYOUT == QGEMM_INTERLEAVED ? p.C + 4 * (ci + cj * p.ldc) + c_lane
                                                  : p.C + c_lane * p.psC + ci + cj * p.ldc;
        if (!p.beta_zero) {
          const double cin = inb ? *dst : 0.0;
          double Cq[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) Cq[j] = __shfl_sync(0xffffffffu, cin, src_base | (j << 2));
#pragma unroll
          for (int j = 0; j < 4; ++j) out = fma(lb[j], Cq[j], out);
        }
        if (p.tri && qi == qn && c_lane != 0) out = 0.0;  // Hermitian diagonal is real
        if (inb) *dst = out;
      }
  return true;
}

}  // namespace fp64
}  // namespace qg
