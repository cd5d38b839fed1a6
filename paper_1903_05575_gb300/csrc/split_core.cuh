// Split-BF16 quaternion GEMM on the fifth-generation tensor cores (tcgen05):
// device code shared by the single-problem path (split_bf16.cu) and the
// grouped path (grouped.cu).
//
// Real form.  With a = op(A)_{i kappa}, b = op(B)_{kappa n}, the Hamilton
// product (Sec. 2.1, Eq. quaternion_prod) is linear in a:
//     (a b)^c = sum_j sign(j, j xor c) a^j b^(j xor c),
// sign(p, q) the sign of the basis product e_p e_q (Eq. quaternion_alg).  So
//     C'(m x 4n) = A'(m x 4k) * B'(4k x 4n),
//     A'[i][4 kappa + j]         = a^j                                (A as stored)
//     B'[4 kappa + j][4 n + c]   = sign(j, j xor c) b^(j xor c)       (B expanded)
//     C'[i][4 n + c]             = (op(A) op(B))_{i n}^c
// which is one real GEMM with exactly the 16 m n k multiplies of the
// quaternion product; conjugation of A or B only flips signs of A' / B'.
//
// Precision.  Each FP32 value x is split into three BF16 terms by
// round-to-nearest: hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid)
// (both differences exact in FP32).  The six leading term products
// hh, hm, mh, hl, mm, lh run on tcgen05.mma kind::f16 (BF16 in, FP32 out in
// tensor memory); mid*lo, lo*mid and lo*lo (relative size 2^-24) are dropped.
// The FP32 tensor-memory accumulator is drained every `chunk` k-blocks into a
// register accumulator (two TMEM buffers, so the MMAs never wait for the
// drain); the tensor core's in-accumulator additions are biased, so the
// chunk is short and the register sum takes the rest.  The epilogue forms
// alpha P and beta C in FP32 and sums them in FP64 before the one rounding.
//
// Kernel.  Persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ...; one
// warp issues TMA loads (3-D boxes: K x rows x term, 64-byte swizzle) into a
// 3-stage ring, one warp issues the MMAs (M=128, N=256, K=16) into one of two
// TMEM accumulators and commits them to mbarriers, eight warps drain TMEM and
// run the epilogue of a tile while the MMAs of the next one proceed.  Ring
// slots, barrier phases and TMEM buffers are indexed by running counters that
// continue across tiles.  Every wait is bounded.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace qg {
namespace split {

// ---------------------------------------------------------------- sizes ---
constexpr int BM = 128;            // rows of C per tile (TMEM lanes)
constexpr int BN = 256;            // columns of C' per tile = 64 quaternion columns
constexpr int BNQ = BN / 4;
constexpr int BK = 32;             // reals of K per stage (64 bytes: one swizzle row)
constexpr int STAGES = 3;
constexpr int TERMS = 3;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // warp 0 TMA, warp 1 MMA, 2..9 drain/epilogue
constexpr uint32_t kATermBytes = BM * BK * 2;  // 8 KB
constexpr uint32_t kBTermBytes = BN * BK * 2;  // 16 KB
constexpr uint32_t kStageA = TERMS * kATermBytes;
constexpr uint32_t kStageB = TERMS * kBTermBytes;
constexpr uint32_t kStageBytes = kStageA + kStageB;  // 72 KB
constexpr uint32_t kTmemCols = 2 * BN;               // two accumulator buffers
constexpr size_t kSmemBytes = 1024 + STAGES * kStageBytes + 256;
constexpr int kGroupM = 8;                           // row tiles per raster group

// The six kept term products (A term, B term): hh, hm, mh, hl, mm, lh.
__host__ __device__ constexpr int term_a(int tp) { return tp == 2 || tp == 4 ? 1 : (tp == 5 ? 2 : 0); }
__host__ __device__ constexpr int term_b(int tp) { return tp == 1 || tp == 4 ? 1 : (tp == 3 ? 2 : 0); }

// ------------------------------------------------------ tcgen05 helpers ---
// Shared-memory matrix descriptor, K-major, 64-byte swizzle: 8-row groups
// 512 bytes apart (SBO), leading offset unused, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>(1) << 16;                  // LBO (ignored for swizzled K-major)
  d |= static_cast<uint64_t>(512 >> 4) << 32;           // SBO
  d |= static_cast<uint64_t>(1) << 46;                  // version
  d |= static_cast<uint64_t>(4) << 61;                  // SWIZZLE_64B
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                                      // D format F32
         | (1u << 7)                                    // A format BF16
         | (1u << 10)                                   // B format BF16
         | (static_cast<uint32_t>(N >> 3) << 17)        // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);       // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// 32 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "elect.sync _|p, 0xffffffff;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(pred));
  return pred != 0;
}

// --------------------------------------------------------- split helper ---
struct Split3 {
  __nv_bfloat16 t[3];
};
__device__ __forceinline__ Split3 split3(float x) {
  Split3 s;
  s.t[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(s.t[0]);
  s.t[1] = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(s.t[1]);
  s.t[2] = __float2bfloat16_rn(r2);
  return s;
}

// ----------------------------------------------------------- pre-pass ---
// One 32 x 32 tile of the op-matrix X (rows r = i for A or n for B; columns
// kappa), read coalesced from the stored layout through shared memory, split,
// and written K-major with kw components per kappa (4; 2 or 1 when the left
// operand is complex or real, whose missing components are zero):
//   A:  A'_t[r][kw kappa + j]                            j < kw
//   B:  B'_t[4 r + c][kw kappa + j] = sign(j, j^c) * t(b^(j^c))
// (row pitch kp).  Columns kappa >= kq up to kp/kw are zeros (K padding).
// An operand stores `width` components per element (4, 2 or 1); the rest
// read as zero.
struct PrepArgs {
  const float *X;
  int64_t ld, ps;       // stored leading dimension, plane stride
  int64_t rows;         // rows of the op-matrix (m for A, n for B)
  int64_t kq;           // quaternion K
  int64_t kp;           // padded real K (multiple of BK)
  int64_t term_stride;  // elements between terms in the output
  __nv_bfloat16 *out;
  int layout;
  int row_contig;       // stored row index == op row (contiguous along r)
  uint32_t negmask;     // bit j: negate component j of the input (conjugation)
  int width;            // components stored per element
  int kw;               // components per kappa in the output
};

__device__ __forceinline__ float4 load_elem(const PrepArgs &p, int64_t sr, int64_t sc) {
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  if (p.layout == QGEMM_INTERLEAVED) {
    const float *e = p.X + p.width * (sr + sc * p.ld);
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < p.width) v[s] = e[s];
  } else {
    const float *e = p.X + sr + sc * p.ld;
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < p.width) v[s] = e[s * p.ps];
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

template <int KW>
__device__ __forceinline__ void store_terms(__nv_bfloat16 *dst, const __nv_bfloat16 (&w)[4]) {
  if (KW == 4) {
    *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(w);
  } else if (KW == 2) {
    *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(w);
  } else {
    dst[0] = w[0];
  }
}

template <bool IS_B, int KW>
__device__ __forceinline__ void prep_tile_kw(const PrepArgs &p, int64_t rt, int64_t kt,
                                             float4 (*tile)[33]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t r0 = rt * 32, k0 = kt * 32;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int a = tx, b = ty + 8 * s;
    const int rr = p.row_contig ? a : b;
    const int kk = p.row_contig ? b : a;
    const int64_t r = r0 + rr, kq = k0 + kk;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < p.rows && kq < p.kq) {
      v = load_elem(p, p.row_contig ? r : kq, p.row_contig ? kq : r);
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
    if (r >= p.rows || KW * kq >= p.kp) continue;
    const float4 v = tile[kk][rr];
    const float comp[4] = {v.x, v.y, v.z, v.w};
    Split3 sp[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) sp[j] = split3(comp[j]);
    if (!IS_B) {
#pragma unroll
      for (int t = 0; t < TERMS; ++t) {
        __align__(8) __nv_bfloat16 w[4] = {sp[0].t[t], sp[1].t[t], sp[2].t[t], sp[3].t[t]};
        store_terms<KW>(p.out + t * p.term_stride + r * p.kp + KW * kq, w);
      }
    } else {
#pragma unroll
      for (int t = 0; t < TERMS; ++t)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          __align__(8) __nv_bfloat16 w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int q = j ^ c;
            const __nv_bfloat16 x = sp[q].t[t];
            w[j] = basis_sign(j, q) < 0 ? __hneg(x) : x;
          }
          store_terms<KW>(p.out + t * p.term_stride + (4 * r + c) * p.kp + KW * kq, w);
        }
    }
  }
}

template <bool IS_B>
__device__ __forceinline__ void prep_tile(const PrepArgs &p, int64_t rt, int64_t kt,
                                          float4 (*tile)[33]) {
  if (p.kw == 4)
    prep_tile_kw<IS_B, 4>(p, rt, kt, tile);
  else if (p.kw == 2)
    prep_tile_kw<IS_B, 2>(p, rt, kt, tile);
  else
    prep_tile_kw<IS_B, 1>(p, rt, kt, tile);
}

// --------------------------------------------------------- GEMM params ---
// Per-problem parameters of the GEMM kernel.
struct GemmParams {
  int64_t m, n;           // quaternion sizes of C
  int num_kb;             // k-blocks of BK reals (0: C <- beta C)
  int num_mt, num_nt;     // tiles
  int layout;
  int beta_zero;
  int c_vec4;             // interleaved C 16-byte aligned: float4 access
  float *C;
  int64_t ldc, psC;
  float alpha[4], beta[4];
  int tri;                // 0 full; 1 lower (row >= col) only; 2 upper; real diagonal
  int swap;               // 1: the kernel computed D = (op(A) op(B))^H; store C = conj(D)^T
  int krange;             // k-range of a tile when op(A) or op(B) is triangular (GemmDesc)
  // K split (single problems): tile t of the launch is share z = t / (num_mt
  // num_nt) of its tile's k-blocks, whose product P (FP32) goes to part +
  // z m n 4 (dense, interleaved, leading dimension m) for a second kernel.
  int ksplit;             // 0 or 1: no split
  float *part;
};

// k-blocks [lo, hi) of tile (mt, nt), share z: all of K, or the part where a
// triangular operand can be nonzero for the tile's rows or columns; then
// share z of it when the problem splits K.
__host__ __device__ inline void kb_range(const GemmParams &g, int mt, int nt, int z, int &lo,
                                         int &hi) {
  lo = 0;
  hi = g.num_kb;
  const int64_t rq0 = static_cast<int64_t>(mt) * BM, cq0 = static_cast<int64_t>(nt) * BNQ;
  if (g.krange == 1) {
    const int64_t e = (4 * (rq0 + BM) + BK - 1) / BK;
    if (e < hi) hi = static_cast<int>(e);
  }
  if (g.krange == 2) lo = static_cast<int>(4 * rq0 / BK);
  if (g.krange == 3) lo = static_cast<int>(4 * cq0 / BK);
  if (g.krange == 4) {
    const int64_t e = (4 * (cq0 + BNQ) + BK - 1) / BK;
    if (e < hi) hi = static_cast<int>(e);
  }
  if (lo > hi) lo = hi;
  if (g.ksplit > 1) {
    const int64_t span = hi - lo;
    const int l2 = lo + static_cast<int>(span * z / g.ksplit);
    hi = lo + static_cast<int>(span * (z + 1) / g.ksplit);
    lo = l2;
  }
}

// Device descriptor of one problem of a grouped batch.
struct alignas(128) SplitProb {
  CUtensorMap tmA;  // A' : (kp, m, 3) bf16
  CUtensorMap tmB;  // B' : (kp, 4n, 3) bf16
  PrepArgs pa, pb;
  GemmParams g;
};

struct SmemCtl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t accfull[2];
  uint64_t accempty[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

template <class Err>
__device__ __forceinline__ void set_abort(SmemCtl *ctl) {
  atomicCAS(Err::word(), 0, QGEMM_ERR_TIMEOUT);
  *reinterpret_cast<volatile int *>(&ctl->abort) = 1;
}
__device__ __forceinline__ bool aborted(SmemCtl *ctl) {
  return *reinterpret_cast<volatile int *>(&ctl->abort) != 0;
}
// Bounded wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                           SmemCtl *ctl) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (aborted(ctl) || globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// True when tile (mt, nt) has no element in the stored triangle of C.
__device__ __forceinline__ bool tile_skip(const GemmParams &g, int mt, int nt) {
  if (g.tri == 1) return static_cast<int64_t>(mt) * BM + BM - 1 < static_cast<int64_t>(nt) * BNQ;
  if (g.tri == 2) return static_cast<int64_t>(nt) * BNQ + BNQ - 1 < static_cast<int64_t>(mt) * BM;
  return false;
}

// Tile t -> problem parameters, tensor maps and tile coordinates.
template <bool GROUPED>
__device__ __forceinline__ void tile_of(int t, const GemmParams &single, const CUtensorMap *smA,
                                        const CUtensorMap *smB, const SplitProb *probs,
                                        const int4 *tiles, const GemmParams *&g,
                                        const CUtensorMap *&mA, const CUtensorMap *&mB, int &mt,
                                        int &nt, int &z) {
  if (GROUPED) {
    const int4 e = tiles[t];
    const SplitProb *pr = probs + e.x;
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
    z = 0;
    if (single.ksplit > 1) {  // share z of tile t % (tiles of C)
      const int per = single.num_mt * single.num_nt;
      z = t / per;
      t %= per;
    }
    const int per_group = kGroupM * single.num_nt;
    const int first_m = (t / per_group) * kGroupM;
    const int gsize = min(single.num_mt - first_m, kGroupM);
    mt = first_m + (t % per_group) % gsize;
    nt = (t % per_group) / gsize;
    // a triangular operand: the tiles with the longest k-range first, so the
    // CTAs' round-robin shares stay balanced
    if (single.krange == 1) mt = single.num_mt - 1 - mt;
    if (single.krange == 4) nt = single.num_nt - 1 - nt;
  }
}

// Address of element (ci, cj) of C: the first component (interleaved) or the
// component-0 plane entry (planes).
__device__ __forceinline__ float *c_elem(const GemmParams &g, int64_t ci, int64_t cj) {
  return g.layout == QGEMM_INTERLEAVED ? g.C + 4 * (ci + cj * g.ldc) : g.C + ci + cj * g.ldc;
}

// Prefetches into L2 the C elements that epilogue() will read for row i and
// the 32 quaternion columns from nbase (only those inside C).  Issued when a
// tile's first chunk reaches the drain, so the epilogue's reads of C hit L2
// instead of waiting on DRAM one element after another.
__device__ __forceinline__ void prefetch_c(const GemmParams &g, int64_t i, int64_t nbase) {
  if (g.beta_zero || i >= g.m) return;
#pragma unroll 4
  for (int q = 0; q < 32; ++q) {
    const int64_t nn = nbase + q;
    if (nn >= g.n) break;
    const int64_t ci = g.swap ? nn : i, cj = g.swap ? i : nn;
    const float *e = c_elem(g, ci, cj);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(e));
    if (g.layout != QGEMM_INTERLEAVED) {
#pragma unroll
      for (int s = 1; s < 4; ++s) asm volatile("prefetch.global.L2 [%0];" ::"l"(e + s * g.psC));
    }
  }
}

// Epilogue of one tile for one drain thread: row i, 32 quaternion columns
// starting at nbase, accumulated P in acc.  out = alpha P + beta C (left
// products); alpha P and beta C in FP32, their sum in FP64, one rounding.
// C is read in batches of kCBatch elements, all loads of a batch before its
// stores (a larger batch does not fit the drain warps' register budget).
constexpr int kCBatch = 4;
__device__ __forceinline__ void epilogue(const GemmParams &g, int64_t i, int64_t nbase,
                                         const float (&acc)[128]) {
  if (i >= g.m) return;
  if (g.tri == 2 && nbase + 31 < i) return;
  float al[4], be[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    al[s] = g.alpha[s];
    be[s] = g.beta[s];
  }
#pragma unroll
  for (int qb = 0; qb < 32; qb += kCBatch) {
    float cin[kCBatch][4];
#pragma unroll
    for (int u = 0; u < kCBatch; ++u) {
      const int64_t nn = nbase + qb + u;
#pragma unroll
      for (int s = 0; s < 4; ++s) cin[u][s] = 0.f;
      if (g.beta_zero || nn >= g.n) continue;
      // element (ci, cj) of C; a transposed problem holds (AB)^H: take conj(D)^T
      const int64_t ci = g.swap ? nn : i, cj = g.swap ? i : nn;
      const float *src = c_elem(g, ci, cj);
      if (g.layout == QGEMM_INTERLEAVED && g.c_vec4) {
        const float4 c4 = *reinterpret_cast<const float4 *>(src);
        cin[u][0] = c4.x; cin[u][1] = c4.y; cin[u][2] = c4.z; cin[u][3] = c4.w;
      } else {
        const int64_t step = g.layout == QGEMM_INTERLEAVED ? 1 : g.psC;
#pragma unroll
        for (int s = 0; s < 4; ++s) cin[u][s] = src[s * step];
      }
    }
#pragma unroll
    for (int u = 0; u < kCBatch; ++u) {
      const int q = qb + u;
      const int64_t nn = nbase + q;
      if (nn >= g.n) continue;
      if ((g.tri == 1 && i < nn) || (g.tri == 2 && i > nn)) continue;
      float P[4] = {acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]};
      const int64_t ci = g.swap ? nn : i, cj = g.swap ? i : nn;
      if (g.swap) {
        P[1] = -P[1];
        P[2] = -P[2];
        P[3] = -P[3];
      }
      float out[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float ap = 0.f, bc = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int s = c ^ j;  // the sign is a compile-time constant here
          const bool neg = basis_sign(s, j) < 0;
          ap = fmaf(neg ? -al[s] : al[s], P[j], ap);
          bc = fmaf(neg ? -be[s] : be[s], cin[u][j], bc);
        }
        out[c] = g.beta_zero
                     ? ap
                     : static_cast<float>(static_cast<double>(ap) + static_cast<double>(bc));
      }
      if (g.tri && i == nn) out[1] = out[2] = out[3] = 0.f;  // Hermitian diagonal is real
      float *dst0 = c_elem(g, ci, cj);
      if (g.layout == QGEMM_INTERLEAVED) {
        if (g.c_vec4)
          *reinterpret_cast<float4 *>(dst0) = make_float4(out[0], out[1], out[2], out[3]);
        else
#pragma unroll
          for (int s = 0; s < 4; ++s) dst0[s] = out[s];
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) dst0[s * g.psC] = out[s];
      }
    }
  }
}

// K split: the product P of share z for row i and the 32 quaternion columns
// from nbase, stored to the share's slab (dense, interleaved, ld m).
__device__ __forceinline__ void store_partial(const GemmParams &g, int64_t i, int64_t nbase, int z,
                                              const float (&acc)[128]) {
  if (i >= g.m) return;
  float *slab = g.part + static_cast<int64_t>(z) * g.m * g.n * 4;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int64_t nn = nbase + q;
    if (nn >= g.n) break;
    *reinterpret_cast<float4 *>(slab + 4 * (i + nn * g.m)) =
        make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
}

// Persistent split-BF16 GEMM.  Single problem: tensor maps and parameters
// are kernel parameters, tiles rasterised in groups of kGroupM row tiles.
// Grouped: tiles[t] = (problem, row tile, column tile), per-problem maps and
// parameters in probs.  Err::word() is the device status word.
template <class Err, bool GROUPED>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const GemmParams single, const SplitProb *__restrict__ probs,
                const int4 *__restrict__ tiles, int ntiles, int chunk, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *ring = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  SmemCtl *ctl = reinterpret_cast<SmemCtl *>(ring + STAGES * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
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
    // ---------------- TMA producer ----------------
    if (elect_one()) {
      if (!GROUPED) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
      }
      uint32_t s_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const GemmParams *g;
        const CUtensorMap *mA, *mB;
        int mt, nt, z;
        tile_of<GROUPED>(t, single, &tmA, &tmB, probs, tiles, g, mA, mB, mt, nt, z);
        if (tile_skip(*g, mt, nt)) continue;
        int kb_lo, kb_hi;
        kb_range(*g, mt, nt, z, kb_lo, kb_hi);
        for (int kb = kb_lo; kb < kb_hi; ++kb, ++s_run) {
          const int st = s_run % STAGES;
          if (!wait_phase(&ctl->empty[st], ((s_run / STAGES) & 1) ^ 1, limit_ns, ctl)) {
            set_abort<Err>(ctl);
            ok = false;
            break;
          }
          unsigned char *sa = ring + st * kStageBytes;
          mbar_arrive_expect_tx(&ctl->full[st], kStageBytes);
          tma_load_3d(sa, mA, &ctl->full[st], kb * BK, mt * BM, 0);
          tma_load_3d(sa + kStageA, mB, &ctl->full[st], kb * BK, nt * BN, 0);
        }
      }
      if (!ok) {  // let this CTA's copies in flight land before it retires
        for (uint32_t q = s_run > STAGES ? s_run - STAGES : 0; q < s_run; ++q)
          mbar_wait_bounded(&ctl->full[q % STAGES], (q / STAGES) & 1, limit_ns);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (elect_one()) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      const uint32_t ring_addr = smem_u32(ring);
      uint32_t s_run = 0, c_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const GemmParams *g;
        const CUtensorMap *mA, *mB;
        int mt, nt, z;
        tile_of<GROUPED>(t, single, &tmA, &tmB, probs, tiles, g, mA, mB, mt, nt, z);
        if (tile_skip(*g, mt, nt)) continue;
        int kb_lo, nkb;
        kb_range(*g, mt, nt, z, kb_lo, nkb);
        for (int kb = kb_lo; kb < nkb && ok; ++c_run) {
          const int b = c_run & 1;
          if (!wait_phase(&ctl->accempty[b], ((c_run >> 1) & 1) ^ 1, limit_ns, ctl)) {
            set_abort<Err>(ctl);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + b * BN;
          const int kb_end = min(nkb, kb + chunk);
          bool first = true;
          for (; kb < kb_end; ++kb, ++s_run) {
            const int st = s_run % STAGES;
            if (!wait_phase(&ctl->full[st], (s_run / STAGES) & 1, limit_ns, ctl)) {
              set_abort<Err>(ctl);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = ring_addr + st * kStageBytes;
            const uint32_t sb = sa + kStageA;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
              for (int tp = 0; tp < 6; ++tp) {
                const uint64_t ad = smem_desc_sw64(sa + term_a(tp) * kATermBytes + ks * 32);
                const uint64_t bd = smem_desc_sw64(sb + term_b(tp) * kBTermBytes + ks * 32);
                umma_bf16(d, ad, bd, idesc, first ? 0u : 1u);
                first = false;
              }
            }
            umma_commit(&ctl->empty[st]);  // frees the stage when these MMAs finish
          }
          if (!ok) break;
          umma_commit(&ctl->accfull[b]);  // chunk accumulator ready for the drain
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
      umma_commit(&ctl->done);
      mbar_wait_bounded(&ctl->done, 0, limit_ns);
    }
  } else {
    // ---------------- drain + epilogue (8 warps) ----------------
    const int ew = warp - 2;
    const int quad = warp & 3;   // TMEM lanes 32*quad .. +31 (hardware rule: warp % 4)
    const int half = ew >> 2;    // columns [128*half, 128*half + 128)
    const uint32_t lane_base = static_cast<uint32_t>(32 * quad) << 16;
    uint32_t c_run = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const GemmParams *g;
      const CUtensorMap *mA, *mB;
      int mt, nt, z;
      tile_of<GROUPED>(t, single, &tmA, &tmB, probs, tiles, g, mA, mB, mt, nt, z);
      if (tile_skip(*g, mt, nt)) continue;
      int kb_lo, kb_hi;
      kb_range(*g, mt, nt, z, kb_lo, kb_hi);
      const int nch = (kb_hi - kb_lo + chunk - 1) / chunk;
      if (g->ksplit <= 1)
        prefetch_c(*g, static_cast<int64_t>(mt) * BM + 32 * quad + lane,
                   static_cast<int64_t>(nt) * BNQ + 32 * half);
      float acc[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) acc[i] = 0.f;
      for (int ch = 0; ch < nch; ++ch, ++c_run) {
        const int b = c_run & 1;
        if (!wait_phase(&ctl->accfull[b], (c_run >> 1) & 1, limit_ns, ctl)) {
          set_abort<Err>(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + lane_base + b * BN + half * 128;
        // 32 columns per load: the drain warps' register budget is 168 per
        // thread (10 warps per CTA, three on some SM sub-partitions)
#pragma unroll
        for (int piece = 0; piece < 4; ++piece) {
          float v[32];
          tmem_ld32(base + piece * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[piece * 32 + i] += v[i];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->accempty[b]);
      }
      if (!ok) break;
      if (g->ksplit > 1)
        store_partial(*g, static_cast<int64_t>(mt) * BM + 32 * quad + lane,
                      static_cast<int64_t>(nt) * BNQ + 32 * half, z, acc);
      else
        epilogue(*g, static_cast<int64_t>(mt) * BM + 32 * quad + lane,
                 static_cast<int64_t>(nt) * BNQ + 32 * half, acc);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace split
}  // namespace qg

namespace qg {
namespace split {

// --------------------------------------------------------- fused path ---
// The same product without a workspace: FP32 tiles of op(A) and op(B) come in
// by TMA in their stored layout (3-D boxes as in the FP64 path, zero fill past
// the edges), two converter warps split them into the three BF16 terms and
// write A' and the sign-expanded B' directly into the 64-byte-swizzled
// K-major layout of the MMA operands, then hand the stage to the MMA warp
// (generic-proxy writes made visible to the tensor core by
// fence.proxy.async).  Used where the operand pre-pass would cost more HBM
// traffic than it saves (many small problems).
constexpr int FSTAGES = 2;                          // BF16 operand stages
constexpr int FSTAGING = 3;                         // FP32 staging slots
constexpr int kConvWarps = 2;
constexpr int kFusedThreads = kThreads + 32 * kConvWarps;
constexpr int FKQ = BK / 4;                         // quaternion k per stage (8)
constexpr uint32_t kStagingA = BM * FKQ * 16;       // 16 KB FP32 op(A) tile
constexpr uint32_t kStagingB = BNQ * FKQ * 16;      // 8 KB FP32 op(B) tile
constexpr uint32_t kStagingBytes = kStagingA + kStagingB;
constexpr size_t kFusedSmemBytes =
    1024 + FSTAGES * kStageBytes + FSTAGING * kStagingBytes + 256;

// Per-problem parameters of the fused path.
struct FusedOps {
  int layout;
  int ta, tb;          // op(A) / op(B) transposed (T or H)
  uint32_t conj_a;     // component sign masks (bit s: negate component s)
  uint32_t conj_b;
};

struct alignas(128) FusedProb {
  CUtensorMap tmA;     // FP32 stored A, 3-D box
  CUtensorMap tmB;     // FP32 stored B, 3-D box
  FusedOps o;
  GemmParams g;
};

struct FusedCtl {
  uint64_t sfull[FSTAGING];   // FP32 staging landed (TMA)
  uint64_t sempty[FSTAGING];  // FP32 staging consumed (converters)
  uint64_t full[FSTAGES];     // BF16 stage written (converters)
  uint64_t empty[FSTAGES];    // BF16 stage consumed (MMA commit)
  uint64_t accfull[2];
  uint64_t accempty[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

// Byte offset of element (row, k) (k < 32 bf16) in a K-major tile with
// 64-byte rows and the 64-byte swizzle (16-byte chunk index XOR bits 1..2 of
// the row), the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_64B.
__device__ __forceinline__ uint32_t sw64_offset(int row, int k) {
  const int chunk = (k >> 3) ^ ((row >> 1) & 3);
  return static_cast<uint32_t>(row * 64 + chunk * 16 + (k & 7) * 2);
}

// Index (in floats) of component s of op-tile element (r, kk) in the FP32
// staging tile.  The TMA box order is the stored order: for the stored
// element (sr, sc) of a box with R stored rows and CC stored columns,
// interleaved: s + 4 (sr + R sc);  planes: sr + R (sc + CC s).
__device__ __forceinline__ int staging_idx(int layout, bool trans, int R_op, int r, int kk,
                                           int s) {
  // op-tile is R_op rows x FKQ k; stored tile is (R_op x FKQ) or transposed
  const int sr = trans ? kk : r, sc = trans ? r : kk;
  const int R = trans ? FKQ : R_op, CC = trans ? R_op : FKQ;
  if (layout == QGEMM_INTERLEAVED) return s + 4 * (sr + R * sc);
  return sr + R * (sc + CC * s);
}

__device__ __forceinline__ void store_bf16x4(unsigned char *tile, int row, int k0,
                                             __nv_bfloat16 a, __nv_bfloat16 b,
                                             __nv_bfloat16 c, __nv_bfloat16 d) {
  __align__(8) __nv_bfloat16 w[4] = {a, b, c, d};
  *reinterpret_cast<uint2 *>(tile + sw64_offset(row, k0)) = *reinterpret_cast<const uint2 *>(w);
}

// Converter: FP32 staging slot -> BF16 stage (A' rows i, B' rows 4n + c).
__device__ __forceinline__ void convert_stage(const float *stA, const float *stB,
                                              unsigned char *stage, const FusedOps &o,
                                              int ctid) {
  // A': 128 rows x 8 quaternion k; thread handles (row, kk) pairs
  for (int e = ctid; e < BM * FKQ; e += 32 * kConvWarps) {
    const int r = e % BM, kk = e / BM;
    float v[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      v[s] = stA[staging_idx(o.layout, o.ta, BM, r, kk, s)];
      if ((o.conj_a >> s) & 1u) v[s] = -v[s];
    }
    Split3 sp[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) sp[s] = split3(v[s]);
#pragma unroll
    for (int t = 0; t < TERMS; ++t)
      store_bf16x4(stage + t * kATermBytes, r, 4 * kk, sp[0].t[t], sp[1].t[t], sp[2].t[t],
                   sp[3].t[t]);
  }
  // B': 64 quaternion columns x 8 quaternion k -> rows 4n + c
  unsigned char *sb = stage + kStageA;
  for (int e = ctid; e < BNQ * FKQ; e += 32 * kConvWarps) {
    const int n = e % BNQ, kk = e / BNQ;
    float v[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      // op(B) tile element (kk, n): use the op-row = n convention of staging_idx
      v[s] = stB[o.tb ? staging_idx(o.layout, false, BNQ, n, kk, s)
                      : staging_idx(o.layout, true, BNQ, n, kk, s)];
      if ((o.conj_b >> s) & 1u) v[s] = -v[s];
    }
    Split3 sp[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) sp[s] = split3(v[s]);
#pragma unroll
    for (int t = 0; t < TERMS; ++t)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        __nv_bfloat16 w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int q = j ^ c;
          w[j] = basis_sign(j, q) < 0 ? __hneg(sp[q].t[t]) : sp[q].t[t];
        }
        store_bf16x4(sb + t * kBTermBytes, 4 * n + c, 4 * kk, w[0], w[1], w[2], w[3]);
      }
  }
}

__device__ __forceinline__ void tma_stage(float *dst, const CUtensorMap *map, uint64_t *bar,
                                          int layout, int r0, int c0) {
  if (layout == QGEMM_INTERLEAVED)
    tma_load_3d(dst, map, bar, 0, r0, c0);
  else
    tma_load_3d(dst, map, bar, r0, c0, 0);
}

template <bool GROUPED>
__device__ __forceinline__ void fused_tile_of(int t, const GemmParams &single,
                                              const FusedOps &single_o, const CUtensorMap *smA,
                                              const CUtensorMap *smB, const FusedProb *probs,
                                              const int4 *tiles, const GemmParams *&g,
                                              const FusedOps *&o, const CUtensorMap *&mA,
                                              const CUtensorMap *&mB, int &mt, int &nt) {
  if (GROUPED) {
    const int4 e = tiles[t];
    const FusedProb *pr = probs + e.x;
    g = &pr->g;
    o = &pr->o;
    mA = &pr->tmA;
    mB = &pr->tmB;
    mt = e.y;
    nt = e.z;
  } else {
    g = &single;
    o = &single_o;
    mA = smA;
    mB = smB;
    const int per_group = kGroupM * single.num_nt;
    const int first_m = (t / per_group) * kGroupM;
    const int gsize = min(single.num_mt - first_m, kGroupM);
    mt = first_m + (t % per_group) % gsize;
    nt = (t % per_group) / gsize;
    // a triangular operand: the tiles with the longest k-range first, so the
    // CTAs' round-robin shares stay balanced
    if (single.krange == 1) mt = single.num_mt - 1 - mt;
    if (single.krange == 4) nt = single.num_nt - 1 - nt;
  }
}

template <class Err>
__device__ __forceinline__ void fused_abort(FusedCtl *ctl) {
  atomicCAS(Err::word(), 0, QGEMM_ERR_TIMEOUT);
  *reinterpret_cast<volatile int *>(&ctl->abort) = 1;
}
__device__ __forceinline__ bool fused_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                           FusedCtl *ctl) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*reinterpret_cast<volatile int *>(&ctl->abort) != 0 || globaltimer_ns() - t0 > limit_ns)
      return false;
  }
}

// Warps: 0 TMA (FP32 staging), 1 MMA, 2..9 drain + epilogue, 10..11 convert.
template <class Err, bool GROUPED>
__global__ void __launch_bounds__(kFusedThreads, 1)
    fused_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const GemmParams single, const FusedOps single_o,
                 const FusedProb *__restrict__ probs, const int4 *__restrict__ tiles, int ntiles,
                 int chunk, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *ring = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  float *staging = reinterpret_cast<float *>(ring + FSTAGES * kStageBytes);
  FusedCtl *ctl = reinterpret_cast<FusedCtl *>(reinterpret_cast<unsigned char *>(staging) +
                                               FSTAGING * kStagingBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < FSTAGING; ++s) {
      mbar_init(&ctl->sfull[s], 1);
      mbar_init(&ctl->sempty[s], kConvWarps);
    }
    for (int s = 0; s < FSTAGES; ++s) {
      mbar_init(&ctl->full[s], kConvWarps);
      mbar_init(&ctl->empty[s], 1);
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
    // ---------------- TMA producer: FP32 tiles ----------------
    if (elect_one()) {
      uint32_t s_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const GemmParams *g;
        const FusedOps *o;
        const CUtensorMap *mA, *mB;
        int mt, nt;
        fused_tile_of<GROUPED>(t, single, single_o, &tmA, &tmB, probs, tiles, g, o, mA, mB, mt,
                               nt);
        if (tile_skip(*g, mt, nt)) continue;
        const int nkb = g->num_kb;
        const int layout = o->layout, ta = o->ta, tb = o->tb;
        for (int kb = 0; kb < nkb; ++kb, ++s_run) {
          const int st = s_run % FSTAGING;
          if (!fused_wait(&ctl->sempty[st], ((s_run / FSTAGING) & 1) ^ 1, limit_ns, ctl)) {
            fused_abort<Err>(ctl);
            ok = false;
            break;
          }
          float *sa = staging + st * (kStagingBytes / 4);
          float *sb = sa + kStagingA / 4;
          mbar_arrive_expect_tx(&ctl->sfull[st], kStagingBytes);
          const int k0 = kb * FKQ;
          tma_stage(sa, mA, &ctl->sfull[st], layout, ta ? k0 : mt * BM, ta ? mt * BM : k0);
          tma_stage(sb, mB, &ctl->sfull[st], layout, tb ? nt * BNQ : k0, tb ? k0 : nt * BNQ);
        }
      }
      if (!ok) {
        for (uint32_t q = s_run > FSTAGING ? s_run - FSTAGING : 0; q < s_run; ++q)
          mbar_wait_bounded(&ctl->sfull[q % FSTAGING], (q / FSTAGING) & 1, limit_ns);
      }
    }
  } else if (warp >= 2 + kEpiWarps) {
    // ---------------- converters ----------------
    const int ctid = threadIdx.x - 32 * (2 + kEpiWarps);
    uint32_t s_run = 0, b_run = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const GemmParams *g;
      const FusedOps *o;
      const CUtensorMap *mA, *mB;
      int mt, nt;
      fused_tile_of<GROUPED>(t, single, single_o, &tmA, &tmB, probs, tiles, g, o, mA, mB, mt,
                             nt);
      if (tile_skip(*g, mt, nt)) continue;
      const FusedOps ops = *o;
      const int nkb = g->num_kb;
      for (int kb = 0; kb < nkb; ++kb, ++s_run, ++b_run) {
        const int ss = s_run % FSTAGING, bs = b_run % FSTAGES;
        if (!fused_wait(&ctl->sfull[ss], (s_run / FSTAGING) & 1, limit_ns, ctl) ||
            !fused_wait(&ctl->empty[bs], ((b_run / FSTAGES) & 1) ^ 1, limit_ns, ctl)) {
          fused_abort<Err>(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        const float *sa = staging + ss * (kStagingBytes / 4);
        convert_stage(sa, sa + kStagingA / 4, ring + bs * kStageBytes, ops, ctid);
        fence_proxy_async_smem();  // the tensor core reads what the threads wrote
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&ctl->sempty[ss]);
          mbar_arrive(&ctl->full[bs]);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (elect_one()) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      const uint32_t ring_addr = smem_u32(ring);
      uint32_t b_run = 0, c_run = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const GemmParams *g;
        const FusedOps *o;
        const CUtensorMap *mA, *mB;
        int mt, nt;
        fused_tile_of<GROUPED>(t, single, single_o, &tmA, &tmB, probs, tiles, g, o, mA, mB, mt,
                               nt);
        if (tile_skip(*g, mt, nt)) continue;
        const int nkb = g->num_kb;  // the fused path runs all of K
        for (int kb = 0; kb < nkb && ok; ++c_run) {
          const int b = c_run & 1;
          if (!fused_wait(&ctl->accempty[b], ((c_run >> 1) & 1) ^ 1, limit_ns, ctl)) {
            fused_abort<Err>(ctl);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + b * BN;
          const int kb_end = min(nkb, kb + chunk);
          bool first = true;
          for (; kb < kb_end; ++kb, ++b_run) {
            const int st = b_run % FSTAGES;
            if (!fused_wait(&ctl->full[st], (b_run / FSTAGES) & 1, limit_ns, ctl)) {
              fused_abort<Err>(ctl);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = ring_addr + st * kStageBytes;
            const uint32_t sb = sa + kStageA;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
              for (int tp = 0; tp < 6; ++tp) {
                const uint64_t ad = smem_desc_sw64(sa + term_a(tp) * kATermBytes + ks * 32);
                const uint64_t bd = smem_desc_sw64(sb + term_b(tp) * kBTermBytes + ks * 32);
                umma_bf16(d, ad, bd, idesc, first ? 0u : 1u);
                first = false;
              }
            }
            umma_commit(&ctl->empty[st]);
          }
          if (!ok) break;
          umma_commit(&ctl->accfull[b]);
        }
      }
      umma_commit(&ctl->done);
      mbar_wait_bounded(&ctl->done, 0, limit_ns);
    }
  } else {
    // ---------------- drain + epilogue (8 warps) ----------------
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int half = ew >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(32 * quad) << 16;
    uint32_t c_run = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const GemmParams *g;
      const FusedOps *o;
      const CUtensorMap *mA, *mB;
      int mt, nt;
      fused_tile_of<GROUPED>(t, single, single_o, &tmA, &tmB, probs, tiles, g, o, mA, mB, mt,
                             nt);
      if (tile_skip(*g, mt, nt)) continue;
      const int nkb = g->num_kb;
      const int nch = (nkb + chunk - 1) / chunk;
      prefetch_c(*g, static_cast<int64_t>(mt) * BM + 32 * quad + lane,
                 static_cast<int64_t>(nt) * BNQ + 32 * half);
      float acc[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) acc[i] = 0.f;
      for (int ch = 0; ch < nch; ++ch, ++c_run) {
        const int b = c_run & 1;
        if (!fused_wait(&ctl->accfull[b], (c_run >> 1) & 1, limit_ns, ctl)) {
          fused_abort<Err>(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + lane_base + b * BN + half * 128;
#pragma unroll
        for (int piece = 0; piece < 4; ++piece) {
          float v[32];
          tmem_ld32(base + piece * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[piece * 32 + i] += v[i];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->accempty[b]);
      }
      if (!ok) break;
      epilogue(*g, static_cast<int64_t>(mt) * BM + 32 * quad + lane,
               static_cast<int64_t>(nt) * BNQ + 32 * half, acc);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace split
}  // namespace qg
