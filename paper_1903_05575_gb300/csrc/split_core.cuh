// Split-BF16 quaternion GEMM on the fifth-generation tensor cores (tcgen05):
// device code shared by the single-problem path (split_bf16.cu) and the
// grouped path (grouped.cu).
//
// Component form.  With a = op(A)_{i kappa} and b = op(B)_{kappa n}, the
// Hamilton product (Sec. 2.1, Eq. quaternion_prod) is
//     (a b)^c = sum over p xor j = c of sign(p, j) a^p b^j,
// sign(p, j) the sign of the basis product e_p e_j (Eq. quaternion_alg).  So
// component c of op(A) op(B) is the signed sum of the four real products
// A^p (B^j)^T with p xor j = c, where X^s is the real matrix of component s
// of X (the plane of Eq. quaternion_mat_def): sixteen real products, exactly
// the 16 m n k multiplies of the quaternion product.  The planes are stored
// K-major (BF16 terms, below) and each component c of the result accumulates
// in its own tensor-memory region; the sign is the MMA instruction's negate
// bit, so no operand is ever sign-expanded.  The MMAs that share one A plane
// and one sign take it from the tensor core's operand collector (fill / use
// / lastuse), so shared memory supplies it once per group.  A complex or
// real factor simply has fewer planes.
//
// Scalars.  alpha is applied to op(A) by the pre-pass, in double-float
// arithmetic (pairs of FP32 with error-free products and sums), before the
// split: (alpha op(A)) op(B) = alpha (op(A) op(B)) (associativity; the
// scalar acts from the left, Sec. 2.2).  beta C (FP32 products) is where a
// tile's accumulation starts: C is read at the start of the tile, while its
// first MMAs run, and enters the compensated sum below like one more chunk,
// so the end of a tile only stores.
//
// Precision.  Each value x (an FP32 input, or alpha x in double-float) is
// split by round-to-nearest into three BF16 terms hi + mid + lo, with a
// residual below 2^-27 |x|.  The six leading term products hh, hm, mh, hl, mm,
// lh run on tcgen05.mma kind::f16 (BF16 in, FP32 accumulate in tensor memory);
// mid lo, lo mid and lo lo (below 2^-27 of a product) are dropped.  The
// accumulator is drained every chunk of K into a register sum by a
// compensated addition (TwoSum) whose rounding error is written back into the
// tensor-memory accumulator, where the next chunk of the same buffer adds
// onto it.  So the running sum keeps the accuracy of the chunk sums instead
// of losing one FP32 rounding of the whole sum per chunk; GB300's FP64 pipe is
// 64 times narrower than its FP32 pipe, so the FP64-class steps run as
// error-free FP32 transformations.
//
// Kernel.  Persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ...; one
// warp issues TMA loads (4-D boxes: kappa x rows x planes x terms, 32-byte
// swizzle) into a 3-stage ring, one warp issues the MMAs (M = 128, N <= 64,
// K = 16) into one of two TMEM accumulator sets and commits them to
// mbarriers, eight warps drain TMEM and store a tile while the MMAs of the
// next one proceed.  Ring slots, barrier phases and TMEM buffers
// are indexed by running counters that continue across tiles.  Every wait is
// bounded.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace qg {
namespace split {

// ---------------------------------------------------------------- sizes ---
constexpr int BM = 128;            // rows of C per tile (TMEM lanes)
constexpr int BNQ = 64;            // quaternion columns of C per tile (largest MMA N)
constexpr int KQ = 16;             // kappa per stage: one MMA K step (32-byte rows)
constexpr int STAGES = 3;
constexpr int TERMS = 3;
constexpr int PLANES = 4;
constexpr int kChunk = 1;          // stages per TMEM drain
constexpr int kEpiWarps = 8;
// warp 0 TMA, warp 1 MMA, warps 2-3 idle (warpgroup 0), warps 4..11 drain /
// epilogue (warpgroups 1 and 2)
constexpr int kThreads = 128 + 32 * kEpiWarps;
// Registers per thread after the split of the launch's 384 x 168: warpgroup
// 0 gives up to kRegsCtl, the drain warpgroups take kRegsDrain (128 x 56 +
// 256 x 224 = 64512 <= 64512; per SM sub-partition 56 + 2 x 224 = 504 <= 512).
constexpr int kRegsCtl = 56;
constexpr int kRegsDrain = 224;
static_assert(128 * kRegsCtl + 32 * kEpiWarps * kRegsDrain <= kThreads * 168, "register split");
constexpr uint32_t kAPlaneBytes = BM * KQ * 2;   // 4 KB
constexpr uint32_t kBPlaneBytes = BNQ * KQ * 2;  // 2 KB
constexpr uint32_t kStageA = TERMS * PLANES * kAPlaneBytes;  // 48 KB
constexpr uint32_t kStageB = TERMS * PLANES * kBPlaneBytes;  // 24 KB
constexpr uint32_t kStageBytes = kStageA + kStageB;           // 72 KB
constexpr uint32_t kBufCols = PLANES * BNQ;                   // one accumulator set
constexpr uint32_t kTmemCols = 2 * kBufCols;                  // two sets
constexpr size_t kSmemBytes = 1024 + STAGES * kStageBytes + 256;
constexpr int kGroupM = 8;                                    // row tiles per raster group
// The largest quaternion k: a share's 32-bit stage counters and the TMA
// coordinates stay in range.
constexpr int64_t kMaxK = int64_t(1) << 30;

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
// The same MMA with the A operand taken into (fill), reused from (use) or
// released from (lastuse) the tensor core's operand collector: consecutive
// MMAs that share A then read it from shared memory once.
#define QG_UMMA_COLLECTOR(NAME, QUAL)                                                       \
  __device__ __forceinline__ void NAME(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,     \
                                       uint32_t idesc, uint32_t accumulate) {               \
    asm volatile(                                                                           \
        "{\n\t.reg .pred p;\n\t"                                                        \
        "setp.ne.b32 p, %4, 0;\n\t"                                                       \
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::" QUAL " [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem), \
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)                                 \
        : "memory");                                                                        \
  }
QG_UMMA_COLLECTOR(umma_bf16_fill, "fill")
QG_UMMA_COLLECTOR(umma_bf16_use, "use")
QG_UMMA_COLLECTOR(umma_bf16_lastuse, "lastuse")
#undef QG_UMMA_COLLECTOR
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

// K-major, 32-byte swizzle (one 16-element BF16 row per 32 bytes): 8-row
// groups 256 bytes apart (SBO), leading offset unused, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>(1) << 16;                  // LBO (ignored for swizzled K-major)
  d |= static_cast<uint64_t>(256 >> 4) << 32;           // SBO
  d |= static_cast<uint64_t>(1) << 46;                  // version
  d |= static_cast<uint64_t>(6) << 61;                  // SWIZZLE_32B
  return d;
}
// Instruction-descriptor bit that negates the B operand of one MMA.
constexpr uint32_t kNegB = 1u << 14;

// Two 32-bit words as one 64-bit register (low word first).
__device__ __forceinline__ uint64_t pack2(uint32_t lo, uint32_t hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}

__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr, uint64_t (&v)[8]) {
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
  for (int i = 0; i < 8; ++i) v[i] = pack2(r[2 * i], r[2 * i + 1]);
}
// 16 columns as 8 packed pairs, without the wait (the caller waits once for
// a batch of loads with tmem_ld_wait).
__device__ __forceinline__ void tmem_ld16x2_nowait(uint32_t taddr, uint64_t (&v)[8]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = pack2(r[2 * i], r[2 * i + 1]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_st16x2(uint32_t taddr, const uint64_t (&v)[8]) {
  uint32_t r[16];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    r[2 * i] = static_cast<uint32_t>(v[i]);
    r[2 * i + 1] = static_cast<uint32_t>(v[i] >> 32);
  }
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}
// 32 consecutive 32-bit columns of this thread's TMEM lane as 16 packed
// pairs (columns 2i, 2i + 1 in pair i), with the wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr, uint64_t (&v)[16]) {
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
  for (int i = 0; i < 16; ++i) v[i] = pack2(r[2 * i], r[2 * i + 1]);
}
__device__ __forceinline__ void tmem_st32x2(uint32_t taddr, const uint64_t (&v)[16]) {
  uint32_t r[32];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    r[2 * i] = static_cast<uint32_t>(v[i]);
    r[2 * i + 1] = static_cast<uint32_t>(v[i] >> 32);
  }
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// 32 consecutive 32-bit columns of this thread's TMEM lane <- v.  The caller
// waits (tmem_st_wait) before it hands the columns to the MMAs.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane (load with its
// wait; store without).
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
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ------------------------------------------------ double-float helpers ---
// Error-free transformations on FP32 (Knuth's TwoSum; the product error by
// one FMA), on two values at once: packed .f32x2 arithmetic, whose
// instructions round to nearest and are never contracted or reassociated.  A
// pair is a 64-bit register: low word first.
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ uint64_t f2_neg(uint64_t a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ void two_sum2(uint64_t a, uint64_t b, uint64_t &s, uint64_t &e) {
  s = f2_add(a, b);
  const uint64_t bp = f2_sub(s, a);
  const uint64_t ap = f2_sub(s, bp);
  e = f2_add(f2_sub(a, ap), f2_sub(b, bp));
}
__device__ __forceinline__ float lo_of(uint64_t x) {
  return __uint_as_float(static_cast<uint32_t>(x));
}
__device__ __forceinline__ float hi_of(uint64_t x) {
  return __uint_as_float(static_cast<uint32_t>(x >> 32));
}

// Two FP32 values as BF16 (round to nearest even) in one 32-bit word: the
// low word's value in the low half (the lower address once stored).
__device__ __forceinline__ uint32_t bf16x2_rn(uint64_t x) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_of(x)), "f"(lo_of(x)));
  return r;
}
// The two BF16 values of a word back as an FP32 pair (exact).
__device__ __forceinline__ uint64_t bf16x2_to_f2(uint32_t t) {
  return pack2(t << 16, t & 0xffff0000u);
}
// Three BF16 terms of each of two double-float values hi + lo (round to
// nearest), as three words of two BF16 each: hi - t0 is exact in FP32, so
// the residual after three terms is below 2^-27 |hi|.
__device__ __forceinline__ void split3_df2(uint64_t hi, uint64_t lo, uint32_t (&t)[3]) {
  t[0] = bf16x2_rn(hi);
  const uint64_t r1 = f2_add(f2_sub(hi, bf16x2_to_f2(t[0])), lo);
  t[1] = bf16x2_rn(r1);
  t[2] = bf16x2_rn(f2_sub(r1, bf16x2_to_f2(t[1])));
}

// ----------------------------------------------------------- pre-pass ---
// One 32 x 32 tile of the op-matrix X (rows r = i for A or n for B; columns
// kappa), read coalesced from the stored layout through shared memory,
// conjugated when the op says so, multiplied by the pre-pass scalar s (alpha
// on the left for A; conj(alpha) on the right for the B side of a problem the
// grouped path turned around), split into three BF16 terms and written as
// K-major planes:
//   out[((t * planes + c) * rows + r) * kp + kappa] = term t of (s x)^c.
// The GEMM never reads columns kappa >= kq (its tensor maps end at kq and
// read zeros beyond); a thread writes two consecutive columns, so an odd kq
// gets a zero written at kq, inside the pitch kp.  An operand stores `width`
// components per element; the others read as zero.
enum { kScaleNone = 0, kScaleReal = 1, kScaleLeft = 2, kScaleRight = 3 };
struct PrepArgs {
  const float *X;
  int64_t ld, ps;       // stored leading dimension, plane stride
  int64_t rows;         // rows of the op-matrix (m for A, n for B)
  int64_t kq;           // quaternion K
  int64_t kp;           // kappa pitch of the output (multiple of 8)
  __nv_bfloat16 *out;
  int layout;
  int row_contig;       // stored row index == op row (contiguous along r)
  int conj;             // op C or H: negate components 1..3
  int width;            // components stored per element
  int planes;           // planes written (1, 2 or 4)
  int smode;            // kScale*
  float s_hi[4], s_lo[4];
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

// Component c of s x (A side: s on the left) or x s (B side: on the right)
// in double-float, for two elements at once: x[j] holds component j of both
// (packed .f32x2 pairs).  Every product of an s word and x is formed without
// error by FMA and the four products are summed by TwoSum.
template <bool RIGHT>
__device__ __forceinline__ void scale_df2(const PrepArgs &p, int c, const uint64_t (&x)[4],
                                          uint64_t &hi, uint64_t &lo) {
  if (p.smode == kScaleNone) {
    hi = x[c];
    lo = 0ull;
    return;
  }
  const bool real = p.smode == kScaleReal;
  hi = lo = 0ull;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = c ^ j;  // scalar component q meets x^j
    if (real && q != 0) continue;
    const bool neg = RIGHT ? basis_sign(j, q) < 0 : basis_sign(q, j) < 0;
    const uint32_t sh = __float_as_uint(neg ? -p.s_hi[q] : p.s_hi[q]);
    const uint32_t sl = __float_as_uint(neg ? -p.s_lo[q] : p.s_lo[q]);
    const uint64_t kh = pack2(sh, sh), kl = pack2(sl, sl);
    const uint64_t pr = f2_mul(kh, x[j]);
    uint64_t e = f2_fma(kh, x[j], f2_neg(pr));
    e = f2_fma(kl, x[j], e);
    if (real || j == 0) {  // the first (a real s: the only) product
      hi = pr;
      lo = e;
    } else {
      uint64_t sum, e2;
      two_sum2(hi, pr, sum, e2);
      hi = sum;
      lo = f2_add(lo, f2_add(e, e2));
    }
  }
}

// Phase 1 of a tile: element (r, kappa) of the tile into tile[kappa][r]
// (zeros outside the matrix), read along the stored contiguous index.
__device__ __forceinline__ void prep_tile_load(const PrepArgs &p, int64_t rt, int64_t kt,
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
    if (r < p.rows && kq < p.kq) v = load_elem(p, p.row_contig ? r : kq, p.row_contig ? kq : r);
    tile[kk][rr] = v;
  }
}

// Phase 2 of a tile (after phase 1 and a barrier): conjugation, scaling,
// split and the K-major stores.
template <bool IS_B>
__device__ __forceinline__ void prep_tile_split(const PrepArgs &p, int64_t rt, int64_t kt,
                                                float4 (*tile)[33]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = rt * 32, k0 = kt * 32;
  // each thread: columns kappa, kappa + 1 of two rows, every step on the pair
  // (one packed instruction, one 4-byte store of two BF16 per term and plane)
  const int64_t plane_stride = p.rows * p.kp;
  const int kk = 2 * (tx & 15);
  const int64_t kq = k0 + kk;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int rr = (tx >> 4) + 2 * ty + 16 * s;
    const int64_t r = r0 + rr;
    if (r >= p.rows || kq >= p.kq) continue;
    const float4 v0 = tile[kk][rr], v1 = tile[kk + 1][rr];
    uint64_t x[4] = {pack2(__float_as_uint(v0.x), __float_as_uint(v1.x)),
                     pack2(__float_as_uint(v0.y), __float_as_uint(v1.y)),
                     pack2(__float_as_uint(v0.z), __float_as_uint(v1.z)),
                     pack2(__float_as_uint(v0.w), __float_as_uint(v1.w))};
    if (p.conj) {
      x[1] = f2_neg(x[1]);
      x[2] = f2_neg(x[2]);
      x[3] = f2_neg(x[3]);
    }
    // kp is even and kq even: 4-byte aligned
    uint32_t *dst = reinterpret_cast<uint32_t *>(p.out + r * p.kp + kq);
    const int64_t wstride = plane_stride / 2;  // in words of two BF16
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c >= p.planes) break;
      uint64_t hi, lo;
      scale_df2<IS_B>(p, c, x, hi, lo);
      uint32_t t[3];
      split3_df2(hi, lo, t);
#pragma unroll
      for (int tt = 0; tt < TERMS; ++tt) dst[(tt * p.planes + c) * wstride] = t[tt];
    }
  }
}

// One tile, both phases (a CTA per tile).
template <bool IS_B>
__device__ __forceinline__ void prep_tile(const PrepArgs &p, int64_t rt, int64_t kt,
                                          float4 (*tile)[33]) {
  prep_tile_load(p, rt, kt, tile);
  __syncthreads();
  prep_tile_split<IS_B>(p, rt, kt, tile);
}

// --------------------------------------------------------- GEMM params ---
// Per-problem parameters of the GEMM kernel.
struct GemmParams {
  int64_t m, n;           // quaternion sizes of C
  int num_kb;             // stages of KQ kappa (0: C <- beta C)
  int num_mt, num_nt;     // tiles
  int pa, pb;             // planes of the A and B operands (1, 2 or 4)
  int layout;
  int beta_zero, beta_real;
  int c_vec4;             // interleaved C 16-byte aligned: float4 access
  float *C;
  int64_t ldc, psC;
  float beta_f[4];         // beta rounded to FP32 (beta C is formed in FP32)
  int tri;                // 0 full; 1 lower (row >= col) only; 2 upper; real diagonal
  int swap;               // 1: the kernel computed D = (op(A) op(B))^H; store C = conj(D)^T
  int krange;             // k-range of a tile when op(A) or op(B) is triangular (GemmDesc)
  // K split (single problems): tile t of the launch is share z = t / (num_mt
  // num_nt) of its tile's stages, whose product P (FP32) goes to part + z m n
  // 4 (dense, interleaved, leading dimension m) for a second kernel.
  int ksplit;             // 0 or 1: no split
  float *part;
};

// Sets beta_f from beta.
inline void set_beta(GemmParams &g, const double *beta) {
  for (int s = 0; s < 4; ++s) g.beta_f[s] = static_cast<float>(beta[s]);
}

// Stages [lo, hi) of tile (mt, nt), share z: all of K, or the part where a
// triangular operand can be nonzero for the tile's rows or columns; then
// share z of it when the problem splits K.
__host__ __device__ inline void kb_range(const GemmParams &g, int mt, int nt, int z, int &lo,
                                         int &hi) {
  lo = 0;
  hi = g.num_kb;
  const int64_t rq0 = static_cast<int64_t>(mt) * BM, cq0 = static_cast<int64_t>(nt) * BNQ;
  if (g.krange == 1) {
    const int64_t e = (rq0 + BM + KQ - 1) / KQ;
    if (e < hi) hi = static_cast<int>(e);
  }
  if (g.krange == 2) lo = static_cast<int>(rq0 / KQ);
  if (g.krange == 3) lo = static_cast<int>(cq0 / KQ);
  if (g.krange == 4) {
    const int64_t e = (cq0 + BNQ + KQ - 1) / KQ;
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

// MMA width of tile column nt: the valid quaternion columns rounded up to
// 16 (the M = 128 granule), at most BNQ.
__host__ __device__ inline int tile_ncols(const GemmParams &g, int nt) {
  const int64_t rem = g.n - static_cast<int64_t>(nt) * BNQ;
  const int64_t w = rem >= BNQ ? BNQ : ((rem + 15) / 16) * 16;
  return static_cast<int>(w);
}

// Device descriptor of one problem of a grouped batch.
struct alignas(128) SplitProb {
  CUtensorMap tmA;  // A planes: (kq, m, pa, 3) bf16
  CUtensorMap tmB;  // B planes: (kq, n, pb, 3) bf16
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

// Everything a role needs to know about tile t.  Grouped tiles are entries
// (problem, row tile, first column, stages | MMA width << 24): a problem's
// column tiles are 64, 32 or 16 columns wide (per size bucket), and no role
// waits on the problem's parameters in global memory before it can start
// the tile; they are plain quaternion products.
struct TileInfo {
  const GemmParams *g;
  const CUtensorMap *mA, *mB;
  int mt, nt, z;
  int n0;            // first quaternion column of the tile
  int kb_lo, kb_hi;  // stages of the tile (its share when K is split)
  int ncols;         // MMA width: valid quaternion columns rounded up to 16
  int pa, pb;        // planes of the A and B operands
  bool skip;         // no element of the tile in the stored triangle of C
};

template <bool GROUPED>
__device__ __forceinline__ TileInfo tile_info(int t, int4 e, const GemmParams &single,
                                              const CUtensorMap *smA, const CUtensorMap *smB,
                                              const SplitProb *probs) {
  TileInfo ti;
  if (GROUPED) {
    const SplitProb *pr = probs + e.x;
    ti.g = &pr->g;
    ti.mA = &pr->tmA;
    ti.mB = &pr->tmB;
    ti.mt = e.y;
    ti.nt = 0;
    ti.n0 = e.z;
    ti.z = 0;
    ti.kb_lo = 0;
    ti.kb_hi = e.w & 0xFFFFFF;
    ti.ncols = (e.w >> 24) & 0xFF;
    ti.pa = ti.pb = PLANES;
    ti.skip = false;
  } else {
    tile_of<false>(t, single, smA, smB, probs, nullptr, ti.g, ti.mA, ti.mB, ti.mt, ti.nt, ti.z);
    ti.skip = tile_skip(single, ti.mt, ti.nt);
    kb_range(single, ti.mt, ti.nt, ti.z, ti.kb_lo, ti.kb_hi);
    ti.ncols = tile_ncols(single, ti.nt);
    ti.n0 = ti.nt * BNQ;
    ti.pa = single.pa;
    ti.pb = single.pb;
  }
  return ti;
}

// One drain thread's share of a tile's C: row i of the tile's orientation and
// the nq quaternion columns from nbase.  Element (i, nbase + q) of the tile
// sits at base + q step with its components cs apart (a transposed problem
// walks a row of C instead of a column).  Read from the problem's parameters
// once per tile and kept in registers: the stores to C then never make the
// compiler re-read the parameters (it cannot prove that they differ).
struct CRow {
  float *base;
  int64_t i, nbase, step, cs;
  int nq;         // 0: no element of this thread inside C
  int vec4;       // interleaved, 16-byte aligned: one float4 per element
  int swap, tri;
  int beta_mode;  // 0: beta C not added here (beta = 0, or K split); 1 real beta; 2 general
  float beta[4];
};

__device__ __forceinline__ CRow c_row(const GemmParams &g, int64_t i, int64_t nbase, int64_t nlim,
                                      bool with_beta) {
  CRow r;
  const bool il = g.layout == QGEMM_INTERLEAVED;
  const int64_t w = il ? 4 : 1;
  r.i = i;
  r.nbase = nbase;
  r.nq = (i < g.m && nbase < nlim) ? static_cast<int>(min(static_cast<int64_t>(32), nlim - nbase))
                                   : 0;
  r.swap = g.swap;
  r.tri = g.tri;
  // element (ci, cj) of C is at C + w (ci + cj ldc); transposed: (ci, cj) = (nn, i)
  r.base = r.nq == 0 ? g.C : g.C + (g.swap ? w * (nbase + i * g.ldc) : w * (i + nbase * g.ldc));
  r.step = g.swap ? w : w * g.ldc;
  r.cs = il ? 1 : g.psC;
  r.vec4 = il && g.c_vec4;
  r.beta_mode = (!with_beta || g.beta_zero) ? 0 : g.beta_real ? 1 : 2;
#pragma unroll
  for (int s = 0; s < 4; ++s) r.beta[s] = g.beta_f[s];
  return r;
}

// C of columns [q0, q0 + NQ) of r (zeros outside C, and when beta C is not
// added here).  The loads bypass L1: its few KB beside the operand ring would
// hold only a handful of them in flight.
template <int NQ>
__device__ __forceinline__ void load_c(const CRow &r, int q0, float4 (&cv)[NQ]) {
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    cv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r.beta_mode == 0 || q0 + u >= r.nq) continue;
    const float *e = r.base + (q0 + u) * r.step;
    if (r.vec4)
      cv[u] = __ldcg(reinterpret_cast<const float4 *>(e));
    else
      cv[u] = make_float4(__ldcg(e), __ldcg(e + r.cs), __ldcg(e + 2 * r.cs), __ldcg(e + 3 * r.cs));
  }
}

// acc <- beta C for columns [q0, q0 + NQ) (q0, NQ even) from their C values:
// beta on the left, FP32 products, two columns per packed (.f32x2) FMA.  A
// transposed problem accumulates D = (op(A) op(B))^H and stores conj(D), so
// it starts from conj(beta C).
template <int NQ>
__device__ __forceinline__ void beta_c_into(const CRow &r, int q0, const float4 (&cv)[NQ],
                                            uint64_t (&acc)[64]) {
  // coefficient of C^j in component c: sign(e_{c^j} e_j) beta^{c^j} (a real
  // beta: beta^0 on the diagonal only), times -1 for c > 0 when conjugated
  float k[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float b = r.beta_mode == 1 ? (c == j ? r.beta[0] : 0.f)
                                       : (basis_sign(c ^ j, j) < 0 ? -r.beta[c ^ j] : r.beta[c ^ j]);
      k[c][j] = (c > 0 && r.swap) ? -b : b;
    }
#pragma unroll
  for (int u = 0; u < NQ; u += 2) {
    const uint64_t x[4] = {pack2(__float_as_uint(cv[u].x), __float_as_uint(cv[u + 1].x)),
                           pack2(__float_as_uint(cv[u].y), __float_as_uint(cv[u + 1].y)),
                           pack2(__float_as_uint(cv[u].z), __float_as_uint(cv[u + 1].z)),
                           pack2(__float_as_uint(cv[u].w), __float_as_uint(cv[u + 1].w))};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint64_t v = 0ull;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t kj = __float_as_uint(k[c][j]);
        v = f2_fma(pack2(kj, kj), x[j], v);
      }
      acc[16 * c + ((q0 + u) >> 1)] = v;
    }
  }
}

// Starts the accumulation of a tile at beta C (zero where C is not read), so
// that C enters the compensated sum like one more chunk and the tile's end
// only stores.  The loads go out in batches of 8, 12 and 12 columns and wait
// on memory while the tile's first chunk runs on the tensor cores.
__device__ __forceinline__ void acc_init_beta_c(const CRow &r, uint64_t (&acc)[64]) {
  if (r.beta_mode == 0) {
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0ull;
    return;
  }
  {
    float4 first[8];
    load_c<8>(r, 0, first);
    beta_c_into<8>(r, 0, first, acc);
  }
  float4 rest[12];
  load_c<12>(r, 8, rest);
  beta_c_into<12>(r, 8, rest, acc);
  load_c<12>(r, 20, rest);
  beta_c_into<12>(r, 20, rest, acc);
}

__device__ __forceinline__ float acc_at(const uint64_t (&acc)[64], int c, int q) {
  return (q & 1) ? hi_of(acc[16 * c + (q >> 1)]) : lo_of(acc[16 * c + (q >> 1)]);
}

// Stores the accumulated tile (alpha op(A) op(B) + beta C, or its conjugate
// for a transposed problem) for this thread's row and columns [Q0, Q1): only
// the stored triangle when the problem is a Hermitian update, whose diagonal
// is real.
template <int Q0, int Q1>
__device__ __forceinline__ void store_acc(const CRow &r, const uint64_t (&acc)[64]) {
#pragma unroll
  for (int q = Q0; q < Q1; ++q) {
    if (q >= r.nq) break;
    const int64_t nn = r.nbase + q;
    if ((r.tri == 1 && r.i < nn) || (r.tri == 2 && r.i > nn)) continue;
    float o[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = acc_at(acc, c, q);
    if (r.swap) {
      o[1] = -o[1];
      o[2] = -o[2];
      o[3] = -o[3];
    }
    if (r.tri && r.i == nn) o[1] = o[2] = o[3] = 0.f;
    float *e = r.base + q * r.step;
    // C is not read again by this kernel: the stores bypass L1
    if (r.vec4) {
      __stcg(reinterpret_cast<float4 *>(e), make_float4(o[0], o[1], o[2], o[3]));
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) __stcg(e + s * r.cs, o[s]);
    }
  }
}

// Moves into L2 the C elements that acc_init_beta_c will read (issued for the
// next tile while this one still runs, so those loads hit L2).
__device__ __forceinline__ void prefetch_c(const CRow &r) {
  if (r.beta_mode == 0) return;
#pragma unroll 4
  for (int q = 0; q < 32; ++q) {
    if (q >= r.nq) break;
    const float *e = r.base + q * r.step;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(e));
    if (!r.vec4) {
#pragma unroll
      for (int s = 1; s < 4; ++s) asm volatile("prefetch.global.L2 [%0];" ::"l"(e + s * r.cs));
    }
  }
}

// K split: the product P of share z for row i and the 32 quaternion columns
// from nbase, stored to the share's slab (dense, interleaved, ld m).
__device__ __forceinline__ void store_partial(const GemmParams &g, int64_t i, int64_t nbase, int z,
                                              const uint64_t (&acc)[64]) {
  if (i >= g.m) return;
  float *slab = g.part + static_cast<int64_t>(z) * g.m * g.n * 4;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int64_t nn = nbase + q;
    if (nn >= g.n) break;
    *reinterpret_cast<float4 *>(slab + 4 * (i + nn * g.m)) =
        make_float4(acc_at(acc, 0, q), acc_at(acc, 1, q), acc_at(acc, 2, q), acc_at(acc, 3, q));
  }
}

// Planes j of B whose product with A plane p has the sign of group sg (0:
// positive, 1: negative): bit j of the mask.
__host__ __device__ constexpr uint32_t sign_group(int p, int sg) {
  uint32_t m = 0;
  for (int j = 0; j < PLANES; ++j)
    if ((basis_sign(p, j) < 0) == (sg == 1)) m |= 1u << j;
  return m;
}

__host__ __device__ constexpr int low_bit(uint32_t m) {
  return (m & 1u) ? 0 : (m & 2u) ? 1 : (m & 4u) ? 2 : 3;
}
__host__ __device__ constexpr int high_bit(uint32_t m) {
  return (m & 8u) ? 3 : (m & 4u) ? 2 : (m & 2u) ? 1 : 0;
}

// True when the MMA of pass 0 for planes (p, j) is the first of its stage to
// write component p xor j (pass 0 visits p ascending, then the sign groups,
// then j ascending; every component is written in pass 0).
__host__ __device__ constexpr bool first_touch(int PA, int PB, int p, int j) {
  for (int p2 = 0; p2 < PA; ++p2)
    for (int sg = 0; sg < 2; ++sg)
      for (int j2 = 0; j2 < PB; ++j2) {
        if (!((sign_group(p2, sg) >> j2) & 1u)) continue;
        if (p2 == p && j2 == j) return true;
        if ((p2 ^ j2) == (p ^ j)) return false;
      }
  return false;
}

// The MMAs of one stage into accumulator set d0 (component c at d0 + c BNQ),
// for PA planes of A and PB of B: every A term ta and plane p times B terms
// tb (ta + tb <= 2: hh, hm, hl, mh, mm, lh) and planes j go to component
// p xor j with the sign of e_p e_j.
//  - Order: the small term products (lh; mh, mm; hl, hm) before hh, so most
//    of the tensor core's accumulator additions happen while the sum is
//    about 2^-8 of its final size (its additions round at that scale).
//  - Collector: the MMAs of one pass that share A(ta, p) and a sign form a
//    group that reads A from shared memory once; the negation is taken when
//    A enters the collector (measured: a negate bit on a collector `use` has
//    no effect), so positive and negative products are separate groups.
//    Within a group the B terms of one plane j are consecutive: measured on
//    GB300, this stream issues at 2180 TFLOP/s of BF16 MMAs, against 1420
//    with the B terms outer and the planes inner.
//  - The first MMA into a component overwrites it unless `carry` (the
//    component holds the error written back by the drain).
// Everything but the stage's base descriptors and `carry` is a compile-time
// constant, so the stream unrolls into plain MMA issues.
template <int PA, int PB>
__device__ __forceinline__ void issue_stage(uint32_t d0, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc_n, bool carry) {
  // passes: (A term, first B term, last B term): lh; mh, mm; hl, hm; hh
  constexpr int kPassTa[4] = {2, 1, 0, 0};
  constexpr int kPassTb0[4] = {0, 0, 1, 0};
  constexpr int kPassTb1[4] = {0, 1, 2, 0};
  const uint32_t acc_first = carry ? 1u : 0u;
#pragma unroll
  for (int pass = 0; pass < 4; ++pass) {
    const int ta = kPassTa[pass], tb0 = kPassTb0[pass], tb1 = kPassTb1[pass];
#pragma unroll
    for (int p = 0; p < PA; ++p) {
      const uint64_t ad = adesc + (((ta * PA + p) * kAPlaneBytes) >> 4);
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const uint32_t grp = sign_group(p, sg) & ((1u << PB) - 1u);
        if (grp == 0) continue;
        const int jf = low_bit(grp), jl = high_bit(grp);
        const uint32_t id = idesc_n | (sg ? kNegB : 0u);
#pragma unroll
        for (int o = 0; o < 3 * PLANES; ++o) {
          const int j = o / 3, tb = tb0 + o % 3;
          if (tb > tb1 || j >= PB || !((grp >> j) & 1u)) continue;
          const uint64_t bd = bdesc + (((tb * PB + j) * kBPlaneBytes) >> 4);
          const uint32_t d = d0 + (p ^ j) * BNQ;
          const uint32_t acc = (pass == 0 && first_touch(PA, PB, p, j)) ? acc_first : 1u;
          const bool first = j == jf && tb == tb0;
          const bool last = j == jl && tb == tb1;
          if (first && last)
            umma_bf16(d, ad, bd, id, acc);
          else if (first)
            umma_bf16_fill(d, ad, bd, id, acc);
          else if (last)
            umma_bf16_lastuse(d, ad, bd, id, acc);
          else
            umma_bf16_use(d, ad, bd, id, acc);
        }
      }
    }
  }
}

// issue_stage for the plane counts of a problem (1, 2 or 4 each).
__device__ __forceinline__ void issue_stage_planes(int pa, int pb, uint32_t d0, uint64_t adesc,
                                                   uint64_t bdesc, uint32_t idesc_n, bool carry) {
#define QG_ISSUE(A_, B_) \
  case A_ * 8 + B_: issue_stage<A_, B_>(d0, adesc, bdesc, idesc_n, carry); break;
  switch (pa * 8 + pb) {
    QG_ISSUE(4, 4) QG_ISSUE(4, 2) QG_ISSUE(4, 1) QG_ISSUE(2, 4) QG_ISSUE(1, 4)
    QG_ISSUE(2, 2) QG_ISSUE(2, 1) QG_ISSUE(1, 2)
    default: issue_stage<1, 1>(d0, adesc, bdesc, idesc_n, carry); break;
  }
#undef QG_ISSUE
}

// Persistent split-BF16 GEMM.  Single problem: tensor maps and parameters
// are kernel parameters, tiles rasterised in groups of kGroupM row tiles.
// Grouped: tiles[t] = (problem, row tile, column tile), per-problem maps and
// parameters in probs.  Err::word() is the device status word.
// debug_skip > 0 makes the TMA warp leave out the copies of its running stage
// debug_skip - 1 (fault injection for the bounded waits; 0 in normal use).
template <class Err, bool GROUPED>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const GemmParams single, const SplitProb *__restrict__ probs,
                const int4 *__restrict__ tiles, int ntiles, uint64_t limit_ns, int debug_skip) {
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
  bool producer = false;  // the TMA thread, and the stages it issued
  uint32_t issued = 0;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (elect_one()) {
      if (!GROUPED) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
      }
      uint32_t s_run = 0;
      bool ok = true;
      int4 e_next = make_int4(0, 0, 0, 0);
      if (GROUPED && static_cast<int>(blockIdx.x) < ntiles) e_next = tiles[blockIdx.x];
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int4 e = e_next;  // the next entry loads while this tile runs
        if (GROUPED && t + static_cast<int>(gridDim.x) < ntiles) e_next = tiles[t + gridDim.x];
        const TileInfo ti = tile_info<GROUPED>(t, e, single, &tmA, &tmB, probs);
        if (ti.skip) continue;
        const CUtensorMap *mA = ti.mA, *mB = ti.mB;
        if (GROUPED) {
          tma_prefetch_desc(mA);
          tma_prefetch_desc(mB);
        }
        const int mt = ti.mt, n0 = ti.n0;
        const uint32_t bytes = static_cast<uint32_t>(ti.pa) * TERMS * kAPlaneBytes +
                               static_cast<uint32_t>(ti.pb) * TERMS * kBPlaneBytes;
        for (int kb = ti.kb_lo; kb < ti.kb_hi; ++kb, ++s_run) {
          const int st = s_run % STAGES;
          if (!wait_phase(&ctl->empty[st], ((s_run / STAGES) & 1) ^ 1, limit_ns, ctl)) {
            set_abort<Err>(ctl);
            ok = false;
            break;
          }
          if (debug_skip > 0 && s_run == static_cast<uint32_t>(debug_skip - 1)) continue;
          unsigned char *sa = ring + st * kStageBytes;
          mbar_arrive_expect_tx(&ctl->full[st], bytes);
          tma_load_4d(sa, mA, &ctl->full[st], kb * KQ, mt * BM, 0, 0);
          tma_load_4d(sa + kStageA, mB, &ctl->full[st], kb * KQ, n0, 0, 0);
        }
      }
      producer = true;
      issued = s_run;
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (elect_one()) {
      const uint32_t ring_addr = smem_u32(ring);
      uint32_t s_run = 0, c_run = 0;
      bool ok = true;
      int4 e_next = make_int4(0, 0, 0, 0);
      if (GROUPED && static_cast<int>(blockIdx.x) < ntiles) e_next = tiles[blockIdx.x];
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int4 e = e_next;  // the next entry loads while this tile runs
        if (GROUPED && t + static_cast<int>(gridDim.x) < ntiles) e_next = tiles[t + gridDim.x];
        const TileInfo ti = tile_info<GROUPED>(t, e, single, &tmA, &tmB, probs);
        if (ti.skip) continue;
        const int nkb = ti.kb_hi;
        const uint32_t idesc = idesc_bf16(BM, ti.ncols);
        const int pa = ti.pa, pb = ti.pb;
        int ch = 0;
        for (int kb = ti.kb_lo; kb < nkb && ok; ++c_run, ++ch) {
          const int b = c_run & 1;
          if (!wait_phase(&ctl->accempty[b], ((c_run >> 1) & 1) ^ 1, limit_ns, ctl)) {
            set_abort<Err>(ctl);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + b * kBufCols;
          const int kb_end = min(nkb, kb + kChunk);
          bool carry = ch >= 2;
          for (; kb < kb_end; ++kb, ++s_run) {
            const int st = s_run % STAGES;
            if (!wait_phase(&ctl->full[st], (s_run / STAGES) & 1, limit_ns, ctl)) {
              set_abort<Err>(ctl);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = ring_addr + st * kStageBytes;
            issue_stage_planes(pa, pb, d, smem_desc_sw32(sa), smem_desc_sw32(sa + kStageA),
                               idesc, carry);
            carry = true;  // later stages of the chunk add onto it
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
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsDrain));
    // ---------------- drain + epilogue (8 warps) ----------------
    const int ew = warp - 4;
    const int quad = warp & 3;   // TMEM lanes 32*quad .. +31 (hardware rule: warp % 4)
    const int half = ew >> 2;    // quaternion columns [32*half, 32*half + 32) of the tile
    const uint32_t lane_base = static_cast<uint32_t>(32 * quad) << 16;
    uint32_t c_run = 0;
    bool ok = true;
    int4 e_next = make_int4(0, 0, 0, 0);
    if (GROUPED && static_cast<int>(blockIdx.x) < ntiles) e_next = tiles[blockIdx.x];
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int4 e = e_next;  // the next entry loads while this tile runs
      if (GROUPED && t + static_cast<int>(gridDim.x) < ntiles) e_next = tiles[t + gridDim.x];
      const TileInfo ti = tile_info<GROUPED>(t, e, single, &tmA, &tmB, probs);
      if (ti.skip) continue;
      const GemmParams *g = ti.g;
      const int mt = ti.mt, z = ti.z;
      // this thread's columns: from nbase to the tile's end nlim
      const int64_t nbase = static_cast<int64_t>(ti.n0) + 32 * half;
      const int64_t nlim = min(g->n, static_cast<int64_t>(ti.n0) + ti.ncols);
      const int nch = (ti.kb_hi - ti.kb_lo + kChunk - 1) / kChunk;
      const bool mine = 32 * half < ti.ncols;          // this warp's columns hold data
      const int nacc = ti.pa > ti.pb ? ti.pa : ti.pb;  // components the MMAs write
      const bool split_k = !GROUPED && single.ksplit > 1;  // grouped problems never split K
      const int64_t row = static_cast<int64_t>(mt) * BM + 32 * quad + lane;
      // beta C is added here unless K is split (the reduction kernel adds it)
      const CRow cr = c_row(*g, row, nbase, mine ? nlim : nbase, !split_k);
      // the next tile's C moves into L2 four chunks before this tile ends
      // (much earlier, the streaming operands of the other tiles evict it)
      const int pf_chunk = nch > 4 ? nch - 4 : 0;
      const int t_next = t + static_cast<int>(gridDim.x);
      uint64_t acc[64];  // packed pairs: component c, columns 2i, 2i + 1 in acc[16 c + i]
      acc_init_beta_c(cr, acc);
      for (int ch = 0; ch < nch; ++ch, ++c_run) {
        const int b = c_run & 1;
        if (ch == pf_chunk && t_next < ntiles) {
          const TileInfo tn = tile_info<GROUPED>(t_next, e_next, single, &tmA, &tmB, probs);
          const int64_t nb2 = static_cast<int64_t>(tn.n0) + 32 * half;
          if (!tn.skip && 32 * half < tn.ncols)
            prefetch_c(c_row(*tn.g, static_cast<int64_t>(tn.mt) * BM + 32 * quad + lane, nb2,
                             min(tn.g->n, static_cast<int64_t>(tn.n0) + tn.ncols),
                             !split_k));
        }
        if (!wait_phase(&ctl->accfull[b], (c_run >> 1) & 1, limit_ns, ctl)) {
          set_abort<Err>(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        // the rounding errors go back to TMEM when chunk ch + 2 of this tile
        // accumulates onto them (same buffer)
        const bool carry = ch + 2 < nch;
        if (mine) {
          const uint32_t base = tmem + lane_base + b * kBufCols + 32 * half;
          // two batches of four 16-column loads, one wait each (fewer load
          // round trips); TwoSum on packed pairs (.f32x2 arithmetic: half
          // the instructions)
#pragma unroll
          for (int bt = 0; bt < 2; ++bt) {  // components 2 bt, 2 bt + 1: one load wait
            uint64_t v[4][8];
#pragma unroll
            for (int pc = 0; pc < 4; ++pc)
              tmem_ld16x2_nowait(base + (2 * bt + (pc >> 1)) * BNQ + 16 * (pc & 1), v[pc]);
            tmem_ld_wait();
#pragma unroll
            for (int pc = 0; pc < 4; ++pc) {
              const int c = 2 * bt + (pc >> 1), h = 8 * (pc & 1);
              // a component the MMAs do not write (narrow factors) adds zero
              const bool live = c < nacc;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                uint64_t sum, err;
                two_sum2(acc[16 * c + h + q], live ? v[pc][q] : 0ull, sum, err);
                acc[16 * c + h + q] = sum;
                v[pc][q] = err;
              }
              if (carry) tmem_st16x2(base + c * BNQ + 2 * h, v[pc]);
            }
          }
          if (carry) tmem_st_wait();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->accempty[b]);
      }
      if (!ok) break;
      // stored in two parts, the first before the test of `mine`: with one
      // store loop after it, the compiler kept more of the accumulator live
      // and spilled (ptxas -v)
      if (mine && !split_k) store_acc<0, 8>(cr, acc);
      if (!mine) continue;
      if (split_k)
        store_partial(*g, row, nbase, z, acc);
      else
        store_acc<8, 32>(cr, acc);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (producer && aborted(ctl)) {
    // copies the MMA warp never waited for land before the CTA retires
    for (uint32_t q = issued > STAGES ? issued - STAGES : 0; q < issued; ++q) {
      if (debug_skip > 0 && q == static_cast<uint32_t>(debug_skip - 1)) continue;
      mbar_wait_bounded(&ctl->full[q % STAGES], (q / STAGES) & 1, limit_ns);
    }
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace split
}  // namespace qg
