// Split-BF16 quaternion GEMM on the fifth-generation tensor cores (tcgen05).
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
// chunk is short (2 k-blocks) and the register sum takes the rest.  The epilogue forms alpha P and beta C in
// FP32 and sums them in FP64 before the one rounding to FP32.
//
// Data path.  Pre-pass kernels read op(A), op(B) in any supported layout
// (coalesced through a shared-memory transpose where needed), split them and
// write A' and the expanded B' as BF16, K-major, zero-padded in K, into the
// caller's workspace.  The GEMM kernel is warp-specialised: one warp issues
// TMA loads (3-D boxes: K x rows x term, 64-byte swizzle) into a 3-stage
// shared-memory ring, one warp issues the MMAs (M=128, N=256, K=16) into
// tensor memory and commits them to mbarriers, eight warps drain tensor
// memory and run the epilogue.  Every wait is bounded.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace qg {

__device__ int g_split_error;

namespace {

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

// The six kept term products (A term, B term): hh, hm, mh, hl, mm, lh.
__constant__ int2 kTermPairs[6] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};

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
// and written K-major.  For A:  A'_t[r][4 kappa + j]  (row pitch kp).
// For B:  B'_t[4 r + c][4 kappa + j] = sign(j, j^c) * t(b^(j^c))  (row pitch kp).
struct PrepArgs {
  const float *X;
  int64_t ld, ps;     // stored leading dimension, plane stride
  int64_t rows;       // rows of the op-matrix (m for A, n for B)
  int64_t kq;         // quaternion K
  int64_t kp;         // padded real K (multiple of BK)
  int64_t term_stride;  // elements between terms in the output
  __nv_bfloat16 *out;
  int layout;
  int row_contig;     // stored row index == op row (contiguous along r)
  uint32_t negmask;   // bit j: negate component j of the input (conjugation)
};

template <bool IS_B>
__global__ void __launch_bounds__(256) split_prepass_kernel(const PrepArgs p) {
  __shared__ float4 tile[32][33];  // [kappa][r]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * 32;
  // load: the thread index tx walks the stored-contiguous dimension
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int a = tx, b = ty + 8 * s;
    const int rr = p.row_contig ? a : b;  // op row offset
    const int kk = p.row_contig ? b : a;  // kappa offset
    const int64_t r = r0 + rr, kq = k0 + kk;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < p.rows && kq < p.kq) {
      // stored element: (r, kq) if row_contig else (kq, r)
      const int64_t sr = p.row_contig ? r : kq, sc = p.row_contig ? kq : r;
      if (p.layout == QGEMM_INTERLEAVED) {
        const float *e = p.X + 4 * (sr + sc * p.ld);
        v = make_float4(e[0], e[1], e[2], e[3]);
      } else {
        const float *e = p.X + sr + sc * p.ld;
        v = make_float4(e[0], e[p.ps], e[2 * p.ps], e[3 * p.ps]);
      }
      if (p.negmask & 2u) v.y = -v.y;
      if (p.negmask & 4u) v.z = -v.z;
      if (p.negmask & 8u) v.w = -v.w;
    }
    tile[kk][rr] = v;
  }
  __syncthreads();
  // write: tx walks kappa (K-major output rows), ty + 8s walks op rows
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int kk = tx, rr = ty + 8 * s;
    const int64_t r = r0 + rr, kq = k0 + kk;
    if (r >= p.rows || 4 * kq >= p.kp) continue;
    const float4 v = tile[kk][rr];  // zero beyond kq (padding)
    const float comp[4] = {v.x, v.y, v.z, v.w};
    Split3 sp[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) sp[j] = split3(comp[j]);
    if (!IS_B) {
#pragma unroll
      for (int t = 0; t < TERMS; ++t) {
        __nv_bfloat16 *dst = p.out + t * p.term_stride + r * p.kp + 4 * kq;
        __align__(8) __nv_bfloat16 w[4] = {sp[0].t[t], sp[1].t[t], sp[2].t[t], sp[3].t[t]};
        *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(w);
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
          __nv_bfloat16 *dst = p.out + t * p.term_stride + (4 * r + c) * p.kp + 4 * kq;
          *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(w);
        }
    }
  }
}

// ----------------------------------------------------------- the GEMM ---
struct GemmArgs {
  int64_t m, n;           // quaternion sizes of C
  int num_kb;             // k-blocks of BK reals
  int chunk;              // k-blocks per TMEM drain
  int num_mt, num_nt;     // tiles
  float *C;
  int64_t ldc, psC;
  int layout;
  int beta_zero;
  int c_vec4;             // interleaved C 16-byte aligned: float4 access
  float alpha[4], beta[4];
  uint64_t limit_ns;
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

__device__ __forceinline__ void set_abort(SmemCtl *ctl) {
  atomicCAS(&g_split_error, 0, QGEMM_ERR_TIMEOUT);
  *reinterpret_cast<volatile int *>(&ctl->abort) = 1;
}
__device__ __forceinline__ bool aborted(SmemCtl *ctl) {
  return *reinterpret_cast<volatile int *>(&ctl->abort) != 0;
}

__global__ void __launch_bounds__(kThreads, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const GemmArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned ring (the swizzle pattern repeats every 512 bytes)
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *ring = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  SmemCtl *ctl = reinterpret_cast<SmemCtl *>(ring + STAGES * kStageBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // tile id -> (mt, nt), grouped so concurrently running CTAs share panels
  const int tile = blockIdx.x;
  constexpr int GROUP = 8;
  const int per_group = GROUP * p.num_nt;
  const int gidx = tile / per_group;
  const int first_m = gidx * GROUP;
  const int gsize = min(p.num_mt - first_m, GROUP);
  const int mt = first_m + (tile % per_group) % gsize;
  const int nt = (tile % per_group) / gsize;

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
  const int num_chunks = (p.num_kb + p.chunk - 1) / p.chunk;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (elect_one()) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      for (int kb = 0; kb < p.num_kb; ++kb) {
        const int st = kb % STAGES;
        const uint32_t par = ((kb / STAGES) & 1) ^ 1;
        if (!mbar_wait_bounded(&ctl->empty[st], par, p.limit_ns) || aborted(ctl)) {
          set_abort(ctl);
          break;
        }
        unsigned char *sa = ring + st * kStageBytes;
        mbar_arrive_expect_tx(&ctl->full[st], kStageBytes);
        tma_load_3d(sa, &tmA, &ctl->full[st], kb * BK, mt * BM, 0);
        tma_load_3d(sa + kStageA, &tmB, &ctl->full[st], kb * BK, nt * BN, 0);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (elect_one()) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      const uint32_t ring_addr = smem_u32(ring);
      int kb = 0;
      bool ok = true;
      for (int ch = 0; ch < num_chunks && ok; ++ch) {
        const int b = ch & 1;
        if (!mbar_wait_bounded(&ctl->accempty[b], ((ch >> 1) & 1) ^ 1, p.limit_ns) ||
            aborted(ctl)) {
          set_abort(ctl);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + b * BN;
        const int kb_end = min(p.num_kb, kb + p.chunk);
        bool first = true;
        for (; kb < kb_end; ++kb) {
          const int st = kb % STAGES;
          if (!mbar_wait_bounded(&ctl->full[st], (kb / STAGES) & 1, p.limit_ns) ||
              aborted(ctl)) {
            set_abort(ctl);
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
              const int2 pr = kTermPairs[tp];
              const uint64_t ad = smem_desc_sw64(sa + pr.x * kATermBytes + ks * 32);
              const uint64_t bd = smem_desc_sw64(sb + pr.y * kBTermBytes + ks * 32);
              umma_bf16(d, ad, bd, idesc, first ? 0u : 1u);
              first = false;
            }
          }
          umma_commit(&ctl->empty[st]);  // frees the stage when these MMAs finish
        }
        if (!ok) break;
        umma_commit(&ctl->accfull[b]);  // chunk accumulator ready for the drain
      }
      // all MMAs issued by this thread complete before TMEM is released
      umma_commit(&ctl->done);
      mbar_wait_bounded(&ctl->done, 0, p.limit_ns);
    }
  } else {
    // ---------------- drain + epilogue (8 warps) ----------------
    const int ew = warp - 2;
    const int quad = warp & 3;        // TMEM lanes 32*quad .. +31 (hardware rule: warp % 4)
    const int half = ew >> 2;         // columns [128*half, 128*half + 128)
    const uint32_t lane_base = static_cast<uint32_t>(32 * quad) << 16;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.f;
    bool ok = true;
    for (int ch = 0; ch < num_chunks; ++ch) {
      const int b = ch & 1;
      if (!mbar_wait_bounded(&ctl->accfull[b], (ch >> 1) & 1, p.limit_ns) || aborted(ctl)) {
        set_abort(ctl);
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
    if (ok) {
      // epilogue: out = alpha P + beta C, left products; alpha P and beta C in
      // FP32, their sum in FP64, one rounding to float.
      const int64_t i = static_cast<int64_t>(mt) * BM + 32 * quad + lane;
      const int64_t nbase = static_cast<int64_t>(nt) * BNQ + 32 * half;
      if (i < p.m) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int64_t nn = nbase + q;
          if (nn >= p.n) continue;
          const float P[4] = {acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]};
          float cin[4] = {0.f, 0.f, 0.f, 0.f};
          float *dst0;
          if (p.layout == QGEMM_INTERLEAVED) {
            dst0 = p.C + 4 * (i + nn * p.ldc);
            if (!p.beta_zero) {
              if (p.c_vec4) {
                const float4 c4 = *reinterpret_cast<const float4 *>(dst0);
                cin[0] = c4.x; cin[1] = c4.y; cin[2] = c4.z; cin[3] = c4.w;
              } else {
#pragma unroll
                for (int s = 0; s < 4; ++s) cin[s] = dst0[s];
              }
            }
          } else {
            dst0 = p.C + i + nn * p.ldc;
            if (!p.beta_zero) {
#pragma unroll
              for (int s = 0; s < 4; ++s) cin[s] = dst0[s * p.psC];
            }
          }
          float out[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float ap = 0.f, bc = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int s = c ^ j;
              const float sa = basis_sign(s, j) < 0 ? -p.alpha[s] : p.alpha[s];
              const float sb = basis_sign(s, j) < 0 ? -p.beta[s] : p.beta[s];
              ap = fmaf(sa, P[j], ap);
              bc = fmaf(sb, cin[j], bc);
            }
            out[c] = p.beta_zero ? ap : static_cast<float>(static_cast<double>(ap) +
                                                           static_cast<double>(bc));
          }
          if (p.layout == QGEMM_INTERLEAVED) {
            if (p.c_vec4)
              *reinterpret_cast<float4 *>(dst0) = make_float4(out[0], out[1], out[2], out[3]);
            else
#pragma unroll
              for (int s = 0; s < 4; ++s) dst0[s] = out[s];
          } else {
#pragma unroll
            for (int s = 0; s < 4; ++s) dst0[s * p.psC] = out[s];
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------- tcgen05 probe ---
// Back-to-back M=128, N=256, K=16 BF16 MMAs on a fixed shared-memory tile
// (contents irrelevant), one CTA per SM: the tensor-pipe throughput of the
// instruction shape the GEMM uses.
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(int iters, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  unsigned char *buf = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kATermBytes + kBTermBytes) / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(buf)[i] = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tbase, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0 && elect_one()) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
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
    tmem_dealloc(tbase, BN);
  }
}

// ----------------------------------------------------------- host side ---
struct SplitPlan {
  int64_t kp;           // padded real K
  size_t a_bytes, b_bytes, b_offset, total;
};

SplitPlan plan_for(const GemmDesc &d) {
  SplitPlan s;
  s.kp = ((4 * d.k + BK - 1) / BK) * BK;
  s.a_bytes = static_cast<size_t>(TERMS) * d.m * s.kp * 2;
  s.b_bytes = static_cast<size_t>(TERMS) * 4 * d.n * s.kp * 2;
  s.b_offset = (s.a_bytes + 1023) & ~static_cast<size_t>(1023);
  s.total = s.b_offset + s.b_bytes;
  return s;
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
                   int layout, __nv_bfloat16 *out, int64_t term_stride, cudaStream_t stream) {
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
  const int64_t gx = (rows + 31) / 32, gy = (kp / 4 + 31) / 32;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (is_b)
    split_prepass_kernel<true><<<grid, 256, 0, stream>>>(a);
  else
    split_prepass_kernel<false><<<grid, 256, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? QGEMM_SUCCESS : QGEMM_ERR_CUDA;
}

}  // namespace

int split_workspace_bytes(const GemmDesc &d, size_t *bytes) {
  if (d.k == 0 || d.m == 0 || d.n == 0) {
    *bytes = 0;
    return QGEMM_SUCCESS;
  }
  *bytes = plan_for(d).total;
  return QGEMM_SUCCESS;
}

int launch_split_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream) {
  const SplitPlan pl = plan_for(d);
  if (ws_bytes < pl.total || ws == nullptr) return QGEMM_ERR_WORKSPACE;
  auto *wa = static_cast<__nv_bfloat16 *>(ws);
  auto *wb = reinterpret_cast<__nv_bfloat16 *>(static_cast<unsigned char *>(ws) + pl.b_offset);
  int rc = launch_prepass(false, d.A, d.opA, d.m, d.k, pl.kp, d.layout, wa, d.m * pl.kp, stream);
  if (rc) return rc;
  rc = launch_prepass(true, d.B, d.opB, d.n, d.k, pl.kp, d.layout, wb, 4 * d.n * pl.kp, stream);
  if (rc) return rc;

  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  if (!encode_bf16_3d(&tmA, wa, pl.kp, d.m, BM) || !encode_bf16_3d(&tmB, wb, pl.kp, 4 * d.n, BN))
    return QGEMM_ERR_UNSUPPORTED;
  GemmArgs g;
  g.m = d.m;
  g.n = d.n;
  g.num_kb = static_cast<int>(pl.kp / BK);
  g.chunk = chunk_for(g.num_kb);
  g.num_mt = static_cast<int>((d.m + BM - 1) / BM);
  g.num_nt = static_cast<int>((d.n + BNQ - 1) / BNQ);
  g.C = static_cast<float *>(d.C);
  g.ldc = d.ldc;
  g.psC = d.psc;
  g.layout = d.layout;
  g.beta_zero = d.beta_zero ? 1 : 0;
  g.c_vec4 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
  for (int s = 0; s < 4; ++s) {
    g.alpha[s] = static_cast<float>(d.alpha[s]);
    g.beta[s] = static_cast<float>(d.beta[s]);
  }
  g.limit_ns = wait_limit_ns();
  const int64_t tiles = static_cast<int64_t>(g.num_mt) * g.num_nt;
  if (tiles > 0x7fffffff || pl.kp / BK > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  rc = set_smem(split_gemm_kernel, kSmemBytes);
  if (rc) return rc;
  split_gemm_kernel<<<static_cast<unsigned>(tiles), kThreads, kSmemBytes, stream>>>(tmA, tmB, g);
  return cudaGetLastError() == cudaSuccess ? QGEMM_SUCCESS : QGEMM_ERR_CUDA;
}

int probe_tcgen05_bf16(double seconds, double *tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 1024 + kATermBytes + kBTermBytes;
  int rc = set_smem(tc_probe_kernel, smem);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 1024;
  float ms = 0.f;
  rc = QGEMM_SUCCESS;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    tc_probe_kernel<<<sms, 128, smem, stream>>>(iters, wait_limit_ns());
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
    *tflops = 2.0 * BM * BN * 16 * 2.0 * iters * sms / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
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
