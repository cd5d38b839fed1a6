// FP64 quaternion GEMM on the FP64 FMA pipe (DFMA): C <- alpha op(A) op(B) +
// beta C (Sec. 3.1, Eq. general_gemm) for full quaternion operands.
//
// Measured on GB300 (qgemm_probe_peak): the FP64 FMA pipe runs 1.26 TFLOP/s,
// the FP64 tensor pipe (DMMA m16n8k4) 1.10, and the two do not add (0.40
// together).  So the plain product takes the FMA pipe; the DMMA kernel
// (fp64_dmma.cu) keeps the cases this kernel leaves out (K split, one
// triangle, k-ranges, mixed types, grids too small to fill the GPU).
//
// Each element product is the Hamilton product (Sec. 2.1, Eq.
// quaternion_prod): component c of a b is the sum over j of sign(c^j, j)
// a^(c^j) b^j, 16 FMAs whose signs are the FMA's operand negation (free).
// A CTA of 256 threads computes a 32 x 32 quaternion tile of C; thread (ty,
// tx) holds the 2 x 2 quaternions at rows 2 ty + {0, 1}, columns 2 tx + {0,
// 1} in 16 FP64 accumulators.  K advances by 16 quaternions: op(A) and op(B)
// tiles are staged in shared memory (conjugated there for op C / H, zeros past
// the edges), and each kappa takes 64 FMAs per thread against 4 shared-memory
// quaternion reads.  The pipe runs about 2 FMAs per cycle per SM, so one
// 16-kappa step of a tile is about 130k cycles of FMAs against a few thousand
// for its loads: two CTAs per SM cover the staging of one with the FMAs of
// the other.
#include <cstring>

#include "common.cuh"

namespace qg {
namespace {

constexpr int kTQ = 32;  // quaternion rows / columns of C per CTA
constexpr int kKQ = 16;  // quaternion kappa per shared-memory step
constexpr int kGroupM = 16;  // row tiles per raster group

// One quaternion in registers or shared memory.
struct alignas(32) Qd {
  double x, y, z, w;
};

struct DfmaArgs {
  const double *A, *B;
  double *C;
  int64_t m, n, k;
  int64_t lda, ldb, ldc;    // leading dimensions (elements)
  int64_t psA, psB, psC;    // plane strides (reals; split-plane layout)
  int planes;               // 1: split-plane layout, 0: interleaved
  int transA, transB, conjA, conjB;
  int beta_zero;
  int64_t tiles_m, tiles_n;  // tile grid
  double alpha[4], beta[4];
};

// Element (r, c) of a STORED operand with four components.
__device__ __forceinline__ Qd load_q(const double *X, int64_t ld, int64_t ps, int planes,
                                          int64_t r, int64_t c) {
  if (!planes) {
    const double *e = X + 4 * (r + c * ld);
    return Qd{e[0], e[1], e[2], e[3]};
  }
  const double *e = X + r + c * ld;
  return Qd{e[0], e[ps], e[2 * ps], e[3 * ps]};
}

// acc += a b (Hamilton product, signs as FMA negations).
__device__ __forceinline__ void qmac(double (&acc)[4], const Qd &a, const Qd &b) {
  const double av[4] = {a.x, a.y, a.z, a.w};
  const double bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = c ^ j;
      acc[c] = basis_sign(p, j) < 0 ? fma(-av[p], bv[j], acc[c]) : fma(av[p], bv[j], acc[c]);
    }
}

// s x (s on the left) added to out.
__device__ __forceinline__ void qmac_left(double (&out)[4], const double (&s)[4],
                                          const double (&x)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = c ^ j;
      out[c] = basis_sign(p, j) < 0 ? fma(-s[p], x[j], out[c]) : fma(s[p], x[j], out[c]);
    }
}

__global__ void __launch_bounds__(256, 2) fp64_dfma_kernel(const DfmaArgs a) {
  __shared__ Qd As[kKQ][kTQ];  // op(A)(i0 + i, k0 + kappa) at As[kappa][i]
  __shared__ Qd Bs[kKQ][kTQ];  // op(B)(k0 + kappa, n0 + n) at Bs[kappa][n]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // raster: groups of kGroupM row tiles walked column by column, so the CTAs
  // running at one time share a few row and column panels (read from L2)
  const int64_t t = blockIdx.x;
  const int64_t grp = t / (kGroupM * a.tiles_n);
  const int64_t r0 = grp * kGroupM;
  const int64_t rows = min(static_cast<int64_t>(kGroupM), a.tiles_m - r0);
  const int64_t local = t - grp * kGroupM * a.tiles_n;
  const int64_t i0 = (r0 + local % rows) * kTQ;
  const int64_t n0 = (local / rows) * kTQ;
  double acc[2][2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[u][v][c] = 0.0;

  for (int64_t k0 = 0; k0 < a.k; k0 += kKQ) {
    // staging: 512 elements of each operand, two per thread, consecutive
    // threads along the stored contiguous index
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;
      {
        // op(A)(i, kappa): stored (i, kappa) for N / C, (kappa, i) for T / H
        const int i = a.transA ? (e >> 4) : (e & 31);
        const int kk = a.transA ? (e & 15) : (e >> 5);
        const int64_t gi = i0 + i, gk = k0 + kk;
        Qd v = Qd{0.0, 0.0, 0.0, 0.0};
        if (gi < a.m && gk < a.k)
          v = a.transA ? load_q(a.A, a.lda, a.psA, a.planes, gk, gi)
                       : load_q(a.A, a.lda, a.psA, a.planes, gi, gk);
        if (a.conjA) {
          v.y = -v.y;
          v.z = -v.z;
          v.w = -v.w;
        }
        As[kk][i] = v;
      }
      {
        // op(B)(kappa, n): stored (kappa, n) for N / C, (n, kappa) for T / H
        const int nn = a.transB ? (e & 31) : (e >> 4);
        const int kk = a.transB ? (e >> 5) : (e & 15);
        const int64_t gn = n0 + nn, gk = k0 + kk;
        Qd v = Qd{0.0, 0.0, 0.0, 0.0};
        if (gn < a.n && gk < a.k)
          v = a.transB ? load_q(a.B, a.ldb, a.psB, a.planes, gn, gk)
                       : load_q(a.B, a.ldb, a.psB, a.planes, gk, gn);
        if (a.conjB) {
          v.y = -v.y;
          v.z = -v.z;
          v.w = -v.w;
        }
        Bs[kk][nn] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKQ; ++kk) {
      const Qd a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const Qd b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      qmac(acc[0][0], a0, b0);
      qmac(acc[0][1], a0, b1);
      qmac(acc[1][0], a1, b0);
      qmac(acc[1][1], a1, b1);
    }
    __syncthreads();
  }

  // epilogue: alpha P + beta C, both scalars on the left, in FP64
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int64_t gi = i0 + 2 * ty + u, gn = n0 + 2 * tx + v;
      if (gi >= a.m || gn >= a.n) continue;
      double out[4] = {0.0, 0.0, 0.0, 0.0};
      qmac_left(out, a.alpha, acc[u][v]);
      double *e = a.planes ? a.C + gi + gn * a.ldc : a.C + 4 * (gi + gn * a.ldc);
      const int64_t cs = a.planes ? a.psC : 1;
      if (!a.beta_zero) {
        const double cv[4] = {e[0], e[cs], e[2 * cs], e[3 * cs]};
        qmac_left(out, a.beta, cv);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) e[s * cs] = out[s];
    }
}

}  // namespace

// The DFMA kernel serves a plain product of quaternion operands whose grid
// of 32 x 32 tiles fills the GPU: at least 8 tiles per SM, and the waves of
// the CTAs that fit at once at least 90 % full (the DMMA kernel's 16 x 16
// tiles fill smaller or ragged grids better).
bool fp64_dfma_eligible(const GemmDesc &d, int sms) {
  if (d.tri || d.krange || d.swap || d.kwidth != 4 || d.A.width != 4 || d.B.width != 4 ||
      d.k <= 0)
    return false;
  const int64_t tiles = ((d.m + kTQ - 1) / kTQ) * ((d.n + kTQ - 1) / kTQ);
  if (tiles < 8LL * sms) return false;
  static int per_sm = 0;  // resident CTAs per SM (fixed by the kernel's resources)
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fp64_dfma_kernel, 256, 0) !=
            cudaSuccess ||
        v <= 0) {
      cudaGetLastError();
      v = 2;
    }
    per_sm = v;
  }
  const int64_t slots = static_cast<int64_t>(per_sm) * sms;
  const int64_t waves = (tiles + slots - 1) / slots;
  return static_cast<double>(tiles) >= 0.9 * static_cast<double>(waves * slots);
}

int launch_fp64_dfma(const GemmDesc &d, cudaStream_t stream) {
  DfmaArgs a{};
  a.A = static_cast<const double *>(d.A.ptr);
  a.B = static_cast<const double *>(d.B.ptr);
  a.C = static_cast<double *>(d.C);
  a.m = d.m;
  a.n = d.n;
  a.k = d.k;
  a.lda = d.A.ld;
  a.ldb = d.B.ld;
  a.ldc = d.ldc;
  a.psA = d.A.ps;
  a.psB = d.B.ps;
  a.psC = d.psc;
  a.planes = d.layout == QGEMM_SPLIT_PLANES ? 1 : 0;
  a.transA = op_trans(d.opA) ? 1 : 0;
  a.transB = op_trans(d.opB) ? 1 : 0;
  a.conjA = op_conj(d.opA) ? 1 : 0;
  a.conjB = op_conj(d.opB) ? 1 : 0;
  a.beta_zero = d.beta_zero ? 1 : 0;
  for (int s = 0; s < 4; ++s) {
    a.alpha[s] = d.alpha[s];
    a.beta[s] = d.beta[s];
  }
  a.tiles_m = (d.m + kTQ - 1) / kTQ;
  a.tiles_n = (d.n + kTQ - 1) / kTQ;
  const int64_t tiles = a.tiles_m * a.tiles_n;
  if (tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  fp64_dfma_kernel<<<static_cast<unsigned>(tiles), 256, 0, stream>>>(a);
  return launch_status();
}

}  // namespace qg
