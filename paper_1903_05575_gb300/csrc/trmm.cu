// Triangular matrix product (the XTRMM of the BLAS-3 set the paper builds on
// its GEMM kernels, Sec. 3), out of place, on the GEMM paths of every
// precision:
//     side left:  C <- alpha op(T) B,   T = tri(A) m x m
//     side right: C <- alpha B op(T),   T = tri(A) n x n
// tri(A) is the stored triangle `uplo` of A, zeros elsewhere, the quaternion 1
// on the diagonal for a unit triangle.  One kernel writes T densely into the
// caller's workspace; the product then runs on the GEMM kernels with the
// k-range of every output tile limited to where op(T) can be nonzero (row
// tile [r0, r1) of a lower op(T) needs kappa < r1, of an upper one
// kappa >= r0; on the right side the column tile bounds kappa instead).
#include <cstring>

#include "common.cuh"

namespace qg {
namespace {

// T(r, c) for r, c < K in A's layout with leading dimension K (planes K^2
// apart), 4 components per thread group.
template <typename F, int LAYOUT>
__global__ void __launch_bounds__(256)
    tri_extract_kernel(const F *__restrict__ A, int64_t lda, int64_t psA, F *__restrict__ T,
                       int64_t K, int lower, int unit) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * 32 + (threadIdx.x & 31);
  const int64_t c = static_cast<int64_t>(blockIdx.y) * 8 + (threadIdx.x >> 5);
  if (r >= K || c >= K) return;
  F q[4] = {F(0), F(0), F(0), F(0)};
  if (unit && r == c) {
    q[0] = F(1);
  } else if (lower ? r >= c : r <= c) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
      q[s] = LAYOUT == QGEMM_INTERLEAVED ? A[4 * (r + c * lda) + s] : A[r + c * lda + s * psA];
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (LAYOUT == QGEMM_INTERLEAVED)
      T[4 * (r + c * K) + s] = q[s];
    else
      T[r + c * K + s * K * K] = q[s];
  }
}

template <typename F>
int launch_extract(const void *A, int64_t lda, int64_t psA, void *T, int64_t K, bool lower,
                   bool unit, int layout, cudaStream_t s) {
  const int64_t gx = (K + 31) / 32, gy = (K + 7) / 8;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (layout == QGEMM_INTERLEAVED)
    tri_extract_kernel<F, QGEMM_INTERLEAVED><<<grid, 256, 0, s>>>(
        static_cast<const F *>(A), lda, psA, static_cast<F *>(T), K, lower, unit);
  else
    tri_extract_kernel<F, QGEMM_SPLIT_PLANES><<<grid, 256, 0, s>>>(
        static_cast<const F *>(A), lda, psA, static_cast<F *>(T), K, lower, unit);
  return launch_status();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct TrmmArgs {
  int side, uplo, trans, diag;
  int64_t m, n;
};

// The GEMM that computes the product once T is in the workspace (A and B of
// the GEMM; pointers filled in by the caller), and its triangle k-range.
int trmm_desc(const TrmmArgs &t, const double *alpha, const void *T, const void *B,
              int64_t ldb, int64_t psB, void *C, int64_t ldc, int64_t psC, int layout,
              int precision, GemmDesc *d) {
  const int64_t K = t.side == QGEMM_LEFT ? t.m : t.n;
  const int64_t psT = layout == QGEMM_SPLIT_PLANES ? K * K : 0;
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  int rc;
  if (t.side == QGEMM_LEFT)
    rc = validate_gemm(t.trans, QGEMM_OP_N, t.m, t.n, K, alpha, T, K, psT, B, ldb, psB, zero, C,
                       ldc, psC, layout, precision, d);
  else
    rc = validate_gemm(QGEMM_OP_N, t.trans, t.m, t.n, K, alpha, B, ldb, psB, T, K, psT, zero, C,
                       ldc, psC, layout, precision, d);
  if (rc) return rc;
  // op(T) is lower when (uplo lower) xor (op transposes)
  const bool op_lower = (t.uplo == QGEMM_LOWER) != op_trans(t.trans);
  if (t.side == QGEMM_LEFT)
    d->krange = op_lower ? 1 : 2;   // rows bound kappa: < row end / >= row start
  else
    d->krange = op_lower ? 3 : 4;   // columns bound kappa: >= col start / < col end
  return 0;
}

}  // namespace
}  // namespace qg

using namespace qg;

extern "C" {

size_t qtrmm_workspace_bytes(int side, int uplo, int transA, int diag, int64_t m, int64_t n,
                             int layout, int precision) {
  if ((side != QGEMM_LEFT && side != QGEMM_RIGHT) || (uplo != QGEMM_LOWER && uplo != QGEMM_UPPER))
    return 0;
  if (transA < 0 || transA > 3 || (diag != QGEMM_NON_UNIT && diag != QGEMM_UNIT)) return 0;
  if (m <= 0 || n <= 0 || !precision_ok(precision)) return 0;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return 0;
  const int64_t K = side == QGEMM_LEFT ? m : n;
  const size_t elem = precision_fp64_data(precision) ? 8 : 4;
  const size_t tb = align_up(static_cast<size_t>(K) * K * 4 * elem, 256);
  const TrmmArgs t{side, uplo, transA, diag, m, n};
  const double one[4] = {1.0, 0.0, 0.0, 0.0};
  GemmDesc d;
  // placeholder pointers and strides: only sizes matter for the workspace
  const uintptr_t p = 256;
  const int64_t ps = layout == QGEMM_SPLIT_PLANES ? m * n : 0;
  if (trmm_desc(t, one, reinterpret_cast<const void *>(p), reinterpret_cast<const void *>(p), m,
                ps, reinterpret_cast<void *>(p), m, ps, layout, precision, &d))
    return 0;
  size_t g = 0;
  if (precision == QGEMM_FP32_SPLIT_BF16 && split_workspace_bytes(d, &g)) return 0;
  if (precision == QGEMM_FP64_SLICED_BF16 && sliced_workspace_bytes(d, &g)) return 0;
  return tb + g;
}

int qtrmm(int side, int uplo, int transA, int diag, int64_t m, int64_t n, const double alpha[4],
          const void *A, int64_t lda, int64_t psA, const void *B, int64_t ldb, int64_t psB,
          void *C, int64_t ldc, int64_t psC, int layout, int precision, void *workspace,
          size_t workspace_bytes, void *stream) {
  if (side != QGEMM_LEFT && side != QGEMM_RIGHT) return -1;
  if (uplo != QGEMM_LOWER && uplo != QGEMM_UPPER) return -2;
  if (transA < 0 || transA > 3) return -3;
  if (diag != QGEMM_NON_UNIT && diag != QGEMM_UNIT) return -4;
  if (m < 0) return -5;
  if (n < 0) return -6;
  if (alpha == nullptr) return -7;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return -17;
  if (!precision_ok(precision)) return -18;
  const int64_t K = side == QGEMM_LEFT ? m : n;
  const size_t elem = precision_fp64_data(precision) ? 8 : 4;
  const bool work = m > 0 && n > 0 &&
                    !(alpha[0] == 0.0 && alpha[1] == 0.0 && alpha[2] == 0.0 && alpha[3] == 0.0);
  if (lda < (K > 1 ? K : 1)) return -9;
  if (work) {
    if (A == nullptr || reinterpret_cast<uintptr_t>(A) % elem) return -8;
    if (layout == QGEMM_SPLIT_PLANES && (psA < 0 || psA < lda * K)) return -10;
  }
  if (ldb < (m > 1 ? m : 1)) return -12;
  if (work && (B == nullptr || reinterpret_cast<uintptr_t>(B) % elem)) return -11;
  if (work && layout == QGEMM_SPLIT_PLANES && (psB < 0 || psB < ldb * n)) return -13;
  if (ldc < (m > 1 ? m : 1)) return -15;
  if (m > 0 && n > 0 && (C == nullptr || reinterpret_cast<uintptr_t>(C) % elem)) return -14;
  if (m > 0 && n > 0 && layout == QGEMM_SPLIT_PLANES && (psC < 0 || psC < ldc * n)) return -16;
  if (work && C == B) return -14;  // out of place only
  const size_t tb = align_up(static_cast<size_t>(K) * K * 4 * elem, 256);
  const size_t need = qtrmm_workspace_bytes(side, uplo, transA, diag, m, n, layout, precision);
  if (work) {
    if (workspace == nullptr || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return -19;
    if (workspace_bytes < need) return -20;
  }
  if (m == 0 || n == 0) return QGEMM_SUCCESS;
  int rc = device_ready();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const TrmmArgs t{side, uplo, transA, diag, m, n};
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  GemmDesc d;
  if (!work) {
    // alpha == 0: C <- 0 (C is not read)
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    rc = validate_gemm(QGEMM_OP_N, QGEMM_OP_N, m, n, 0, zero, nullptr, m, 0, nullptr, 1, 0, zero,
                       C, ldc, psC, layout, precision, &d);
    if (rc) return rc;
    return launch_scale(d, precision_fp64_data(precision), s);
  }
  rc = precision_fp64_data(precision)
           ? launch_extract<double>(A, lda, psA, ws, K, uplo == QGEMM_LOWER, diag == QGEMM_UNIT,
                                    layout, s)
           : launch_extract<float>(A, lda, psA, ws, K, uplo == QGEMM_LOWER, diag == QGEMM_UNIT,
                                   layout, s);
  if (rc) return rc;
  rc = trmm_desc(t, alpha, ws, B, ldb, psB, C, ldc, psC, layout, precision, &d);
  if (rc) return QGEMM_ERR_UNSUPPORTED;  // arguments were checked above
  if (precision == QGEMM_FP64) return launch_fp64_gemm(d, s);
  if (precision == QGEMM_FP64_SLICED_BF16)
    return launch_sliced_gemm(d, ws + tb, workspace_bytes - tb, s);
  return launch_split_gemm(d, ws + tb, workspace_bytes - tb, s);
}

}  // extern "C"
