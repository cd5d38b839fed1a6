// Mixed-type products (the quaternion-complex and quaternion-real arithmetic
// of the paper's library, Sec. 5): C <- alpha op(A) op(B) + beta C with C
// quaternion and A, B each quaternion, complex (z^0 e0 + z^1 e1) or real.
//
// Split-BF16 path: the component-plane kernel (split_core.cuh) sums the real
// products A^p (B^j)^T over the planes each factor has, so a complex (real)
// factor on either side has 2 (1) planes: half (a quarter) of the MMAs of the
// quaternion product.  Digit-sliced path: its real form C' = A' B' only needs
// the components the left factor has (A' keeps 2 (1) columns per kappa and
// B' the matching rows of its sign expansion, K' = 2k (k)); a quaternion left
// factor with a narrow right factor is turned around with (AB)^H = B^H A^H
// (Sec. 2.2): the kernel computes D = op(B)^H op(A)^H with the narrow factor
// on the left and stores C = conj(D)^T.  The FP64 DMMA path takes the narrow
// factor on the RIGHT (fp64_mixed.cu: one DMMA spans 4 / width values of
// kappa), turning a narrow left factor around the same way; when both are
// narrow the left one is copied as a quaternion matrix into the workspace.
#include <cstring>

#include "common.cuh"

namespace qg {
namespace {

constexpr int kWidth[3] = {4, 2, 1};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Quaternion copy (rows x cols, ld = rows, planes rows*cols apart) of a
// typed stored matrix with w components per element.
template <int LAYOUT>
__global__ void __launch_bounds__(256)
    embed_kernel(const double *__restrict__ X, int64_t ld, int64_t ps, int w, int64_t rows,
                 int64_t cols, double *__restrict__ Q) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * 32 + (threadIdx.x & 31);
  const int64_t c = static_cast<int64_t>(blockIdx.y) * 8 + (threadIdx.x >> 5);
  if (r >= rows || c >= cols) return;
  double q[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s = 0; s < w; ++s)
    q[s] = LAYOUT == QGEMM_INTERLEAVED ? X[w * (r + c * ld) + s] : X[r + c * ld + s * ps];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (LAYOUT == QGEMM_INTERLEAVED)
      Q[4 * (r + c * rows) + s] = q[s];
    else
      Q[r + c * rows + s * rows * cols] = q[s];
  }
}

int launch_embed(const MatView &v, int layout, double *Q, cudaStream_t s) {
  const int64_t gx = (v.rows + 31) / 32, gy = (v.cols + 7) / 8;
  if (gx == 0 || gy == 0) return QGEMM_SUCCESS;
  if (gx > 0x7fffffff || gy > 65535) return QGEMM_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  const double *X = static_cast<const double *>(v.ptr);
  if (layout == QGEMM_INTERLEAVED)
    embed_kernel<QGEMM_INTERLEAVED><<<grid, 256, 0, s>>>(X, v.ld, v.ps, v.width, v.rows, v.cols, Q);
  else
    embed_kernel<QGEMM_SPLIT_PLANES><<<grid, 256, 0, s>>>(X, v.ld, v.ps, v.width, v.rows, v.cols, Q);
  return launch_status();
}

size_t embed_bytes(const MatView &v) {
  return v.width == 4 ? 0 : align_up(static_cast<size_t>(v.rows) * v.cols * 32, 256);
}

// (op(X))^H = op'(X).
int op_conjtrans(int op) {
  switch (op) {
    case QGEMM_OP_N: return QGEMM_OP_H;
    case QGEMM_OP_H: return QGEMM_OP_N;
    case QGEMM_OP_T: return QGEMM_OP_C;
    default: return QGEMM_OP_T;
  }
}

// Validated descriptor of a mixed product.  FP64: the narrow factor goes to
// the right; digit-sliced: to the left (turned around when needed);
// split-BF16: either side as it is.
int mixed_desc(int typeA, int typeB, int opA, int opB, int64_t m, int64_t n, int64_t k,
               const double *alpha, const void *A, int64_t lda, int64_t psA, const void *B,
               int64_t ldb, int64_t psB, const double *beta, void *C, int64_t ldc, int64_t psC,
               int layout, int precision, GemmDesc *d) {
  if (typeA < 0 || typeA > 2) return -1;
  if (typeB < 0 || typeB > 2) return -2;
  int rc = validate_gemm(opA, opB, m, n, k, alpha, A, lda, psA, B, ldb, psB, beta, C, ldc, psC,
                         layout, precision, d);
  if (rc) return rc - 2;  // qgemm position i is argument i + 2 here
  d->A.width = kWidth[typeA];
  d->B.width = kWidth[typeB];
  if (d->k == 0) return 0;
  auto turn_around = [](GemmDesc *x) {
    GemmDesc t = *x;
    t.m = x->n;
    t.n = x->m;
    t.opA = op_conjtrans(x->opB);
    t.opB = op_conjtrans(x->opA);
    t.A = x->B;
    t.B = x->A;
    t.swap = 1;
    *x = t;
  };
  if (precision == QGEMM_FP64) {
    // the narrow factor on the right (both narrow: the left one is copied)
    if (typeA != 0 && typeB == 0) turn_around(d);
    return 0;
  }
  // split-BF16: the component-plane kernel takes a narrow factor on either
  // side (fewer planes), nothing to rearrange
  if (precision == QGEMM_FP32_SPLIT_BF16) return 0;
  // digit-sliced: the narrow factor on the left
  if (typeA != 0) {
    d->kwidth = kWidth[typeA];
  } else if (typeB != 0) {
    turn_around(d);
    d->kwidth = kWidth[typeB];
  }
  return 0;
}

}  // namespace
}  // namespace qg

using namespace qg;

extern "C" {

size_t qgemm_mixed_workspace_bytes(int typeA, int typeB, int opA, int opB, int64_t m, int64_t n,
                                   int64_t k, int layout, int precision) {
  if (opA < 0 || opA > 3 || opB < 0 || opB > 3 || m <= 0 || n <= 0 || k <= 0) return 0;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return 0;
  const int64_t ra = op_trans(opA) ? k : m, ca = op_trans(opA) ? m : k;
  const int64_t rb = op_trans(opB) ? n : k, cb = op_trans(opB) ? k : n;
  const uintptr_t p = 256;
  const double one[4] = {1.0, 0.0, 0.0, 0.0};
  const bool planes = layout == QGEMM_SPLIT_PLANES;
  GemmDesc d;
  if (mixed_desc(typeA, typeB, opA, opB, m, n, k, one, reinterpret_cast<const void *>(p), ra,
                 planes ? ra * ca : 0, reinterpret_cast<const void *>(p), rb, planes ? rb * cb : 0,
                 one, reinterpret_cast<void *>(p), m, planes ? m * n : 0, layout, precision, &d))
    return 0;
  if (precision == QGEMM_FP64) return embed_bytes(d.A);
  size_t g = 0;
  if (precision == QGEMM_FP32_SPLIT_BF16 && split_workspace_bytes(d, &g)) return 0;
  if (precision == QGEMM_FP64_SLICED_BF16 && sliced_workspace_bytes(d, &g)) return 0;
  return g;
}

int qgemm_mixed(int typeA, int typeB, int opA, int opB, int64_t m, int64_t n, int64_t k,
                const double alpha[4], const void *A, int64_t lda, int64_t psA, const void *B,
                int64_t ldb, int64_t psB, const double beta[4], void *C, int64_t ldc,
                int64_t psC, int layout, int precision, void *workspace, size_t workspace_bytes,
                void *stream) {
  GemmDesc d;
  int rc = mixed_desc(typeA, typeB, opA, opB, m, n, k, alpha, A, lda, psA, B, ldb, psB, beta, C,
                      ldc, psC, layout, precision, &d);
  if (rc) return rc;
  const size_t need =
      d.k > 0 ? qgemm_mixed_workspace_bytes(typeA, typeB, opA, opB, m, n, k, layout, precision)
              : 0;
  if (need > 0) {
    if (workspace == nullptr || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return -21;
    if (workspace_bytes < need) return -22;
  }
  if (m == 0 || n == 0) return QGEMM_SUCCESS;
  rc = device_ready();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d.k == 0) return launch_scale(d, precision_fp64_data(precision), s);
  if (precision == QGEMM_FP64) {
    if (d.A.width != 4) {  // both factors narrow: the left one as a quaternion matrix
      double *Q = static_cast<double *>(workspace);
      rc = launch_embed(d.A, layout, Q, s);
      if (rc) return rc;
      d.A.ptr = Q;
      d.A.ld = d.A.rows > 0 ? d.A.rows : 1;
      d.A.ps = d.A.rows * d.A.cols;
      d.A.width = 4;
    }
    return d.B.width == 4 ? launch_fp64_gemm(d, s) : launch_fp64_mixed(d, s);
  }
  if (precision == QGEMM_FP64_SLICED_BF16)
    return launch_sliced_gemm(d, workspace, workspace_bytes, s);
  return launch_split_gemm(d, workspace, workspace_bytes, s);
}

}  // extern "C"
