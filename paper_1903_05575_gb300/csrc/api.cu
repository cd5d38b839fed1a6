// C ABI entry points: argument validation (BLAS rules), quick returns and
// dispatch to the kernels.  Nothing here computes on the host.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace qg {

namespace {

bool is_zero4(const double q[4]) {
  return q[0] == 0.0 && q[1] == 0.0 && q[2] == 0.0 && q[3] == 0.0;
}

// Checks one operand.  pos is the 1-based position of its pointer argument;
// ld and plane stride follow it.  rows/cols are the stored extent.
int check_operand(int pos, const void *p, int64_t ld, int64_t ps, int64_t rows, int64_t cols,
                  bool referenced, int layout, size_t elem) {
  if (ld < (rows > 1 ? rows : 1)) return -(pos + 1);
  if (!referenced) return 0;
  if (p == nullptr) return -pos;
  if (reinterpret_cast<uintptr_t>(p) % elem != 0) return -pos;
  if (layout == QGEMM_SPLIT_PLANES && cols > 0) {
    // planes must not overlap: plane s spans [s*ps, s*ps + ld*cols)
    if (ps < 0 || ps < ld * cols) return -(pos + 2);
  }
  return 0;
}

}  // namespace

// Validates qgemm() arguments into a GemmDesc.  Positions as in qgemm.h.
int validate_gemm(int opA, int opB, int64_t m, int64_t n, int64_t k, const double *alpha,
                  const void *A, int64_t lda, int64_t psA, const void *B, int64_t ldb,
                  int64_t psB, const double *beta, void *C, int64_t ldc, int64_t psC,
                  int layout, int precision, GemmDesc *d) {
  if (opA < 0 || opA > 3) return -1;
  if (opB < 0 || opB > 3) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  if (alpha == nullptr) return -6;
  if (beta == nullptr) return -13;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return -17;
  if (!precision_ok(precision)) return -18;
  const size_t elem = precision_fp64_data(precision) ? sizeof(double) : sizeof(float);
  const bool alpha_zero = is_zero4(alpha);
  const bool product = m > 0 && n > 0 && k > 0 && !alpha_zero;
  const int64_t ra = op_trans(opA) ? k : m, ca = op_trans(opA) ? m : k;
  const int64_t rb = op_trans(opB) ? n : k, cb = op_trans(opB) ? k : n;
  int rc = check_operand(7, A, lda, psA, ra, ca, product, layout, elem);
  if (rc) return rc;
  rc = check_operand(10, B, ldb, psB, rb, cb, product, layout, elem);
  if (rc) return rc;
  rc = check_operand(14, C, ldc, psC, m, n, m > 0 && n > 0, layout, elem);
  if (rc) return rc;
  d->opA = opA;
  d->opB = opB;
  d->m = m;
  d->n = n;
  d->k = product ? k : 0;
  std::memcpy(d->alpha, alpha, sizeof(d->alpha));
  std::memcpy(d->beta, beta, sizeof(d->beta));
  d->A = MatView{A, ra, ca, lda, psA};
  d->B = MatView{B, rb, cb, ldb, psB};
  d->C = C;
  d->ldc = ldc;
  d->psc = psC;
  d->layout = layout;
  d->beta_zero = is_zero4(beta);
  d->tri = 0;
  d->krange = 0;
  d->kwidth = 4;
  d->swap = 0;
  return 0;
}

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

namespace {
std::atomic<int> g_last_cuda_error{0};
}  // namespace

int record_cuda_error(cudaError_t e) {
  if (e == cudaSuccess) return QGEMM_SUCCESS;
  g_last_cuda_error.store(static_cast<int>(e));
  return QGEMM_ERR_CUDA;
}

int launch_status() { return record_cuda_error(cudaGetLastError()); }

uint64_t wait_limit_ns() {
  static uint64_t v = [] {
    const char *s = std::getenv("QGEMM_WAIT_LIMIT_MS");
    double ms = s ? std::atof(s) : 2000.0;
    if (!(ms > 0.0)) ms = 2000.0;
    return static_cast<uint64_t>(ms * 1e6);
  }();
  return v;
}

int device_ready() {
  static int cache[64];  // 0 unknown, 1 ok, 2 unusable
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_NO_DEVICE;
  }
  if (dev < 0 || dev >= 64) return QGEMM_ERR_NO_DEVICE;
  if (cache[dev] == 0) {
    int major = 0, minor = 0;
    bool ok = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) ==
                  cudaSuccess &&
              cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) ==
                  cudaSuccess;
    cudaGetLastError();
    cache[dev] = (ok && major == 10 && minor == 3 && encode_tiled_fn() != nullptr) ? 1 : 2;
  }
  return cache[dev] == 1 ? QGEMM_SUCCESS : QGEMM_ERR_NO_DEVICE;
}

// Workspace a validated problem needs for its precision.
int workspace_need(const GemmDesc &d, int precision, size_t *need) {
  *need = 0;
  if (d.k == 0) return QGEMM_SUCCESS;
  if (precision == QGEMM_FP32_SPLIT_BF16) return split_workspace_bytes(d, need);
  if (precision == QGEMM_FP64_SLICED_BF16) return sliced_workspace_bytes(d, need);
  return QGEMM_SUCCESS;
}

int launch_product(const GemmDesc &d, int precision, void *ws, size_t ws_bytes,
                   cudaStream_t s) {
  if (precision == QGEMM_FP64) return launch_fp64_gemm_ws(d, ws, ws_bytes, s);
  if (precision == QGEMM_FP64_SLICED_BF16) return launch_sliced_gemm(d, ws, ws_bytes, s);
  return launch_split_gemm(d, ws, ws_bytes, s);
}

}  // namespace qg

using namespace qg;

extern "C" {

int qgemm(int opA, int opB, int64_t m, int64_t n, int64_t k, const double alpha[4],
          const void *A, int64_t lda, int64_t psA, const void *B, int64_t ldb, int64_t psB,
          const double beta[4], void *C, int64_t ldc, int64_t psC, int layout, int precision,
          void *workspace, size_t workspace_bytes, void *stream) {
  GemmDesc d;
  int rc = validate_gemm(opA, opB, m, n, k, alpha, A, lda, psA, B, ldb, psB, beta, C, ldc, psC,
                         layout, precision, &d);
  if (rc) return rc;
  size_t need = 0;
  rc = workspace_need(d, precision, &need);
  if (rc) return rc;
  if (need > 0) {
    if (workspace == nullptr || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return -19;
    if (workspace_bytes < need) return -20;
  }
  if (m == 0 || n == 0) return QGEMM_SUCCESS;
  rc = device_ready();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d.k == 0) return launch_scale(d, precision_fp64_data(precision), s);
  return launch_product(d, precision, workspace, workspace_bytes, s);
}

int qgemm_split_noalloc(int opA, int opB, int64_t m, int64_t n, int64_t k,
                        const double alpha[4], const void *A, int64_t lda, int64_t psA,
                        const void *B, int64_t ldb, int64_t psB, const double beta[4], void *C,
                        int64_t ldc, int64_t psC, int layout, void *stream) {
  GemmDesc d;
  int rc = validate_gemm(opA, opB, m, n, k, alpha, A, lda, psA, B, ldb, psB, beta, C, ldc, psC,
                         layout, QGEMM_FP32_SPLIT_BF16, &d);
  if (rc) return rc;
  size_t need = 0;
  if (d.k > 0) {
    rc = split_workspace_bytes(d, &need);
    if (rc) return rc;
  }
  if (need > static_cast<size_t>(QGEMM_NOALLOC_SCRATCH_BYTES)) return QGEMM_ERR_WORKSPACE;
  if (m == 0 || n == 0) return QGEMM_SUCCESS;
  rc = device_ready();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d.k == 0) return launch_scale(d, false, s);
  void *scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  return launch_split_gemm(d, scratch, static_cast<size_t>(QGEMM_NOALLOC_SCRATCH_BYTES), s);
}

size_t qgemm_workspace_bytes(int opA, int opB, int64_t m, int64_t n, int64_t k, int layout,
                             int precision) {
  if (!precision_ok(precision)) return 0;
  if (opA < 0 || opA > 3 || opB < 0 || opB > 3 || m < 0 || n < 0 || k < 0) return 0;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return 0;
  if (m == 0 || n == 0 || k == 0) return 0;
  GemmDesc d{};
  d.opA = opA;
  d.opB = opB;
  d.m = m;
  d.n = n;
  d.k = k;
  d.layout = layout;
  // FP64: optional; this much lets a small-m n, long-k product split K
  if (precision == QGEMM_FP64) return fp64_splitk_bytes(m, n, fp64_ksplit(d, device_sms()));
  size_t b = 0;
  if (workspace_need(d, precision, &b)) return 0;
  // tensor-core paths: the required part, then the optional K shares
  if (precision == QGEMM_FP64_SLICED_BF16 && b > 0) b += sliced_splitk_bytes(d);
  if (precision == QGEMM_FP32_SPLIT_BF16 && b > 0) {
    const size_t extra = split_splitk_bytes(d);
    if (extra > 0) b = (b + 255) / 256 * 256 + extra;
  }
  return b;
}

int qherk(int uplo, int trans, int64_t n, int64_t k, double alpha, const void *A, int64_t lda,
          int64_t psA, double beta, void *C, int64_t ldc, int64_t psC, int layout, int precision,
          void *workspace, size_t workspace_bytes, void *stream) {
  if (uplo != QGEMM_LOWER && uplo != QGEMM_UPPER) return -1;
  if (trans != QGEMM_OP_N && trans != QGEMM_OP_H) return -2;
  if (n < 0) return -3;
  if (k < 0) return -4;
  // C <- alpha op(A) op(A)^H + beta C  as the product op(A) * (op(A))^H:
  // op(B) is the conjugate transpose of op(A), on the same matrix.
  const int opB = trans == QGEMM_OP_N ? QGEMM_OP_H : QGEMM_OP_N;
  const double al[4] = {alpha, 0.0, 0.0, 0.0}, be[4] = {beta, 0.0, 0.0, 0.0};
  GemmDesc d;
  int rc = validate_gemm(trans, opB, n, n, k, al, A, lda, psA, A, lda, psA, be, C, ldc, psC,
                         layout, precision, &d);
  if (rc) {
    // qgemm positions -> qherk positions
    static const int map[22] = {0, 2, 2, 3, 3, 4, 5, 6, 7, 8, 6, 7, 8, 9, 10, 11, 12, 13, 14,
                                15, 16, 17};
    const int pos = -rc;
    return (pos >= 1 && pos <= 21) ? -map[pos] : rc;
  }
  d.tri = uplo == QGEMM_LOWER ? 1 : 2;
  size_t need = 0;
  rc = workspace_need(d, precision, &need);
  if (rc) return rc;
  if (need > 0) {
    if (workspace == nullptr || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return -15;
    if (workspace_bytes < need) return -16;
  }
  if (n == 0) return QGEMM_SUCCESS;
  rc = device_ready();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d.k == 0) return launch_herk_scale(d, precision_fp64_data(precision), s);
  return launch_product(d, precision, workspace, workspace_bytes, s);
}

size_t qherk_workspace_bytes(int uplo, int trans, int64_t n, int64_t k, int layout,
                             int precision) {
  if (trans != QGEMM_OP_N && trans != QGEMM_OP_H) return 0;
  if (precision == QGEMM_FP64) {  // optional: lets a small-n, long-k update split K
    if ((uplo != QGEMM_LOWER && uplo != QGEMM_UPPER) || n <= 0 || k <= 0) return 0;
    if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return 0;
    GemmDesc d{};
    d.m = d.n = n;
    d.k = k;
    d.tri = uplo == QGEMM_LOWER ? 1 : 2;
    return fp64_splitk_bytes(n, n, fp64_ksplit(d, device_sms()));
  }
  return qgemm_workspace_bytes(trans, trans == QGEMM_OP_N ? QGEMM_OP_H : QGEMM_OP_N, n, n, k,
                               layout, precision);
}

size_t qgemm_backward_workspace_bytes(int64_t mb, int64_t k, int64_t n, int layout,
                                      int precision) {
  size_t a = qgemm_workspace_bytes(QGEMM_OP_N, QGEMM_OP_H, mb, k, n, layout, precision);
  size_t b = qgemm_workspace_bytes(QGEMM_OP_H, QGEMM_OP_N, k, n, mb, layout, precision);
  return a > b ? a : b;
}

int qgemm_backward(int64_t mb, int64_t k, int64_t n, const void *X, int64_t ldx, int64_t psx,
                   const void *W, int64_t ldw, int64_t psw, const void *dY, int64_t lddy,
                   int64_t psdy, void *dX, int64_t lddx, int64_t psdx, void *dW, int64_t lddw,
                   int64_t psdw, int accumulate, int layout, int precision, void *workspace,
                   size_t workspace_bytes, void *stream) {
  if (mb < 0) return -1;
  if (k < 0) return -2;
  if (n < 0) return -3;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return -20;
  if (!precision_ok(precision)) return -21;
  const double one[4] = {1.0, 0.0, 0.0, 0.0};
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  const double *beta = accumulate ? one : zero;
  // Map qgemm()'s -i positions back to this function's argument numbers.
  auto remap = [](int rc, const int *map) -> int {
    if (rc >= 0) return rc;
    int pos = -rc;
    return (pos >= 1 && pos <= 21 && map[pos]) ? -map[pos] : rc;
  };
  // dX = dY W^H : op(A) = dY (mb x n), op(B) = W^H (n x k), C = dX (mb x k)
  static const int mapX[22] = {0, 0, 0, 1, 2, 3, 0, 10, 11, 12, 7, 8, 9, 0, 13, 14, 15, 20, 21,
                               22, 23};
  // dW = X^H dY : op(A) = X^H (k x mb), op(B) = dY (mb x n), C = dW (k x n)
  static const int mapW[22] = {0, 0, 0, 2, 3, 1, 0, 4, 5, 6, 10, 11, 12, 0, 16, 17, 18, 20, 21,
                               22, 23};
  if (dX != nullptr) {
    int rc = qgemm(QGEMM_OP_N, QGEMM_OP_H, mb, k, n, one, dY, lddy, psdy, W, ldw, psw, beta, dX,
                   lddx, psdx, layout, precision, workspace, workspace_bytes, stream);
    if (rc) return remap(rc, mapX);
  }
  if (dW != nullptr) {
    int rc = qgemm(QGEMM_OP_H, QGEMM_OP_N, k, n, mb, one, X, ldx, psx, dY, lddy, psdy, beta, dW,
                   lddw, psdw, layout, precision, workspace, workspace_bytes, stream);
    if (rc) return remap(rc, mapW);
  }
  return QGEMM_SUCCESS;
}

int qgemm_get_last_device_error(void) {
  if (device_ready() != QGEMM_SUCCESS) return QGEMM_ERR_NO_DEVICE;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  int e = fp64_take_device_error();
  int e2 = split_take_device_error();
  int e3 = grouped_take_device_error();
  int e4 = misc_take_device_error();
  int e5 = sliced_take_device_error();
  int e6 = fp64m_take_device_error();
  if (e) return e;
  if (e2) return e2;
  if (e3) return e3;
  if (e4) return e4;
  if (e5) return e5;
  return e6;
}

const char *qgemm_status_string(int status) {
  if (status < 0) return "invalid argument (-status is its 1-based position)";
  switch (status) {
    case QGEMM_SUCCESS: return "success";
    case QGEMM_ERR_UNSUPPORTED: return "combination not supported";
    case QGEMM_ERR_CUDA: return "CUDA runtime error";
    case QGEMM_ERR_TIMEOUT: return "device wait timed out";
    case QGEMM_ERR_NO_DEVICE: return "no usable sm_103 device";
    case QGEMM_ERR_WORKSPACE: return "workspace missing or too small";
    default: return "unknown status";
  }
}

int qgemm_debug_unsatisfied_wait(uint64_t limit_ns, void *stream) {
  int rc = device_ready();
  if (rc) return rc;
  return debug_unsatisfied_wait(limit_ns, static_cast<cudaStream_t>(stream));
}

int qgemm_debug_arm_fault(int path, int stage, uint64_t limit_ns) {
  if (path != QGEMM_FP64 && path != QGEMM_FP32_SPLIT_BF16) return -1;
  if (stage < 0 || stage > 1000000) return -2;
  if (limit_ns < 1000000ull || limit_ns > 10000000000ull) return -3;
  if (path == QGEMM_FP32_SPLIT_BF16)
    split_arm_fault(stage, limit_ns);
  else
    fp64_arm_fault(stage, limit_ns);
  return QGEMM_SUCCESS;
}

int qgemm_probe_peak(int which, double seconds, double *tflops, void *stream) {
  if (which < 0 || which > 22) return -1;
  if (!(seconds > 0.0) || seconds > 60.0) return -2;
  if (tflops == nullptr) return -3;
  int rc = device_ready();
  if (rc) return rc;
  return probe_peak(which, seconds, tflops, static_cast<cudaStream_t>(stream));
}

const char *qgemm_version(void) { return "gb300-qgemm 0.1"; }

const char *qgemm_last_cuda_error(void) {
  return cudaGetErrorString(static_cast<cudaError_t>(g_last_cuda_error.load()));
}

}  // extern "C"
