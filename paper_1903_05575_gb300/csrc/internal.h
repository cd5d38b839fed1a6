// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "qgemm.h"

namespace qg {

// One operand as the kernels see it: element (r, c) of the STORED matrix,
// component s, lives at ptr + s*cs + r*rs + c*ld (reals).  Interleaved:
// cs = 1, rs = 4, ld = 4*ld_q.  Split planes: cs = plane stride, rs = 1.
struct MatView {
  const void *ptr;
  int64_t rows, cols;  // stored extent (elements)
  int64_t ld;          // leading dimension (elements)
  int64_t ps;          // plane stride (reals, split layout only)
  int width = 4;       // components stored per element: 4 quaternion, 2 complex, 1 real
};

// Description of one GEMM after validation.
struct GemmDesc {
  int opA, opB;
  int64_t m, n, k;
  double alpha[4], beta[4];
  MatView A, B;
  void *C;
  int64_t ldc, psc;
  int layout;
  bool beta_zero;
  int tri = 0;  // 0: full C; 1: lower triangle only; 2: upper (Hermitian rank-k update)
  // k-range of an output tile when one operand is triangular (qtrmm): 0 all
  // of K; 1 kappa < tile row end; 2 kappa >= tile row start; 3 kappa >= tile
  // column start; 4 kappa < tile column end.
  int krange = 0;
  // Mixed types (qgemm_mixed): components of op(A) per kappa in the real
  // form (A.width: 4, or 2 / 1 for a complex / real left operand, so K' =
  // kwidth * k), and swap = 1 when the product was turned around,
  // D = op(B)^H op(A)^H, and C = conj(D)^T is stored.
  int kwidth = 4;
  int swap = 0;
};

inline bool op_trans(int op) { return op == QGEMM_OP_T || op == QGEMM_OP_H; }
inline bool op_conj(int op) { return op == QGEMM_OP_C || op == QGEMM_OP_H; }

// Tensor-map encoder from the driver (fetched once, without linking libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();

// Status of the launches just made: QGEMM_SUCCESS, or QGEMM_ERR_CUDA with the
// CUDA error recorded for qgemm_last_cuda_error().
int launch_status();
int record_cuda_error(cudaError_t e);

// FP64 product on the FP64 FMA pipe (fp64_dfma.cu): whether a product takes
// it, and its launch.
bool fp64_dfma_eligible(const GemmDesc &d, int sms);
int launch_fp64_dfma(const GemmDesc &d, cudaStream_t stream);

// Device wait limit for bounded spins (env QGEMM_WAIT_LIMIT_MS, default 2000).
uint64_t wait_limit_ns();

// Checks that a usable device is current; returns a QGEMM status.
int device_ready();

inline bool precision_ok(int p) {
  return p == QGEMM_FP64 || p == QGEMM_FP32_SPLIT_BF16 || p == QGEMM_FP64_SLICED_BF16;
}
inline bool precision_fp64_data(int p) { return p != QGEMM_FP32_SPLIT_BF16; }

// Launchers (return QGEMM status codes).
int launch_fp64_gemm(const GemmDesc &d, cudaStream_t stream);
// The FP64 product with an optional caller workspace: when fp64_ksplit() > 1
// and the workspace holds that many partial products (fp64_splitk_bytes), K
// is split across CTAs and a second kernel sums the partials.
int launch_fp64_gemm_ws(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream);
int fp64_ksplit(const GemmDesc &d, int sms);
size_t fp64_splitk_bytes(int64_t m, int64_t n, int ksplit);
int device_sms();  // SM count of the current device (152 when there is none)
// C <- alpha (sum over z < ks of the partial products in part) + beta C in FP64
// for an FP64 C (d's layout, scalars and triangle); part: ks dense slabs of
// m n interleaved quaternions, summed in z order.
int launch_splitk_reduce(const GemmDesc &d, const double *part, int ks, cudaStream_t stream);
int launch_fp64_mixed(const GemmDesc &d, cudaStream_t stream);
int launch_scale(const GemmDesc &d, bool fp64, cudaStream_t stream);
int launch_herk_scale(const GemmDesc &d, bool fp64, cudaStream_t stream);
int split_workspace_bytes(const GemmDesc &d, size_t *bytes);
int launch_split_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream);
int noalloc_scratch(void **out);
int sliced_workspace_bytes(const GemmDesc &d, size_t *bytes);
// Optional workspace after sliced_workspace_bytes() that lets a single
// digit-sliced product split K (0 when it would not).
size_t sliced_splitk_bytes(const GemmDesc &d);
// Optional workspace after split_workspace_bytes() (rounded up to 256 bytes)
// that lets a single split-BF16 product split K (0 when it would not).
size_t split_splitk_bytes(const GemmDesc &d);
int launch_sliced_gemm(const GemmDesc &d, void *ws, size_t ws_bytes, cudaStream_t stream);
int validate_gemm(int opA, int opB, int64_t m, int64_t n, int64_t k, const double *alpha,
                  const void *A, int64_t lda, int64_t psA, const void *B, int64_t ldb,
                  int64_t psB, const double *beta, void *C, int64_t ldc, int64_t psC,
                  int layout, int precision, GemmDesc *d);

// Device status words of each translation unit (read and cleared).
int fp64_take_device_error();
int split_take_device_error();
int grouped_take_device_error();
int misc_take_device_error();
int sliced_take_device_error();
int fp64m_take_device_error();
int debug_unsatisfied_wait(uint64_t limit_ns, cudaStream_t stream);
// One-shot fault injection: the next split-BF16 GEMM launch leaves out the
// copies of its TMA warp's running stage `stage` and waits at most limit_ns.
void split_arm_fault(int stage, uint64_t limit_ns);
// The same for the next FP64 GEMM launch (its first CTA's ring stage `stage`).
void fp64_arm_fault(int stage, uint64_t limit_ns);
int probe_peak(int which, double seconds, double *tflops, cudaStream_t stream);

}  // namespace qg
