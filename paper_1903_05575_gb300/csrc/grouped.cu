// Grouped persistent quaternion GEMM -- under construction.
#include "common.cuh"

namespace qg {

__device__ int g_grouped_error;

int grouped_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_grouped_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_grouped_error, &z, sizeof(int));
  return v;
}

}  // namespace qg

extern "C" {

int qgemm_batched_grouped(const qgemm_problem *, int64_t, int, int, void *, size_t, void *) {
  return QGEMM_ERR_UNSUPPORTED;
}
size_t qgemm_grouped_workspace_bytes(const qgemm_problem *, int64_t, int, int) { return 0; }
int qgemm_grouped_prepare(const qgemm_problem *, int64_t, int, int, void *, size_t, void *) {
  return QGEMM_ERR_UNSUPPORTED;
}
int qgemm_grouped_launch(void *, void *) { return QGEMM_ERR_UNSUPPORTED; }

}  // extern "C"
