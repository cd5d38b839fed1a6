// Bounded-wait test hook and arithmetic-pipe microbenchmarks.
#include <cstdio>

#include "common.cuh"

namespace qg {

__device__ int g_misc_error;
__device__ double g_probe_sink;

namespace {

// Waits on a barrier that nothing arrives on; the bounded wait must give up.
__global__ void unsatisfied_wait_kernel(uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0, limit_ns)) {
    if (threadIdx.x == 0) atomicCAS(&g_misc_error, 0, QGEMM_ERR_TIMEOUT);
  }
}

// ---- throughput probes: NC independent accumulator chains per thread ----
template <int KIND>
__global__ void probe_kernel(int iters, double seed) {
  const int lane = threadIdx.x & 31;
  const double a0 = seed + lane * 1e-3, a1 = a0 * 0.5, b0 = 1.0 - lane * 1e-4, b1 = b0 * 0.5;
  constexpr int NC = 8;
  double acc[NC][4];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[c][j] = 0.0;
  // KIND 2: even warps run the DMMA chains, odd warps 8x as many DFMA
  // iterations (about the same time alone): do the two pipes add up?
  const bool dmma = KIND == 0 || (KIND == 2 && ((threadIdx.x >> 5) & 1) == 0);
  const int n_it = (KIND == 2 && !dmma) ? 8 * iters : iters;
  for (int it = 0; it < n_it; ++it) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (dmma) {
        asm volatile(
            "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
            "{%0,%1,%2,%3};\n"
            : "+d"(acc[c][0]), "+d"(acc[c][1]), "+d"(acc[c][2]), "+d"(acc[c][3])
            : "d"(a0), "d"(a1), "d"(b0));
      } else {
        asm volatile("fma.rn.f64 %0, %1, %2, %0;\n" : "+d"(acc[c][0]) : "d"(a0), "d"(b0));
        asm volatile("fma.rn.f64 %0, %1, %2, %0;\n" : "+d"(acc[c][1]) : "d"(a1), "d"(b1));
      }
    }
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[c][j];
  if (s == 1234.5678) g_probe_sink = s;  // never true; keeps the chains live
}

__global__ void probe_ffma_kernel(int iters, float seed) {
  const float a = seed + threadIdx.x * 1e-3f, b = 0.999f;
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = static_cast<float>(c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 16; ++c) asm volatile("fma.rn.f32 %0, %1, %2, %0;\n" : "+f"(acc[c]) : "f"(a), "f"(b));
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < 16; ++c) s += acc[c];
  if (s == 1234.5678f) g_probe_sink = s;
}

}  // namespace

int probe_tcgen05_bf16(int which, double seconds, double *tflops, cudaStream_t stream);

int debug_unsatisfied_wait(uint64_t limit_ns, cudaStream_t stream) {
  unsatisfied_wait_kernel<<<1, 32, 0, stream>>>(limit_ns);
  return launch_status();
}

int misc_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_misc_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_misc_error, &z, sizeof(int));
  return v;
}

int probe_peak(int which, double seconds, double *tflops, cudaStream_t stream) {
  if ((which >= 3 && which <= 6) || (which >= 8 && which <= 22))
    return probe_tcgen05_bf16(which, seconds, tflops, stream);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 2, threads = (which == 2 || which == 7) ? 512 : 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double flops_per_iter_thread;
  if (which == 0) flops_per_iter_thread = 2.0 * 16 * 8 * 4 * 8 / 32.0;  // 8 DMMA per warp-iter
  else if (which == 1) flops_per_iter_thread = 2.0 * 2 * 8;
  else if (which == 7) flops_per_iter_thread = 0.5 * (2.0 * 16 * 8 * 4 * 8 / 32.0) + 0.5 * 8 * 32;
  else flops_per_iter_thread = 2.0 * 16;
  auto launch = [&](int iters) {
    if (which == 0) probe_kernel<0><<<blocks, threads, 0, stream>>>(iters, 1.0);
    else if (which == 1) probe_kernel<1><<<blocks, threads, 0, stream>>>(iters, 1.0);
    else if (which == 7) probe_kernel<2><<<blocks, threads, 0, stream>>>(iters, 1.0);
    else probe_ffma_kernel<<<blocks, threads, 0, stream>>>(iters, 1.0f);
  };
  int iters = 256;
  float ms = 0.f;
  int rc = QGEMM_SUCCESS;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, stream);
    launch(iters);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = QGEMM_ERR_CUDA; break; }
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 0.5 * seconds * 1e3) break;
    double scale = (seconds * 1e3) / (ms > 0.01 ? ms : 0.01);
    if (scale > 64) scale = 64;
    iters = static_cast<int>(iters * scale);
    if (iters > (1 << 28)) iters = 1 << 28;
  }
  if (rc == QGEMM_SUCCESS && cudaGetLastError() != cudaSuccess) rc = QGEMM_ERR_CUDA;
  if (rc == QGEMM_SUCCESS)
    *tflops = flops_per_iter_thread * iters * static_cast<double>(blocks) * threads / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace qg
