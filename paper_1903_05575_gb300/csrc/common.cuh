// Device-side helpers shared by the library's kernels: shared-memory
// barriers with bounded waits, tensor-memory-accelerator (TMA) loads, and
// the quaternion basis sign table.  sm_103a only.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace qg {

// Sign of the basis product e_p e_q = sign * e_(p xor q)  (Sec. 2.1,
// Eq. quaternion_alg).  Bit (4p + q) set <=> the sign is negative:
//   e1e1 = e2e2 = e3e3 = -e0,  e1e3 = -e2,  e2e1 = -e3,  e3e2 = -e1.
constexpr uint32_t kBasisNegMask =
    (1u << (4 * 1 + 1)) | (1u << (4 * 1 + 3)) |
    (1u << (4 * 2 + 1)) | (1u << (4 * 2 + 2)) |
    (1u << (4 * 3 + 2)) | (1u << (4 * 3 + 3));

__host__ __device__ constexpr int basis_sign(int p, int q) {
  return ((kBasisNegMask >> (4 * p + q)) & 1u) ? -1 : 1;
}

// Mask of negative entries of the real 4x4 block that maps the components
// b^j of op(B)'s element to the components c of the product op(A)_e * op(B)_e:
// (a b)^c = sum_j sign(c, j) a^(c xor j) b^j with sign(c, j) =
// basis_sign(c^j, j), times -1 for a conjugated A component c^j != 0 and
// for a conjugated B component j != 0.  Bit (4c + j).
__host__ __device__ constexpr uint32_t block_neg_mask(bool conjA, bool conjB) {
  uint32_t mask = 0;
  for (int c = 0; c < 4; ++c)
    for (int j = 0; j < 4; ++j) {
      int p = c ^ j;
      int s = basis_sign(p, j);
      if (conjA && p != 0) s = -s;
      if (conjB && j != 0) s = -s;
      if (s < 0) mask |= 1u << (4 * c + j);
    }
  return mask;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- mbarrier -----------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete, for at most
// limit_ns nanoseconds.  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// ---- TMA ----------------------------------------------------------------
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t c0, int32_t c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t c0, int32_t c1, int32_t c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t c0, int32_t c1, int32_t c2, int32_t c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
      "r"(c3)
      : "memory");
}

// ---- FP64 bit helpers (integer ops: the FP64 pipe is scarce on GB300) ----
__device__ __forceinline__ double flip_sign(double x, uint32_t neg_hi) {
  return __hiloint2double(__double2hiint(x) ^ static_cast<int>(neg_hi), __double2loint(x));
}

}  // namespace qg
