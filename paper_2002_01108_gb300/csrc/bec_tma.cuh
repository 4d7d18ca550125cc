// Tensor-memory-access (TMA) copies and mbarrier waits for the pass kernels
// that stage their tiles in shared memory: 2D tiled loads that complete on
// an mbarrier, 2D tiled stores tracked as bulk groups, and the proxy fence
// that orders a block's shared-memory writes before a store reads them.
// Every wait is bounded (about 0.2 s) and reports running out instead of
// spinning on.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace bec {
namespace {

constexpr long long kTmaSpinCycles = 400000000LL;   // ~0.2 s at 2 GHz

__device__ __forceinline__ uint32_t tma_smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void tma_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// makes the barrier initialisation visible to the asynchronous proxy
__device__ __forceinline__ void tma_fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Waits for the completion of phase parity ph; false when it ran out.
__device__ __forceinline__ bool tma_mbar_wait(uint32_t bar, uint32_t ph) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(ph)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kTmaSpinCycles) return false;
  }
}

// box at element coordinates (c0 innermost, c1) of `map` into shared memory
// at dst; completes `bytes` of transaction on bar (elements outside the
// tensor read as zero)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// shared memory at src to the box at (c0, c1) of `map` (elements outside the
// tensor are not written); part of the thread's current bulk group
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int c0, int c1, uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(src)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2,
                                             uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(src)
      : "memory");
}

__device__ __forceinline__ void tma_commit_group() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// the thread's committed stores have finished reading shared memory
__device__ __forceinline__ void tma_wait_group_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// the thread's committed stores are complete
__device__ __forceinline__ void tma_wait_group0() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// orders this thread's generic-proxy shared-memory writes before later
// asynchronous-proxy reads (a TMA store) of the same memory
__device__ __forceinline__ void tma_fence_proxy_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace
}  // namespace bec
