// tcgen05.cuh -- the pieces of the fifth-generation tensor-core interface
// (sm_103a) that the tensor-core kernels share: shared-memory addresses and
// matrix descriptors, the bounded mbarrier wait, and the global timer.
#pragma once

#include <cstdint>

namespace lrs {
namespace tc {

constexpr unsigned long long kWaitNs = 2000000000ull;   // every mbarrier wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of
// 8 rows x 16 bytes stored contiguously (128 bytes); the two core matrices of
// one MMA's 32-byte K step are 128 bytes apart (leading byte offset),
// consecutive groups of 8 rows 256 bytes apart (stride byte offset); version 1
// at bit 46.  Element (r, k) of a K step sits at byte (r / 8) 256 + (k-byte /
// 16) 128 + (r % 8) 16 + k-byte % 16.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until the mbarrier has completed the phase of the given parity;
// false when that takes longer than kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.b32 %0, 1, 0, q;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (now_ns() - t0 > kWaitNs) return false;
      __nanosleep(64);
    }
  }
}

}  // namespace tc
}  // namespace lrs
