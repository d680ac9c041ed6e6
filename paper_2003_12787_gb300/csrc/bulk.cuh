// Bulk asynchronous copies (the TMA engine without a tensor map) of one
// element's contiguous AoS block from global into shared memory, completing
// on an mbarrier's transaction count: one instruction replaces thousands of
// dependent loads (the transposition on entry of Sec. V-B then runs from
// shared memory).
#pragma once
#include <stdint.h>

namespace stp {
namespace bulk {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Whether a copy of `bytes` from `src` is possible (16-byte alignment and
// size; the shared destination is aligned by the caller).
__device__ __forceinline__ bool can_copy(const void* src, uint64_t bytes) {
  return (reinterpret_cast<uintptr_t>(src) & 15u) == 0 && (bytes & 15u) == 0 && bytes < (1u << 20);
}

// One thread: expect `bytes` on the barrier and start the copy.
__device__ __forceinline__ void start(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, int limit = 1 << 22) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// a later bulk copy into the same bytes (with a barrier in between).
__device__ __forceinline__ void fence_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Orders this thread's earlier generic-proxy global writes before later
// bulk-copy reads of them.
__device__ __forceinline__ void fence_global_writes() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

}  // namespace bulk
}  // namespace stp
