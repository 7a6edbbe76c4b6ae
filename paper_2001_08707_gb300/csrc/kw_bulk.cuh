// One-dimensional TMA bulk copies from global to shared memory, completed on
// a shared-memory mbarrier, and bounded waits on that barrier (inline PTX,
// sm_90 and later; built for sm_103a).
//
// Protocol of one pipeline stage: one thread arms the stage's barrier with the
// byte count it expects (arrive.expect_tx) and issues the copies; each copy
// adds its bytes to the barrier's transaction count when it lands, and the
// phase completes when every expected byte has arrived.  Every consuming
// thread waits for that phase's parity.  A wait gives up after a fixed number
// of polls (each poll may suspend the thread for up to kBulkPollNs), so a
// copy that never lands makes the kernel report an error instead of hanging.
#pragma once
#include <cstdint>

namespace kw {

constexpr uint32_t kBulkPollNs = 1000;        // suspend-time hint of one poll
constexpr int kBulkMaxPolls = 1 << 20;        // about a second at the hint

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}

// Make the initialised barriers visible to the async proxy (the copy engine).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once on the barrier and expect `bytes` more transaction bytes in this phase.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// One poll: true once the phase with parity `parity` has completed.
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kBulkPollNs)
      : "memory");
  return done != 0;
}

// Bounded wait: false if the phase did not complete within kBulkMaxPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kBulkMaxPolls; ++i)
    if (mbar_poll(bar, parity)) return true;
  return false;
}

// Order this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies into the same bytes (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// memory into this block's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace kw
