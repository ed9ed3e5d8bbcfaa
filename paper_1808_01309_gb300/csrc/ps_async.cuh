// Asynchronous global->shared copies for sm_103a, in inline PTX:
//   - 1D bulk copies by the tensor-memory-access (TMA) unit completing on an
//     mbarrier (cp.async.bulk ... mbarrier::complete_tx::bytes),
//   - per-thread 8-byte cp.async for strided tiles (8-byte aligned rows).
// Every wait is bounded: after a limit of polls (PS_WAIT_LIMIT unless the
// caller passes another) it gives up and the caller records an error instead
// of hanging the GPU.  A CTA that gave up still waits, up to PS_DRAIN_LIMIT
// polls, for a copy it has in flight before it exits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ps {

#ifndef PS_WAIT_LIMIT
#define PS_WAIT_LIMIT (1u << 26)
#endif
#ifndef PS_DRAIN_LIMIT
#define PS_DRAIN_LIMIT (1u << 27)
#endif

// Error codes written to the plan's device error word.
enum : int { PS_DEV_OK = 0, PS_DEV_TIMEOUT_XPASS = 1, PS_DEV_TIMEOUT_STRIDED = 2 };

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the async proxy (TMA unit).
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Polls the barrier until the phase with the given parity has completed.
// Returns false if it gave up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = PS_WAIT_LIMIT) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Orders earlier generic-proxy accesses to shared memory before later
// async-proxy (TMA) writes into it.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// TMA 1D bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Per-thread asynchronous 8-byte copy global -> shared.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace ps
