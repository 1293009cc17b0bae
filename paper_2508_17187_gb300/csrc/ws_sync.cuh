// Synchronisation and bulk-copy primitives of the warp-specialised kernels (sm_103a, inline PTX):
// shared-memory mbarriers with bounded waits, the tensor-memory-access (TMA) copies (the tile load
// of a grid window, contiguous bulk loads of factor rows), and the cross-proxy fence that orders
// generic shared-memory accesses before an asynchronous (TMA) write to the same memory.
//
// Every wait is bounded.  A thread whose wait does not complete within kWaitLimitNs of %globaltimer
// (or that finds the CTA's abort flag raised) gives up: it raises the abort flag of its CTA, sets
// the launch's error word (reported to the host as AWG_ERR_TIMEOUT by plan_check) and returns
// false, and its caller leaves its loop.  The other roles of the CTA then give up at their next
// wait, so a broken hand-off ends the launch instead of hanging it.
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the library does not link the driver)
#include <cuda_runtime.h>
#include <stdint.h>

namespace awg {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s; a healthy hand-off takes microseconds

// Error word bits (set by atomicOr in the plan's counters[3]).
constexpr unsigned long long kErrWaitTimeout = 1ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the other threads and to the asynchronous proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive (release semantics at CTA scope: this thread's earlier writes are visible to a thread
// that completes a wait on the phase).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

// Arrive and announce `bytes` of asynchronous (TMA) transfer that complete the phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// One bounded test of the phase: the thread may be suspended until the phase completes, for at
// most about kTryWaitHintNs, so that a waiting warp does not spin on the issue slots.
constexpr unsigned kTryWaitHintNs = 1000000u;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kTryWaitHintNs)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of parity `parity` to complete, at most kWaitLimitNs.  Returns false when it
// gave up or when another thread of the CTA raised `abort_flag` (see the file comment).
static __device__ __noinline__ bool mbar_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                       unsigned long long* err_word) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 3) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > kWaitLimitNs) {
        *abort_flag = 1;
        if (err_word) atomicOr(err_word, kErrWaitTimeout);
        return false;
      }
    }
  }
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later asynchronous-proxy
// accesses (a TMA write into memory the CTA has read).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// TMA tile loads into this CTA's shared memory (no multicast; the tensor map describes memory of
// this GPU), completing `bytes` of the barrier's transaction count.  The x coordinate (c0) of
// every load issued here is 0 or a multiple of 16 bytes by construction (see the callers).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// One contiguous copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// this CTA's shared memory, completing its bytes on the barrier's transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace awg
