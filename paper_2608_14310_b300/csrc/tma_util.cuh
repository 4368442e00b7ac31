// TMA bulk copies and mbarrier waits (inline PTX), shared by the patch-apply kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cav {

__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}
__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded waits.  A wait gives up after WAIT_LIMIT clock cycles (about a second), records
// DEV_TIMEOUT in the status word and returns false; the host reads the word after the call
// and reports IB_ERR_TIMEOUT.  g_wait_stall is a test hook (set from the host through
// ib_test_wait_stall): while it is non-zero every stallable wait (a wait for data: a copy
// landing, a gathered vector) ignores its barrier and runs out after WAIT_LIMIT_STALL cycles,
// so tests can drive the timeout path without a fault; waits for free buffer space are not
// stallable, so copies are in flight when the data waits give up.
// Each translation unit that includes this header holds its own copy of the flag.
constexpr long long WAIT_LIMIT = 1LL << 31;
constexpr long long WAIT_LIMIT_STALL = 1LL << 20;
static __device__ int g_wait_stall = 0;

// The test hook's state, read once at kernel entry (it does not change while kernels run).
__device__ inline bool wait_stall_enabled() { return g_wait_stall != 0; }

// Wait for the phase with the given parity to complete.  `abort` (shared memory, nullable)
// is a CTA-wide flag: a wait also gives up (without recording a status) once another thread
// of the CTA has set it, and a wait that runs out sets it, so the other roles of the CTA stop
// waiting on work that will not come.  `stall`: this wait is stalled by the test hook (the
// caller passes wait_stall_enabled() for waits for data, false otherwise).
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, int* status, volatile int* abort = nullptr,
                                 bool stall = false) {
  if (!stall && mbar_try_wait(bar, parity)) return true;  // the common case: no clock read
  const long long limit = stall ? WAIT_LIMIT_STALL : WAIT_LIMIT;
  const long long t0 = clock64();
  while (stall || !mbar_try_wait(bar, parity)) {
    if (abort && *abort) return false;
    if (clock64() - t0 > limit) {
      atomicExch(status, DEV_TIMEOUT);
      if (abort) *abort = 1;
      return false;
    }
  }
  return true;
}
// Wait for a bulk copy this CTA issued to land before the CTA exits (shared memory must not
// be released with a copy in flight).  Not subject to the stall hook; bounded all the same.
__device__ inline void mbar_drain(uint64_t* bar, uint32_t parity, int* status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_LIMIT) {
      atomicExch(status, DEV_TIMEOUT);
      return;
    }
  }
}
// 1-D bulk copy global -> this CTA's shared memory, completing `bytes` on the mbarrier.
__device__ inline void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Prefetch `bytes` (a multiple of 16) at a 16-byte aligned global address into L2.
__device__ inline void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

}  // namespace cav
