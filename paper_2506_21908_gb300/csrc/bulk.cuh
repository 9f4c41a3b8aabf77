// Bulk asynchronous copies (global -> shared) with mbarrier completion, for FP32 kernels that
// stage their inputs in shared memory.  Every wait has an iteration limit; on expiry the caller's
// error word gets a flag bit and the wait is tried once more (again with a limit), so a kernel
// always ends and every index it uses stays in bounds.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace tddft {

constexpr unsigned BULK_WAIT_LIMIT = 1u << 26;

// Polls allowed for the first try of a bounded wait (BULK_WAIT_LIMIT unless the testing hook of
// the failure-detection path, tddft_set_wait_test_limit, shortened it; the retry after an expired
// first try always has the full limit).  One copy per translation unit.
static __device__ unsigned g_first_wait = BULK_WAIT_LIMIT;

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bulk_try_wait(uint32_t bar, uint32_t parity, unsigned limit = BULK_WAIT_LIMIT) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Non-blocking polls (mbarrier.test_wait): the first try shortened by the testing hook counts
// polls that return at once, where one try_wait may itself suspend until the phase completes.
__device__ __forceinline__ bool bulk_test_wait(uint32_t bar, uint32_t parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// First try of a bounded wait: the full try_wait limit, or the testing hook's short test_wait.
__device__ __forceinline__ bool bulk_first_try(uint32_t bar, uint32_t parity) {
  const unsigned lim = g_first_wait;
  return lim >= BULK_WAIT_LIMIT ? bulk_try_wait(bar, parity) : bulk_test_wait(bar, parity, lim);
}

// Wait for phase `parity` of the barrier; on expiry set bit `flag` of *err.
__device__ __forceinline__ void bulk_wait(uint32_t bar, uint32_t parity, int* err, int flag) {
  if (!bulk_first_try(bar, parity)) {
    atomicOr(err, flag);
    bulk_try_wait(bar, parity);
  }
}

// One thread: barriers with an arrival count of 1, made visible to the copy engine.
__device__ __forceinline__ void bulk_init(uint32_t bar0, uint32_t bar1) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread, before the copies of a phase: the earlier shared-memory reads of the buffer (by
// ordinary loads, ordered by a CTA barrier before this call) precede the copy engine's writes;
// the phase completes when `bytes` have arrived.
__device__ __forceinline__ void bulk_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// dst (shared) and src (global) 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sm_addr(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

}  // namespace tddft
