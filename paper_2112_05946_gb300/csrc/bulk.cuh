// Bulk asynchronous copies from global to shared memory with a transaction-count mbarrier.
//
// One elected thread initialises the CTA's barrier, announces the bytes it expects and
// issues cp.async.bulk for a contiguous run (16-byte aligned source and destination, size a
// multiple of 16); the copy engine moves the run without occupying the threads, and every
// thread then waits on the barrier's phase.  The wait is bounded: a caller that gives up
// records an error, waits once more (bounded) for the copy still in flight, and returns.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace frsg {

// Bound of a barrier wait, in SM clock cycles (about 1 s at 2 GHz).
constexpr long long kBulkWaitCycles = 2000000000LL;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barrier visible to the copy engine (the async proxy).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// dst (shared) <- src (global), `bytes` bytes; completion is counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier to complete; false after `cycles` SM cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > cycles) return false;
    }
    return true;
}

// True when a run of `bytes` bytes from `src` to `dst` can be one bulk copy.
__device__ __forceinline__ bool bulk_ok(const void* dst, const void* src, size_t bytes) {
    return bytes > 0 && bytes < (1u << 20) && (bytes & 15) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
           (smem_addr(dst) & 15) == 0;
}

}  // namespace frsg
