// Fifth-generation tensor-core helpers (tcgen05) for the FP32_TC form of the 2D stage:
// TMEM allocation, shared-memory matrix descriptors for the K-major layout without swizzle,
// kind::tf32 MMA with a 32-bit accumulator in TMEM, completion through an mbarrier, and
// TMEM -> register loads.
//
// K-major, no swizzle: the operand is a grid of core matrices of 8 rows x 16 bytes (4 tf32
// values of K), each stored as 128 contiguous bytes, row r of the core matrix at byte 16 r.
// The descriptor's leading-dimension byte offset (LBO) is the distance between core
// matrices adjacent in K, the stride-dimension byte offset (SBO) the distance between core
// matrices adjacent in M (or N).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bulk.cuh"

namespace frsg {

// Byte offset of element (row, k) of a K-major no-swizzle operand with the given LBO / SBO.
__host__ __device__ __forceinline__ unsigned kmajor_offset(int row, int k, unsigned lbo, unsigned sbo) {
    return (unsigned)(row >> 3) * sbo + (unsigned)(k >> 2) * lbo + (unsigned)(row & 7) * 16u + (unsigned)(k & 3) * 4u;
}

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units, the fixed
// descriptor version 1 at bit 46, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc_kmajor(const void* base, unsigned lbo, unsigned sbo) {
    const uint64_t a = smem_addr(base);
    uint64_t d = (a >> 4) & 0x3FFFull;
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::tf32 with an FP32 accumulator, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                    // D: f32
           | (2u << 7)                  // A: tf32
           | (2u << 10)                 // B: tf32
           | ((uint32_t)(N >> 3) << 17) // N / 8
           | ((uint32_t)(M >> 4) << 24);// M / 16
}

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp; the address is
// written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A B^T, M x N x 8 (one kind::tf32 K step), issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1 : 0)
        : "memory");
}

// Arrive once on the mbarrier when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Generic-proxy shared-memory writes made visible to the tensor cores (the async proxy).
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Eight consecutive 32-bit TMEM columns of this thread's lane (warp w reads lanes 32 (w % 4)
// .. + 31; taddr holds the lane base in its upper half), then wait for the load.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// x rounded to the nearest tf32 value (10-bit mantissa), as a float; x - tf32_round(x) is
// then exact in float: the two halves of the 3xTF32 product.
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace frsg
