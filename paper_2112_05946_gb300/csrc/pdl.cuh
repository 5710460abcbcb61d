// Programmatic dependent launch: a kernel lets the next launch in its stream start as soon as
// all of its CTAs are running (launch_dependents), and waits for the previous kernel's
// completion and memory (wait) only before it touches the state.  Everything before the wait
// reads launch-invariant data (tables, scalars, dt written before the launch); all global
// writes come after it.  Without a programmatic dependency both instructions are no-ops.
#pragma once

#include <cuda_runtime.h>

namespace frsg {

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Asynchronous global -> shared copy of one 4- or 8-byte element (cp.async, L1-allocating):
// the warp does not wait for it; cp_async_wait_all() waits for this thread's copies, and a
// barrier after it publishes them to the CTA.  Several sweeps of loads (tables, then the state
// after pdl_wait) thus stay in flight together instead of one round trip each.
template <typename T>
__device__ __forceinline__ void cp_async(T* dst_shared, const T* src_global) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element of 4 or 8 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src_global), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace frsg
