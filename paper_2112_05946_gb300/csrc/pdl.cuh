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

}  // namespace frsg
