// Programmatic dependent launch between the kernels of consecutive time
// steps.  A kernel launched with the programmatic-serialization attribute may
// start while the kernel before it in the stream is still running, once every
// CTA of that kernel has called pdl_trigger (or exited); pdl_wait then blocks
// until the kernel before it has completed and its memory is visible, before
// any global read.  The ghost kernel is launched this way: the row kernels
// trigger when their march is done, so the ghost kernel's launch overlaps
// their epilogue (measured at 128^3 fp32: 133.4 us per step against 135.2 us
// without).  The row kernels themselves are launched without the attribute
// (with it, their CTAs started while the ghost kernel ran, were placed
// unevenly over the SMs, and the step took 212 us).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

namespace lbmgb {
namespace {

// Wait until the preceding kernel in the stream has completed and its writes
// are visible (returns at once when there is no programmatic dependency).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Let the next kernel in the stream start its prologue.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The launch attribute that allows a kernel to overlap its predecessor as above.
inline cudaLaunchAttribute pdl_attribute() {
    cudaLaunchAttribute a = {};
    a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a.val.programmaticStreamSerializationAllowed = 1;
    return a;
}

}  // namespace
}  // namespace lbmgb
