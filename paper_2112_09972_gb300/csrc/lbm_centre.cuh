// Centre-of-mass partials of a stream-collide launch, reduced in a fixed
// order (warp shuffles, then the last CTA to finish), and the frame origin
// for the next step.  Shared by the row kernels and the generic tile kernel.
// Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbmgb {
namespace {

// Fixed-order reduction of centre partials by the last CTA to finish
// (threadfence-reduction pattern); every thread of the CTA calls it.  C is
// the reduction type (float32 for the float32 and 16-bit storage kernels, so
// that they run no FP64 instruction; float64 for the float64 kernel).  This
// CTA's partials go to parts[4 slot .. 4 slot + 3]; `total` CTAs share the
// counter; the last of them sums slots 0 .. total - 1 in order into sum8
// (the four sums, then x_c, y_c, z_c) and frame (x_c in float32), and resets
// the counter.  `scratch` holds 4 values of C per warp of shared memory.
template <typename C>
__device__ void centre_reduce(C (&cm)[4], C* parts, long long slot, unsigned total, unsigned* counter, double* sum8,
                              float* frame, C* scratch) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = (blockDim.x + 31) >> 5;
    __shared__ unsigned last;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        C a = cm[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) scratch[4 * warp + q] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            C a = lane < nwarps ? scratch[4 * lane + q] : C(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) parts[4 * slot + q] = a;
        }
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(counter, 1u) == total - 1 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (last && warp == 0) {
        __threadfence();
        C s4[4] = {C(0), C(0), C(0), C(0)};
        for (unsigned b = lane; b < total; b += 32)
#pragma unroll
            for (int q = 0; q < 4; ++q) s4[q] += __ldcg(parts + 4LL * b + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s4[q] += __shfl_down_sync(0xffffffffu, s4[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) sum8[q] = (double)s4[q];
            // frame origin x_c = sum w x / sum w (box centre when there is no droplet)
            const bool have = s4[0] > C(0);
            for (int q = 0; q < 3; ++q) {
                const C xc = have ? s4[1 + q] / s4[0] : C(0);
                sum8[4 + q] = (double)xc;
                frame[q] = (float)xc;
            }
            *counter = 0u;
        }
    }
}

// The same over every CTA of the launch, in CTA order, into CentreParts.
template <typename C>
__device__ void centre_epilogue(C (&cm)[4], CentreParts cp, C* scratch) {
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    centre_reduce(cm, reinterpret_cast<C*>(cp.p), cta, total, cp.counter, cp.sum, cp.frame, scratch);
}

}  // namespace
}  // namespace lbmgb
