// Device-side D3Q19 lattice helpers shared by the CUDA translation units of
// the library (not by the CPU oracle).
#pragma once

#include <cuda_runtime.h>

namespace lbmgb {
namespace {

// D3Q19 velocities in the order documented in lbm.h: direction 2k is the
// opposite of direction 2k-1.  Every loop over directions is unrolled, so
// these fold to immediates.
__host__ __device__ __forceinline__ constexpr int cx_(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int cy_(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int cz_(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}

template <typename C>
__host__ __device__ __forceinline__ constexpr C wgt(int i) {
    return i == 0 ? C(1) / C(3) : (i < 7 ? C(1) / C(18) : C(1) / C(36));
}

// Eq. 8 with u2x = 1.5 |u|^2 precomputed.
template <typename C>
__device__ __forceinline__ C feq(int i, C rho, C ux, C uy, C uz, C u2x) {
    const C cu = C(cx_(i)) * ux + C(cy_(i)) * uy + C(cz_(i)) * uz;
    return rho * wgt<C>(i) * (C(1) + C(3) * cu + C(4.5) * cu * cu - u2x);
}

__device__ __forceinline__ int wrap(int a, int n) {
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
}

// Sum of 19 values as f0 + sum over opposite pairs.
template <typename C>
__device__ __forceinline__ C sum19(const C (&f)[19]) {
    C s = f[0];
#pragma unroll
    for (int i = 1; i < 19; i += 2) s += f[i] + f[i + 1];
    return s;
}

}  // namespace
}  // namespace lbmgb
