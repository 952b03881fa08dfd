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

// MRT collision: row k of the D3Q19 moment basis of d'Humieres et al. (2002)
// at direction i (density, energy, energy square, momentum and energy flux,
// stress and its partners, third-order moments), its squared norm, and the
// relaxation rate of moment k: 1/tau for density, momentum and stress (the
// velocity-shift forcing and Eq. 10), r[0..4] = s_e, s_eps, s_q, s_pi, s_m
// for the rest.
__host__ __device__ __forceinline__ constexpr int mrt_row(int k, int i) {
    const int cx = cx_(i), cy = cy_(i), cz = cz_(i);
    const int c2 = cx * cx + cy * cy + cz * cz;
    switch (k) {
        case 0: return 1;
        case 1: return 19 * c2 - 30;
        case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
        case 3: return cx;
        case 4: return (5 * c2 - 9) * cx;
        case 5: return cy;
        case 6: return (5 * c2 - 9) * cy;
        case 7: return cz;
        case 8: return (5 * c2 - 9) * cz;
        case 9: return 3 * cx * cx - c2;
        case 10: return (3 * c2 - 5) * (3 * cx * cx - c2);
        case 11: return cy * cy - cz * cz;
        case 12: return (3 * c2 - 5) * (cy * cy - cz * cz);
        case 13: return cx * cy;
        case 14: return cy * cz;
        case 15: return cx * cz;
        case 16: return (cy * cy - cz * cz) * cx;
        case 17: return (cz * cz - cx * cx) * cy;
        default: return (cx * cx - cy * cy) * cz;
    }
}
__host__ __device__ __forceinline__ constexpr int mrt_norm(int k) {
    int n = 0;
    for (int i = 0; i < 19; ++i) n += mrt_row(k, i) * mrt_row(k, i);
    return n;
}
template <typename C>
__device__ __forceinline__ C mrt_rate(int k, C inv_tau, const C (&r)[5]) {
    return (k == 0 || k == 3 || k == 5 || k == 7 || k == 9 || k == 11 || k == 13 || k == 14 || k == 15)
               ? inv_tau
               : (k == 1 ? r[0] : (k == 2 ? r[1] : ((k == 4 || k == 6 || k == 8) ? r[2] : ((k == 10 || k == 12) ? r[3] : r[4]))));
}

// out_i = f_i - sum_k M_ki s_k (M dev)_k / |M_k|^2 with dev = f - f_eq.
template <typename C>
__device__ __forceinline__ void mrt_relax(const C (&f)[19], const C (&dev)[19], C inv_tau, const C (&r)[5],
                                          C (&out)[19]) {
    C rel[19];
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        C mk = C(0);
#pragma unroll
        for (int i = 0; i < 19; ++i)
            if (mrt_row(k, i) != 0) mk += C(mrt_row(k, i)) * dev[i];
        rel[k] = mrt_rate<C>(k, inv_tau, r) * mk / C(mrt_norm(k));
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        C back = C(0);
#pragma unroll
        for (int k = 0; k < 19; ++k)
            if (mrt_row(k, i) != 0) back += C(mrt_row(k, i)) * rel[k];
        out[i] = f[i] - back;
    }
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
