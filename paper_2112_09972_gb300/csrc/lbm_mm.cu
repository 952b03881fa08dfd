// Maffettone-Minale droplet model (Sec. 2, Eqs. 1, 2, 4, 5 of Milan et al.,
// arXiv:2112.09972) for many gradient histories at once: one thread per
// trajectory integrates the morphology tensor M with classical RK4 and
// records D.  The paper compares its LBM droplets with this model; batching
// it on the GPU gives the model's deformation statistics over as many tracer
// trajectories as the LBM ensemble (Sec. 6).
//
// With tau_d = eta_s R / sigma, Ca(t) = tau_d ||G(t)||_inf (Eq. 3, element-wise
// maximum) and G = A the velocity gradient in lattice units,
//   dM/dt = [ f2(chi, Ca) tau_d (S M + M S) + tau_d (W M - M W)
//             - f1(chi) (M - 3 III_M / II_M I) ] / tau_d
// in LBM time, S and W the symmetric and antisymmetric parts of A (Eq. 2),
// II_M = ((tr M)^2 - M:M) / 2, III_M = det M, f1 and f2 of Eq. 5.  A(t) is the
// table row at integer t, linear in between.  D = (L - W)/(L + W) with L, W
// the square roots of M's extreme eigenvalues (Eq. 4).

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm.h"
#include "lbm_eigen.cuh"

namespace lbmgb_mm {
namespace {

// symmetric 3x3 as 6 entries: xx, xy, xz, yy, yz, zz
template <typename C>
struct Sym {
    C v[6];
};

template <typename C>
__device__ __forceinline__ C at(const Sym<C>& m, int a, int b) {
    constexpr int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return m.v[idx[a][b]];
}

template <typename C>
__device__ __forceinline__ Sym<C> rhs(const Sym<C>& M, const C (&A)[9], C tau_d, C chi) {
    C S[3][3], W[3][3], amax = C(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            S[a][b] = C(0.5) * (A[3 * a + b] + A[3 * b + a]);
            W[a][b] = C(0.5) * (A[3 * a + b] - A[3 * b + a]);
            amax = fmax(amax, fabs(A[3 * a + b]));
        }
    const C Ca = tau_d * amax;
    const C f1 = C(40) * (chi + C(1)) / ((C(3) + C(2) * chi) * (C(16) + C(19) * chi));
    const C f2 = C(5) / (C(3) + C(2) * chi) + C(3) * Ca * Ca / (C(2) + C(6) * Ca * Ca);
    // invariants
    const C tr = M.v[0] + M.v[3] + M.v[5];
    const C mm = M.v[0] * M.v[0] + M.v[3] * M.v[3] + M.v[5] * M.v[5] +
                 C(2) * (M.v[1] * M.v[1] + M.v[2] * M.v[2] + M.v[4] * M.v[4]);
    const C II = C(0.5) * (tr * tr - mm);
    const C III = M.v[0] * (M.v[3] * M.v[5] - M.v[4] * M.v[4]) - M.v[1] * (M.v[1] * M.v[5] - M.v[4] * M.v[2]) +
                  M.v[2] * (M.v[1] * M.v[4] - M.v[3] * M.v[2]);
    const C iso = C(3) * III / II;
    Sym<C> out;
    constexpr int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int a = ia[e], b = ib[e];
        C sm = C(0), ms = C(0), wm = C(0), mw = C(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sm += S[a][k] * at(M, k, b);
            ms += at(M, a, k) * S[k][b];
            wm += W[a][k] * at(M, k, b);
            mw += at(M, a, k) * W[k][b];
        }
        const C flow = f2 * tau_d * (sm + ms) + tau_d * (wm - mw);
        const C relax = f1 * (M.v[e] - (a == b ? iso : C(0)));
        out.v[e] = (flow - relax) / tau_d;
    }
    return out;
}

template <typename C>
__device__ __forceinline__ Sym<C> axpy(const Sym<C>& m, C h, const Sym<C>& k) {
    Sym<C> r;
#pragma unroll
    for (int e = 0; e < 6; ++e) r.v[e] = m.v[e] + h * k.v[e];
    return r;
}

template <typename C>
__device__ double deformation(const Sym<C>& M) {
    double a[3][3] = {{(double)M.v[0], (double)M.v[1], (double)M.v[2]},
                      {(double)M.v[1], (double)M.v[3], (double)M.v[4]},
                      {(double)M.v[2], (double)M.v[4], (double)M.v[5]}};
    double lam[3], v[3][3];
    lbmgb::jacobi3(a, lam, v);
    const double hi = sqrt(fmax(fmax(lam[0], fmax(lam[1], lam[2])), 0.0));
    const double lo = sqrt(fmax(fmin(lam[0], fmin(lam[1], lam[2])), 0.0));
    return hi + lo > 0.0 ? (hi - lo) / (hi + lo) : 0.0;
}

template <typename C>
__global__ void k_mm_rk4(const double* __restrict__ A, long long T, long long n, C tau_d, C chi, int substeps,
                         int record_every, double* __restrict__ D, double* __restrict__ Mout) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    Sym<C> M;
#pragma unroll
    for (int e = 0; e < 6; ++e) M.v[e] = (e == 0 || e == 3 || e == 5) ? C(1) : C(0);
    D[k] = deformation(M);
    const C h = C(1) / C(substeps);
    C a0[9], a1[9];
    for (long long s = 0; s + 1 < T; ++s) {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            a0[j] = (C)A[(s * n + k) * 9 + j];
            a1[j] = (C)A[((s + 1) * n + k) * 9 + j];
        }
        for (int q = 0; q < substeps; ++q) {
            // A at the start, middle and end of the substep (linear in t)
            const C t0 = C(q) * h, tm = (C(q) + C(0.5)) * h, te = C(q + 1) * h;
            C as[9], am[9], ae[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const C d = a1[j] - a0[j];
                as[j] = a0[j] + t0 * d;
                am[j] = a0[j] + tm * d;
                ae[j] = a0[j] + te * d;
            }
            const Sym<C> k1 = rhs(M, as, tau_d, chi);
            const Sym<C> k2 = rhs(axpy(M, C(0.5) * h, k1), am, tau_d, chi);
            const Sym<C> k3 = rhs(axpy(M, C(0.5) * h, k2), am, tau_d, chi);
            const Sym<C> k4 = rhs(axpy(M, h, k3), ae, tau_d, chi);
#pragma unroll
            for (int e = 0; e < 6; ++e)
                M.v[e] += (h / C(6)) * (k1.v[e] + C(2) * k2.v[e] + C(2) * k3.v[e] + k4.v[e]);
        }
        if ((s + 1) % record_every == 0) D[((s + 1) / record_every) * n + k] = deformation(M);
    }
    if (Mout)
#pragma unroll
        for (int e = 0; e < 6; ++e) Mout[k * 6 + e] = (double)M.v[e];
}

}  // namespace
}  // namespace lbmgb_mm

extern "C" int lbm_mm_integrate(const double* A, int64_t T, int64_t n, double tau_d, double chi, int32_t substeps,
                                int32_t record_every, int32_t precision, double* D, double* M, void* cuda_stream) {
    if (!A || !D || T < 1 || n < 1 || !(tau_d > 0.0) || !(chi > 0.0) || substeps < 1 || record_every < 1)
        return LBM_EINVAL;
    if (precision != LBM_FP64 && precision != LBM_FP32) return LBM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    if (precision == LBM_FP64)
        lbmgb_mm::k_mm_rk4<double><<<blocks, threads, 0, s>>>(A, T, n, tau_d, chi, substeps, record_every, D, M);
    else
        lbmgb_mm::k_mm_rk4<float><<<blocks, threads, 0, s>>>(A, T, n, (float)tau_d, (float)chi, substeps,
                                                             record_every, D, M);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
