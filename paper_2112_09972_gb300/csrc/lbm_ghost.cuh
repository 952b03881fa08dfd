// Ghost-node arithmetic (Sec. 2, Eq. 8 at the boundary density; Sec. 3,
// Eq. 14 for the flow) of the ghost kernels of the single box and of the
// batched ensemble, which write the ghost shell that the stream-collide
// kernels pull from.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <limits>

#include "lbm_dev.cuh"
#include "lbm_internal.h"
#include "lbm_lattice.cuh"

namespace lbmgb {
namespace {

// Parameters of the ghost rebuild in its arithmetic type C, converted once
// on the host: the float32 kernels then run no FP64 instruction (this GPU's
// FP64 pipe runs at 1/64 of the float32 rate).
template <typename C>
struct GhostParams {
    C A[9];     // the boundary gradient of the step, row-major
    C rho_b[2]; // ghost densities
    C mach2;    // |u|^2 above this sets the Mach flag
    int frame;  // 1: the flow is centred on the droplet's centre of mass
};
// mach2 for type C: in float32 the largest float not above the double guard
// g, so that for every float u, u > mach2 exactly when (double)u > g.
template <typename C>
GhostParams<C> ghost_params(const Model& m, const double (&A)[9]) {
    GhostParams<C> p;
    for (int j = 0; j < 9; ++j) p.A[j] = (C)A[j];
    for (int s = 0; s < 2; ++s) p.rho_b[s] = (C)m.rho_b[s];
    C g = (C)m.mach2;
    if ((double)g > m.mach2) g = std::nextafter(g, -std::numeric_limits<C>::infinity());
    p.mach2 = g;
    p.frame = m.droplet_frame;
    return p;
}

// The flow at ghost node (x, y, z): u = A (p - x_c), p measured from the box
// centre (Eq. 14), with |u|^2 and 1.5 |u|^2.
template <typename C>
struct GhostFlow {
    C ux, uy, uz, usq, u2x;
};
template <typename C>
__device__ __forceinline__ GhostFlow<C> ghost_flow(const GhostParams<C>& g, const Layout& L, C xc, C yc, C zc, int x,
                                                   int y, int z) {
    const C (&A)[9] = g.A;
    const C px = (C(x) - C(0.5) * C(L.Lx - 1)) - xc, py = (C(y) - C(0.5) * C(L.Ly - 1)) - yc,
            pz = (C(z) - C(0.5) * C(L.Lz - 1)) - zc;
    GhostFlow<C> u;
    u.ux = A[0] * px + A[1] * py + A[2] * pz;
    u.uy = A[3] * px + A[4] * py + A[5] * pz;
    u.uz = A[6] * px + A[7] * py + A[8] * pz;
    u.usq = u.ux * u.ux + u.uy * u.uy + u.uz * u.uz;
    u.u2x = C(1.5) * u.usq;
    return u;
}

// Ghost population (component s, direction i) of Eq. 8.
template <typename C>
__device__ __forceinline__ C ghost_feq(const GhostParams<C>& g, const GhostFlow<C>& u, int i, int s) {
    return feq<C>(i, g.rho_b[s], u.ux, u.uy, u.uz, u.u2x);
}

// 16-bit deviation storage: the deviation of ghost value gv (direction i,
// weight w) from w rs, rs the rho* of the fluid node it streams to.
template <typename T, typename C>
__device__ __forceinline__ unsigned short ghost_dev(C gv, C w, C rs) {
    return dev_from_f<T>((float)(gv - w * rs));
}

}  // namespace
}  // namespace lbmgb
