// Device building blocks of the stream-collide and ghost kernels, shared by
// the single-box kernels (lbm_step.cu) and the batched ensemble kernels
// (lbm_batch.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "lbm_dev.cuh"
#include "lbm_ghost.cuh"
#include "lbm_internal.h"
#include "lbm_centre.cuh"
#include "lbm_lattice.cuh"

namespace lbmgb {
namespace {

// Model scalars in the compute type.
template <typename C>
struct ModelC {
    C inv_tau[2], tau[2], G, rho_b[2];
    C mrt[5];  // MRT free rates s_e, s_eps, s_q, s_pi, s_m (used by MRT instantiations)
};

template <typename S, typename C, bool PER>
struct Puller {
    const S* __restrict__ src;
    Layout L;

    // Element index of population (s, i) pulled into fluid node (x, y, z).
    __device__ __forceinline__ long long idx(int s, int i, int x, int y, int z) const {
        if (PER) {
            return L.at(s, i, wrap(x - cx_(i), L.Lx), wrap(y - cy_(i), L.Ly), wrap(z - cz_(i), L.Lz));
        }
        return L.at(s, i, x, y, z) - ((long long)cz_(i) * L.plane + (long long)cy_(i) * L.row + cx_(i));
    }

    // Pull all 38 populations of fluid node (x, y, z).
    __device__ __forceinline__ void pull(int x, int y, int z, C (&f)[2][19]) const {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 19; ++i) f[s][i] = (C)__ldg(src + idx(s, i, x, y, z));
    }

    // Post-streaming densities at (x, y, z), any position: outside the box
    // the ghost density (or the periodic image).
    __device__ __forceinline__ void rho_at(int x, int y, int z, const ModelC<C>& m, C& ra, C& rb) const {
        if (PER) {
            x = wrap(x, L.Lx); y = wrap(y, L.Ly); z = wrap(z, L.Lz);
        } else if (x < 0 || x >= L.Lx || y < 0 || y >= L.Ly || z < 0 || z >= L.Lz) {
            ra = m.rho_b[0]; rb = m.rho_b[1];
            return;
        }
        C f[2][19];
        pull(x, y, z, f);
        ra = sum19<C>(f[0]);
        rb = sum19<C>(f[1]);
    }
};

// 16-bit deviation storage: the pulled population (s, i >= 1) is rebuilt from
// the node's own rho* and the deviation stored at x - c_i; the rest
// population is the node's own f*_0.
template <typename T, typename C, bool PER>
struct Puller<Dev<T>, C, PER> {
    const Dev<T>* __restrict__ src;
    Layout L;

    // word of the deviation pair of direction i pulled into (x, y, z)
    __device__ __forceinline__ long long idx(int i, int x, int y, int z) const {
        if (PER) return L.dev_word(i, wrap(x - cx_(i), L.Lx), wrap(y - cy_(i), L.Ly), wrap(z - cz_(i), L.Lz));
        return L.dev_word(i, x - cx_(i), y - cy_(i), z - cz_(i));
    }

    __device__ __forceinline__ void pull(int x, int y, int z, C (&f)[2][19]) const {
        const float4 nb = __ldg(reinterpret_cast<const float4*>(src) + L.dev_node(x, y, z));
        f[0][0] = (C)nb.z;
        f[1][0] = (C)nb.w;
        const unsigned* d = reinterpret_cast<const unsigned*>(src);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const float2 v = dev_unpack2<T>(__ldg(d + idx(i, x, y, z)));
            f[0][i] = wgt<C>(i) * (C)nb.x + (C)v.x;
            f[1][i] = wgt<C>(i) * (C)nb.y + (C)v.y;
        }
    }

    __device__ __forceinline__ void rho_at(int x, int y, int z, const ModelC<C>& m, C& ra, C& rb) const {
        if (PER) {
            x = wrap(x, L.Lx); y = wrap(y, L.Ly); z = wrap(z, L.Lz);
        } else if (x < 0 || x >= L.Lx || y < 0 || y >= L.Ly || z < 0 || z >= L.Lz) {
            ra = m.rho_b[0]; rb = m.rho_b[1];
            return;
        }
        C f[2][19];
        pull(x, y, z, f);
        ra = sum19<C>(f[0]);
        rb = sum19<C>(f[1]);
    }
};


// One CTA's share of the stream-collide step: the TX x TY tile at (x0, y0)
// of the x-y plane, marched over planes [zc0, zc1).  blockDim.x may exceed
// TX * TY (the extra threads only help with the halo); every thread must
// call this (it synchronises the block).  Returns the thread's partial
// droplet moments {sum w, sum w x, sum w y, sum w z} of the written state.
template <typename S, typename C, bool PER, bool MRT = false>
__device__ __forceinline__ void tile_march(const S* __restrict__ src, S* __restrict__ dst, const Layout& L,
                                           const ModelC<C>& m, int TX, int TY, int x0, int y0, int zc0, int zc1,
                                           C* ring, int* __restrict__ d_err, C (&cm)[4]) {
    const int RW = TX + 2, RS = RW * (TY + 2);
    const int NT = TX * TY;
    const int H = 2 * RW + 2 * TY;  // halo nodes per plane
    const int t = threadIdx.x;
    const bool in_tile = t < NT;
    const int tx = t % TX, ty = t / TX;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = in_tile && x < L.Lx && y < L.Ly;
    Puller<S, C, PER> P{src, L};

    auto R = [&](int slot, int s, int hx, int hy) -> C& { return ring[(slot * 2 + s) * RS + (hy + 1) * RW + (hx + 1)]; };

    // Densities of the halo ring of plane z into ring slot `slot`.
    auto halo = [&](int z, int slot) {
        for (int h = t; h < H; h += blockDim.x) {
            int hx, hy;
            if (h < RW) { hx = h - 1; hy = -1; }
            else if (h < 2 * RW) { hx = h - RW - 1; hy = TY; }
            else if (h < 2 * RW + TY) { hx = -1; hy = h - 2 * RW; }
            else { hx = TX; hy = h - 2 * RW - TY; }
            C ra, rb;
            P.rho_at(x0 + hx, y0 + hy, z, m, ra, rb);
            R(slot, 0, hx, hy) = ra;
            R(slot, 1, hx, hy) = rb;
        }
    };
    // Densities only (tile + halo) of plane z.
    auto rho_plane = [&](int z, int slot) {
        if (in_tile) {
            C ra, rb;
            P.rho_at(x, y, z, m, ra, rb);
            R(slot, 0, tx, ty) = ra;
            R(slot, 1, tx, ty) = rb;
        }
        halo(z, slot);
    };
    // droplet moments {sum w, sum w x, sum w y, sum w z} of the state written
    // here, w = max(phi, 0); they give the next step's frame origin
    const C pxc = C(x) - C(0.5) * C(L.Lx - 1), pyc = C(y) - C(0.5) * C(L.Ly - 1);

    rho_plane(zc0 - 1, (zc0 - 1) & 3);
    rho_plane(zc0, zc0 & 3);

    for (int z = zc0; z < zc1; ++z) {
        rho_plane(z + 1, (z + 1) & 3);
        __syncthreads();

        if (active) {
            // the node's pulled populations again (second read, from L1/L2)
            C fc[2][19];
            P.pull(x, y, z, fc);
            const int s0 = (z - 1) & 3, s1 = z & 3, s2 = (z + 1) & 3;
            const C rho[2] = {R(s1, 0, tx, ty), R(s1, 1, tx, ty)};
            // momentum of each component (Eq. 6), opposite pairs first
            C j[2][3];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                C jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
                for (int i = 1; i < 19; i += 2) {
                    const C d = fc[s][i] - fc[s][i + 1];
                    if (cx_(i)) jx += C(cx_(i)) * d;
                    if (cy_(i)) jy += C(cy_(i)) * d;
                    if (cz_(i)) jz += C(cz_(i)) * d;
                }
                j[s][0] = jx; j[s][1] = jy; j[s][2] = jz;
            }
            // Shan-Chen force (Eq. 7): F^s = -G rho_s sum_i w_i rho_s'(x + c_i) c_i,
            // with the neighbour pair x + c_i, x - c_i differenced first
            C acc[2][3] = {{C(0), C(0), C(0)}, {C(0), C(0), C(0)}};
#pragma unroll
            for (int i = 1; i < 19; i += 2) {
                const int sp = cz_(i) == 0 ? s1 : (cz_(i) > 0 ? s2 : s0);
                const int sm = cz_(i) == 0 ? s1 : (cz_(i) > 0 ? s0 : s2);
                const C da = wgt<C>(i) * (R(sp, 0, tx + cx_(i), ty + cy_(i)) - R(sm, 0, tx - cx_(i), ty - cy_(i)));
                const C db = wgt<C>(i) * (R(sp, 1, tx + cx_(i), ty + cy_(i)) - R(sm, 1, tx - cx_(i), ty - cy_(i)));
                if (cx_(i)) { acc[0][0] += C(cx_(i)) * da; acc[1][0] += C(cx_(i)) * db; }
                if (cy_(i)) { acc[0][1] += C(cy_(i)) * da; acc[1][1] += C(cy_(i)) * db; }
                if (cz_(i)) { acc[0][2] += C(cz_(i)) * da; acc[1][2] += C(cz_(i)) * db; }
            }
            // common velocity u' and per-component shifted velocity
            const C den = rho[0] * m.inv_tau[0] + rho[1] * m.inv_tau[1];
            C up[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) up[a] = (j[0][a] * m.inv_tau[0] + j[1][a] * m.inv_tau[1]) / den;
            if (!(isfinite(rho[0]) && isfinite(rho[1]))) atomicOr(d_err, 1);
            {
                const C phi = (rho[0] - rho[1]) / (rho[0] + rho[1]);
                const C wphi = phi > C(0) ? phi : C(0);
                cm[0] += wphi;
                cm[1] += wphi * pxc;
                cm[2] += wphi * pyc;
                cm[3] += wphi * (C(z) - C(0.5) * C(L.Lz - 1));
            }
            C rest[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                // tau_s F^s / rho_s = -G tau_s * (the other component's sum)
                const C sh = -m.G * m.tau[s];
                const C ux = up[0] + sh * acc[1 - s][0];
                const C uy = up[1] + sh * acc[1 - s][1];
                const C uz = up[2] + sh * acc[1 - s][2];
                const C u2x = C(1.5) * (ux * ux + uy * uy + uz * uz);
                // post-collision populations: BGK, or MRT relaxation of the moments
                C out[19];
                if constexpr (MRT) {
                    C dv[19];
#pragma unroll
                    for (int i = 0; i < 19; ++i) dv[i] = fc[s][i] - feq<C>(i, rho[s], ux, uy, uz, u2x);
                    mrt_relax<C>(fc[s], dv, m.inv_tau[s], m.mrt, out);
                } else {
#pragma unroll
                    for (int i = 1; i < 19; ++i) {
                        const C f = fc[s][i];
                        out[i] = f - (f - feq<C>(i, rho[s], ux, uy, uz, u2x)) * m.inv_tau[s];
                    }
                }
                // moving populations; the rest population then closes the
                // mass balance exactly (sum of outputs = rho), which keeps
                // fp32 rounding from drifting the interface
                C others = C(0);
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    const C o = out[i];
                    if constexpr (is_dev_t<S>::value) {
                        // deviation from w_i times the density of the node
                        // this population streams to (ring plane z + c_iz)
                        const int sd = cz_(i) == 0 ? s1 : (cz_(i) > 0 ? s2 : s0);
                        const C ref = wgt<C>(i) * R(sd, s, tx + cx_(i), ty + cy_(i));
                        const unsigned short b = dev_from_f<decltype(dev_tag(S{}))>((float)(o - ref));
                        reinterpret_cast<unsigned short*>(dst)[L.dev_at(s, i, x, y, z)] = b;
                        others += ref + (C)dev_to_f<decltype(dev_tag(S{}))>(b);
                    } else {
                        const S os = (S)o;
                        dst[L.at(s, i, x, y, z)] = os;
                        others += (C)os;
                    }
                }
                rest[s] = rho[s] - others;
            }
            if constexpr (is_dev_t<S>::value) {
                reinterpret_cast<float4*>(dst)[L.dev_node(x, y, z)] =
                    make_float4((float)rho[0], (float)rho[1], (float)rest[0], (float)rest[1]);
            } else {
                dst[L.at(0, 0, x, y, z)] = (S)rest[0];
                dst[L.at(1, 0, x, y, z)] = (S)rest[1];
            }
        }
    }
}

// Half h (0 or 1) of a 32-byte sector (32-byte aligned, elements of 4 or 8
// bytes) that holds the bits v at element `lane` and zeros elsewhere: one
// 16-byte store.  Two threads of a warp that write the two halves in the
// same instruction write the sector in one request.
template <typename E>
__device__ __forceinline__ void store_half_sector(E* sector, int lane, E v, int h) {
    static_assert(sizeof(E) == 4 || sizeof(E) == 8, "4- or 8-byte elements");
    constexpr int N = 16 / (int)sizeof(E);
    E e[N];
#pragma unroll
    for (int k = 0; k < N; ++k) e[k] = h * N + k == lane ? v : E(0);
    uint4 w;
    memcpy(&w, e, 16);
    reinterpret_cast<uint4*>(sector)[h] = w;
}
// The whole sector from one thread (both halves); half < 0 in the ghost
// kernels below.
template <typename E>
__device__ __forceinline__ void store_sector_part(E* sector, int lane, E v, int half) {
    if (half < 0) {
        store_half_sector(sector, lane, v, 0);
        store_half_sector(sector, lane, v, 1);
    } else {
        store_half_sector(sector, lane, v, half);
    }
}

// Ghost populations of shell node (x, y, z) of box L (Eq. 8 at the boundary
// density and the flow A (p - x_c), p measured from the box centre; Eq. 14):
// written only for the directions that stream into the box.  Sets error
// bit 2 when the ghost speed exceeds the Mach guard.  half: for an x-face
// node whose values sit alone in sectors of row padding, the half of each
// such sector this thread writes (0 or 1, a pair of threads per node), or
// -1 when the thread writes whole sectors alone; any other ghost value is
// written by the thread with half <= 0.
template <typename S, typename C>
__device__ __forceinline__ void ghost_node(S* __restrict__ f, const Layout& L, const GhostParams<C>& g, C xc, C yc,
                                           C zc, int x, int y, int z, int half, int* __restrict__ d_err) {
    const GhostFlow<C> u = ghost_flow<C>(g, L, xc, yc, zc, x, y, z);
    // An x-face ghost sits alone in a 32-byte sector of row padding (x0 is
    // one sector; when Lx fills whole sectors, so is the stretch after the
    // row).  That sector is written whole -- the value and zero padding,
    // which nothing reads -- so that no partial sector is merged with DRAM.
    constexpr int SEC = 32 / (int)sizeof(S);
    const bool whole = (x == -1 || x == L.Lx) && L.x0 == SEC && L.Lx % SEC == 0;
    const int lane = x == -1 ? SEC - 1 : 0;  // the ghost's place in its sector
    bool any = false;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int xi = x + cx_(i), yi = y + cy_(i), zi = z + cz_(i);
        if (xi < 0 || xi >= L.Lx || yi < 0 || yi >= L.Ly || zi < 0 || zi >= L.Lz) continue;
        any = true;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const S v = (S)ghost_feq<C>(g, u, i, s);
            if (whole) store_sector_part<S>(f + L.at(s, i, x, y, z) - lane, lane, v, half);
            else if (half <= 0) f[L.at(s, i, x, y, z)] = v;
        }
    }
    if (any && u.usq > g.mach2) atomicOr(d_err, 2);
}

// The same for 16-bit deviation storage: the deviation of each inward ghost
// population from w_i rho*(y), y = (x, y, z) + c_i the fluid node it streams
// to (rho* of the state in f), both components of a direction in one 32-bit
// word; x-face words that sit alone in sectors of row padding are written as
// whole sectors (half as in ghost_node).
template <typename T, typename C>
__device__ __forceinline__ void ghost_node_dev(Dev<T>* __restrict__ f, const Layout& L, const GhostParams<C>& gp,
                                               C xc, C yc, C zc, int x, int y, int z, int half,
                                               int* __restrict__ d_err) {
    const GhostFlow<C> u = ghost_flow<C>(gp, L, xc, yc, zc, x, y, z);
    const float4* nb = reinterpret_cast<const float4*>(f);
    unsigned* w32 = reinterpret_cast<unsigned*>(f);
    // words of a row: x0 padding words, the Lx nodes, padding up to pitch
    const bool whole = (x == -1 && L.x0 % 8 == 0) ||
                       (x == L.Lx && (L.x0 + L.Lx) % 8 == 0 && L.pitch >= L.x0 + L.Lx + 8);
    const int lane = x == -1 ? 7 : 0;  // the word's place in its sector
    bool any = false;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int xi = x + cx_(i), yi = y + cy_(i), zi = z + cz_(i);
        if (xi < 0 || xi >= L.Lx || yi < 0 || yi >= L.Ly || zi < 0 || zi >= L.Lz) continue;
        any = true;
        const float4 r = nb[L.dev_node(xi, yi, zi)];
        const C rs[2] = {(C)r.x, (C)r.y};
        unsigned short h[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) h[s] = ghost_dev<T, C>(ghost_feq<C>(gp, u, i, s), wgt<C>(i), rs[s]);
        const unsigned word = (unsigned)h[0] | ((unsigned)h[1] << 16);  // A in the low half
        if (whole) store_sector_part<unsigned>(w32 + L.dev_word(i, x, y, z) - lane, lane, word, half);
        else if (half <= 0) w32[L.dev_word(i, x, y, z)] = word;
    }
    if (any && u.usq > gp.mach2) atomicOr(d_err, 2);
}

// Shell node of face `face` at face coordinates (a, b), or false when
// (a, b) lies outside that face.  Faces 0/1: x = -1 / Lx over y, z in
// [-1, L]; 2/3: y = -1 / Ly over x in [0, Lx), z in [-1, Lz]; 4/5:
// z = -1 / Lz over x in [0, Lx), y in [0, Ly).  Together they cover the
// shell once.
__device__ __forceinline__ bool shell_node(const Layout& L, int face, int a, int b, int& x, int& y, int& z) {
    if (face < 2) {
        if (a >= L.Ly + 2 || b >= L.Lz + 2) return false;
        x = face ? L.Lx : -1; y = a - 1; z = b - 1;
    } else if (face < 4) {
        if (a >= L.Lx || b >= L.Lz + 2) return false;
        y = face == 3 ? L.Ly : -1; x = a; z = b - 1;
    } else {
        if (a >= L.Lx || b >= L.Ly) return false;
        z = face == 5 ? L.Lz : -1; x = a; y = b;
    }
    return true;
}

}  // namespace
}  // namespace lbmgb
