// Time-step kernels of the two-component Shan-Chen lattice Boltzmann method
// (Milan, Biferale, Sbragaglia, Toschi, arXiv:2112.09972, Sec. 2 Eqs. 6-10,
// Sec. 3 Eq. 14) for sm_103a:
//
//   k_init            -- equilibrium initial state of a tanh droplet in u = A(0) x
//   k_ghost           -- ghost-node rebuild: g_i^eq(rho_b, A(t) (x - x_c)) on the
//                        shell one layer outside the box, for the directions
//                        that stream into the box (Eq. 8, Eq. 14)
//   k_stream_collide  -- fused pull streaming (Eq. 9), component densities
//                        (Eq. 6), Shan-Chen force (Eq. 7), velocity-shift
//                        forcing and BGK relaxation (Eqs. 9, 10); its epilogue
//                        reduces the droplet's centre of mass x_c of the state
//                        it writes (the frame origin of the next step)
//   k_centre          -- the same centre of mass from stored populations
//
// The stream-collide kernel is bandwidth bound (about 1.5 flop per byte), so
// it uses no tensor cores.  Each CTA owns a TX x TY tile of the x-y plane and
// marches along z.  The force at plane z needs the post-streaming densities
// of planes z-1, z, z+1 including a one-node halo around the tile; those live
// in a four-slot ring of density planes in shared memory.  Each plane is
// pulled twice: one plane ahead to sum its densities into the ring, and again
// for the collision.  The second read, and the halo nodes' reads, are served
// by L1/L2 (the neighbouring tiles march the same planes at about the same
// time), so DRAM sees about one read and one write of every population while
// no populations are held on chip across planes, which keeps registers and
// shared memory low and occupancy high.
//
// Sums of populations with opposite velocities are formed as differences of
// the pair first (c_{2k} = -c_{2k-1}); in fp32 this keeps the cancellation in
// momentum and force sums exact where the pair values are close.

#include <cuda_runtime.h>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"

namespace lbmgb {
namespace {

// ----------------------------------------------------------------------------
// Initial state.
template <typename S>
__global__ void k_init(S* __restrict__ f, Layout L, double R, double xi, double rho_hi, double rho_lo, Grad A) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    if (n >= N) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    const double px = x - 0.5 * (L.Lx - 1), py = y - 0.5 * (L.Ly - 1), pz = z - 0.5 * (L.Lz - 1);
    const double r = sqrt(px * px + py * py + pz * pz);
    const double th = tanh((r - R) / xi);
    const double rho[2] = {rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 - th), rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 + th)};
    const double ux = A.a[0] * px + A.a[1] * py + A.a[2] * pz;
    const double uy = A.a[3] * px + A.a[4] * py + A.a[5] * pz;
    const double uz = A.a[6] * px + A.a[7] * py + A.a[8] * pz;
    const double u2x = 1.5 * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 19; ++i) f[L.at(s, i, x, y, z)] = (S)feq<double>(i, rho[s], ux, uy, uz, u2x);
}

// ----------------------------------------------------------------------------
// Ghost nodes.  The shell is covered face by face without overlap:
// x = -1 and x = Lx over y, z in [-1, L]; y = -1 and y = Ly over x in [0, Lx),
// z in [-1, Lz]; z = -1 and z = Lz over x in [0, Lx), y in [0, Ly).  A ghost
// population i is written only if it streams into the box (y + c_i inside).
// Corner nodes stream into no fluid node and write nothing.
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_ghost(S* __restrict__ f, Layout L, Model m, Grad A, CentreParts cp,
                                               int* __restrict__ d_err) {
    // frame origin: the droplet's centre of mass of the current state
    C xc = C(0), yc = C(0), zc = C(0);
    if (m.droplet_frame) {
        xc = (C)cp.sum[4];
        yc = (C)cp.sum[5];
        zc = (C)cp.sum[6];
    }
    // grid: x = fast face coordinate (32-wide blocks), y = slow face
    // coordinate, z = face (0/1: x = -1 / Lx over y, z in [-1, L]; 2/3: y = -1 / Ly
    // over x in [0, Lx), z in [-1, Lz]; 4/5: z = -1 / Lz over x, y inside)
    const int face = blockIdx.z;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y * blockDim.y + threadIdx.y;
    int x, y, z;
    if (face < 2) {
        if (a >= L.Ly + 2 || b >= L.Lz + 2) return;
        x = face ? L.Lx : -1; y = a - 1; z = b - 1;
    } else if (face < 4) {
        if (a >= L.Lx || b >= L.Lz + 2) return;
        y = face == 3 ? L.Ly : -1; x = a; z = b - 1;
    } else {
        if (a >= L.Lx || b >= L.Ly) return;
        z = face == 5 ? L.Lz : -1; x = a; y = b;
    }
    // position relative to the frame origin, then the flow and Eq. 8 in the
    // compute type of the populations (fp64 arithmetic is slow on this part)
    const C px = (C(x) - C(0.5) * C(L.Lx - 1)) - xc, py = (C(y) - C(0.5) * C(L.Ly - 1)) - yc,
            pz = (C(z) - C(0.5) * C(L.Lz - 1)) - zc;
    const C ux = (C)A.a[0] * px + (C)A.a[1] * py + (C)A.a[2] * pz;
    const C uy = (C)A.a[3] * px + (C)A.a[4] * py + (C)A.a[5] * pz;
    const C uz = (C)A.a[6] * px + (C)A.a[7] * py + (C)A.a[8] * pz;
    const C usq = ux * ux + uy * uy + uz * uz;
    const C u2x = C(1.5) * usq;
    bool any = false;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int xi = x + cx_(i), yi = y + cy_(i), zi = z + cz_(i);
        if (xi < 0 || xi >= L.Lx || yi < 0 || yi >= L.Ly || zi < 0 || zi >= L.Lz) continue;
        any = true;
#pragma unroll
        for (int s = 0; s < 2; ++s) f[L.at(s, i, x, y, z)] = (S)feq<C>(i, (C)m.rho_b[s], ux, uy, uz, u2x);
    }
    if (any && (double)usq > m.mach2) atomicOr(d_err, 2);
}

// Fixed-order reduction of the per-CTA centre partials by the last CTA to
// finish (threadfence-reduction pattern); every thread of the CTA calls it.
// `scratch` holds 4 doubles per warp of shared memory.
__device__ void centre_epilogue(double (&cm)[4], CentreParts cp, double* scratch) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = (blockDim.x + 31) >> 5;
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    __shared__ unsigned last;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double a = cm[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) scratch[4 * warp + q] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double a = lane < nwarps ? scratch[4 * lane + q] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) cp.p[4 * cta + q] = a;
        }
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(cp.counter, 1u) == total - 1 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (last && warp == 0) {
        __threadfence();
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        for (unsigned b = lane; b < total; b += 32)
#pragma unroll
            for (int q = 0; q < 4; ++q) s4[q] += __ldcg(cp.p + 4LL * b + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s4[q] += __shfl_down_sync(0xffffffffu, s4[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) cp.sum[q] = s4[q];
            // frame origin x_c = sum w x / sum w (box centre when there is no droplet)
            const bool have = s4[0] > 0.0;
            for (int q = 0; q < 3; ++q) cp.sum[4 + q] = have ? s4[1 + q] / s4[0] : 0.0;
            *cp.counter = 0u;
        }
    }
}

// ----------------------------------------------------------------------------
// Fused pull-stream + Shan-Chen force + collision.
template <typename C>
struct ModelC {
    C inv_tau[2], tau[2], G, rho_b[2];
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
        return L.at(s, i, x, y, z) - ((long long)cz_(i) * L.plane + (long long)cy_(i) * L.pitch + cx_(i));
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

template <typename S, typename C, bool PER, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, Layout L,
                                                          ModelC<C> m, int TX, int TY, int zchunk, CentreParts cp,
                                                          int* __restrict__ d_err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* ring = reinterpret_cast<C*>(smem_raw);
    const int RW = TX + 2, RS = RW * (TY + 2);
    const int NT = TX * TY;
    const int H = 2 * RW + 2 * TY;  // halo nodes per plane
    const int t = threadIdx.x;
    const int tx = t % TX, ty = t / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < L.Lx && y < L.Ly;
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, L.Lz);
    Puller<S, C, PER> P{src, L};

    auto R = [&](int slot, int s, int hx, int hy) -> C& { return ring[(slot * 2 + s) * RS + (hy + 1) * RW + (hx + 1)]; };

    // Densities of the halo ring of plane z into ring slot `slot`.
    auto halo = [&](int z, int slot) {
        for (int h = t; h < H; h += NT) {
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
        C ra, rb;
        P.rho_at(x, y, z, m, ra, rb);
        R(slot, 0, tx, ty) = ra;
        R(slot, 1, tx, ty) = rb;
        halo(z, slot);
    };
    // droplet moments {sum w, sum w x, sum w y, sum w z} of the state written
    // here, w = max(phi, 0); they give the next step's frame origin.  Summed
    // over the thread's z column in the compute type, then reduced in double.
    C cm[4] = {C(0), C(0), C(0), C(0)};
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
            const long long base = L.at(0, 0, x, y, z);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                // tau_s F^s / rho_s = -G tau_s * (the other component's sum)
                const C sh = -m.G * m.tau[s];
                const C ux = up[0] + sh * acc[1 - s][0];
                const C uy = up[1] + sh * acc[1 - s][1];
                const C uz = up[2] + sh * acc[1 - s][2];
                const C u2x = C(1.5) * (ux * ux + uy * uy + uz * uz);
                // moving populations; the rest population then closes the
                // mass balance exactly (sum of outputs = rho), which keeps
                // fp32 rounding from drifting the interface
                C others = C(0);
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    const C f = fc[s][i];
                    const C g = feq<C>(i, rho[s], ux, uy, uz, u2x);
                    const S o = (S)(f - (f - g) * m.inv_tau[s]);
                    dst[base + (long long)(s * 19 + i) * L.array] = o;
                    others += (C)o;
                }
                dst[base + (long long)(s * 19) * L.array] = (S)(rho[s] - others);
            }
        }
    }
    double cmd[4] = {(double)cm[0], (double)cm[1], (double)cm[2], (double)cm[3]};
    centre_epilogue(cmd, cp, reinterpret_cast<double*>(smem_raw));
}

// Centre-of-mass partials of the stored populations (the first step's frame
// origin after an initialisation or an upload of populations).
template <typename S>
__global__ void __launch_bounds__(256) k_centre(const S* __restrict__ f, Layout L, CentreParts cp) {
    __shared__ double scratch[32];
    double cm[4] = {0.0, 0.0, 0.0, 0.0};
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
        const long long b = L.at(0, 0, x, y, z);
        double ra = 0.0, rb = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            ra += (double)f[b + (long long)i * L.array];
            rb += (double)f[b + (long long)(19 + i) * L.array];
        }
        const double phi = (ra - rb) / (ra + rb);
        const double w = phi > 0.0 ? phi : 0.0;
        cm[0] += w;
        cm[1] += w * (x - 0.5 * (L.Lx - 1));
        cm[2] += w * (y - 0.5 * (L.Ly - 1));
        cm[3] += w * (z - 0.5 * (L.Lz - 1));
    }
    centre_epilogue(cm, cp, scratch);
}

template <typename C>
ModelC<C> model_c(const Model& m) {
    ModelC<C> r;
    for (int s = 0; s < 2; ++s) {
        r.tau[s] = (C)m.tau[s];
        r.inv_tau[s] = (C)(1.0 / m.tau[s]);
        r.rho_b[s] = (C)m.rho_b[s];
    }
    r.G = (C)m.G;
    return r;
}

template <typename S, typename C, int MAXT>
cudaError_t stream_collide_t(const void* src, void* dst, const Layout& L, const Model& m, const Shape& sh,
                             CentreParts cp, int* d_err, cudaStream_t s) {
    const ModelC<C> mc = model_c<C>(m);
    if (m.periodic) {
        auto k = k_stream_collide<S, C, true, MAXT>;
        if (sh.smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
        k<<<sh.grid, sh.threads, sh.smem, s>>>((const S*)src, (S*)dst, L, mc, sh.tx, sh.ty, sh.zchunk, cp, d_err);
    } else {
        auto k = k_stream_collide<S, C, false, MAXT>;
        if (sh.smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
        k<<<sh.grid, sh.threads, sh.smem, s>>>((const S*)src, (S*)dst, L, mc, sh.tx, sh.ty, sh.zchunk, cp, d_err);
    }
    return cudaGetLastError();
}

constexpr int kMaxThreadsF32 = 512;
constexpr int kMaxThreadsF64 = 256;

}  // namespace

Layout make_layout(int Lx, int Ly, int Lz, int elem_bytes) {
    Layout L;
    L.Lx = Lx; L.Ly = Ly; L.Lz = Lz;
    const int align = 32 / elem_bytes;  // elements per 32-byte sector
    L.x0 = align;
    L.pitch = ((L.x0 + Lx + 1 + align - 1) / align) * align;
    L.ny = Ly + 2;
    L.nz = Lz + 2;
    L.array = (long long)L.ny * L.pitch;
    L.plane = 38LL * L.array;
    L.total = (long long)L.nz * L.plane;
    return L;
}

Shape choose_shape(const Layout& L, int elem_bytes, int periodic, int ty_req, int zchunk_req, int num_sms) {
    Shape sh;
    sh.rows = 0;
    if (ty_req <= 0 && rows_kernel_applies(L, elem_bytes == 4 ? 1 : 0, periodic)) {
        // one CTA per row
        const int resident = rows_kernel_resident_ctas(L);
        if (resident > 0) {
            // as many z chunks as fill the resident CTA slots once, but at
            // least ~32 planes per chunk: each chunk re-reads two planes
            int chunks = resident / L.Ly;
            const int by_depth = (L.Lz + 31) / 32;
            if (chunks > by_depth) chunks = by_depth;
            if (zchunk_req > 0) chunks = (L.Lz + zchunk_req - 1) / zchunk_req;
            if (chunks < 1) chunks = 1;
            if (chunks > L.Lz) chunks = L.Lz;
            sh.rows = 1;
            sh.tx = L.Lx;
            sh.ty = 1;
            sh.zchunk = (L.Lz + chunks - 1) / chunks;
            sh.grid = dim3(1, L.Ly, (L.Lz + sh.zchunk - 1) / sh.zchunk);
            sh.threads = L.Lx;
            sh.smem = 0;
            return sh;
        }
    }
    const int maxt = elem_bytes == 8 ? kMaxThreadsF64 : kMaxThreadsF32;
    sh.tx = L.Lx <= maxt ? L.Lx : 128;
    if (sh.tx > maxt) sh.tx = maxt;
    int ty = ty_req > 0 ? ty_req : maxt / sh.tx;
    if (ty < 1) ty = 1;
    while (ty > 1 && sh.tx * ty > maxt) --ty;
    if (ty > L.Ly) ty = L.Ly;
    sh.ty = ty;
    const int tiles = ((L.Lx + sh.tx - 1) / sh.tx) * ((L.Ly + sh.ty - 1) / sh.ty);
    int zc = zchunk_req;
    if (zc <= 0) {
        const int want = 2 * (num_sms > 0 ? num_sms : 152);
        int chunks = (want + tiles - 1) / tiles;
        if (chunks < 1) chunks = 1;
        zc = (L.Lz + chunks - 1) / chunks;
        if (zc < 4) zc = 4;
    }
    if (zc > L.Lz) zc = L.Lz;
    sh.zchunk = zc;
    sh.grid = dim3((L.Lx + sh.tx - 1) / sh.tx, (L.Ly + sh.ty - 1) / sh.ty, (L.Lz + zc - 1) / zc);
    sh.threads = sh.tx * sh.ty;
    sh.smem = (size_t)4 * 2 * (sh.tx + 2) * (sh.ty + 2) * elem_bytes;
    const size_t red = (size_t)((sh.threads + 31) / 32) * 4 * sizeof(double);
    if (sh.smem < red) sh.smem = red;
    return sh;
}

cudaError_t launch_init(int prec, void* f, const Layout& L, double R, double xi, double rho_hi, double rho_lo,
                        Grad A0, cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const int T = 256;
    const unsigned blocks = (unsigned)((N + T - 1) / T);
    if (prec == 0) k_init<double><<<blocks, T, 0, s>>>((double*)f, L, R, xi, rho_hi, rho_lo, A0);
    else k_init<float><<<blocks, T, 0, s>>>((float*)f, L, R, xi, rho_hi, rho_lo, A0);
    return cudaGetLastError();
}

cudaError_t launch_ghost(int prec, void* f, const Layout& L, const Model& m, Grad A, CentreParts cp, int* d_err,
                         cudaStream_t s) {
    const int fast = (L.Lx > L.Ly + 2 ? L.Lx : L.Ly + 2);
    const int slow = (L.Lz + 2 > L.Ly ? L.Lz + 2 : L.Ly);
    const dim3 block(32, 8, 1);
    const dim3 grid((fast + 31) / 32, (slow + 7) / 8, 6);
    if (prec == 0) k_ghost<double, double><<<grid, block, 0, s>>>((double*)f, L, m, A, cp, d_err);
    else k_ghost<float, float><<<grid, block, 0, s>>>((float*)f, L, m, A, cp, d_err);
    return cudaGetLastError();
}

cudaError_t launch_centre(int prec, const void* f, const Layout& L, CentreParts cp, cudaStream_t s) {
    if (prec == 0) k_centre<double><<<cp.n, 256, 0, s>>>((const double*)f, L, cp);
    else k_centre<float><<<cp.n, 256, 0, s>>>((const float*)f, L, cp);
    return cudaGetLastError();
}

cudaError_t launch_stream_collide(int prec, const void* src, void* dst, const Layout& L, const Model& m,
                                  const Shape& sh, CentreParts cp, int* d_err, cudaStream_t s) {
    if (sh.rows) return launch_stream_collide_rows(src, dst, L, m, sh.zchunk, cp, d_err, s);
    if (prec == 0) return stream_collide_t<double, double, kMaxThreadsF64>(src, dst, L, m, sh, cp, d_err, s);
    return stream_collide_t<float, float, kMaxThreadsF32>(src, dst, L, m, sh, cp, d_err, s);
}

}  // namespace lbmgb
