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

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"
#include "lbm_pdl.cuh"
#include "lbm_tile.cuh"

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

// Initial densities of the tanh droplet at fluid node (x, y, z) (the same
// arithmetic for a node and for the neighbours that refer to it).
__device__ __forceinline__ void init_rho(const Layout& L, double R, double xi, double rho_hi, double rho_lo, int x,
                                         int y, int z, double (&rho)[2]) {
    const double px = x - 0.5 * (L.Lx - 1), py = y - 0.5 * (L.Ly - 1), pz = z - 0.5 * (L.Lz - 1);
    const double r = sqrt(px * px + py * py + pz * pz);
    const double th = tanh((r - R) / xi);
    rho[0] = rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 - th);
    rho[1] = rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 + th);
}

// Initial state in 16-bit deviation storage: the same equilibria as k_init,
// stored as deviations from w_i rho*(x + c_i) (the ghost density rho_b
// outside the box), the rest population closing each node's mass.
template <typename T>
__global__ void k_init_dev(Dev<T>* __restrict__ f, Layout L, double R, double xi, double rho_hi, double rho_lo,
                           Grad A) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    if (n >= N) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    const double px = x - 0.5 * (L.Lx - 1), py = y - 0.5 * (L.Ly - 1), pz = z - 0.5 * (L.Lz - 1);
    double rho[2];
    init_rho(L, R, xi, rho_hi, rho_lo, x, y, z, rho);
    const double ux = A.a[0] * px + A.a[1] * py + A.a[2] * pz;
    const double uy = A.a[3] * px + A.a[4] * py + A.a[5] * pz;
    const double uz = A.a[6] * px + A.a[7] * py + A.a[8] * pz;
    const double u2x = 1.5 * (ux * ux + uy * uy + uz * uz);
    const float rs[2] = {(float)rho[0], (float)rho[1]};
    const float rb[2] = {(float)rho_lo, (float)rho_hi};
    unsigned short* d = reinterpret_cast<unsigned short*>(f);
    float rest[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float others = 0.f;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int xi_ = x + cx_(i), yi = y + cy_(i), zi = z + cz_(i);
            float rd = rb[s];
            if (xi_ >= 0 && xi_ < L.Lx && yi >= 0 && yi < L.Ly && zi >= 0 && zi < L.Lz) {
                double rn[2];
                init_rho(L, R, xi, rho_hi, rho_lo, xi_, yi, zi, rn);
                rd = (float)rn[s];
            }
            const float ref = wgt<float>(i) * rd;
            const float g = (float)feq<double>(i, rho[s], ux, uy, uz, u2x);
            const unsigned short b = dev_from_f<T>(g - ref);
            d[L.dev_at(s, i, x, y, z)] = b;
            others += ref + dev_to_f<T>(b);
        }
        rest[s] = rs[s] - others;
    }
    reinterpret_cast<float4*>(f)[L.dev_node(x, y, z)] = make_float4(rs[0], rs[1], rest[0], rest[1]);
}

// ----------------------------------------------------------------------------
// Ghost nodes (see shell_node for the face enumeration).  Corner nodes stream
// into no fluid node and write nothing.
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_ghost(S* __restrict__ f, Layout L, GhostParams<C> g, CentreParts cp,
                                               int* __restrict__ d_err) {
    // the previous stream-collide launch wrote the frame origin (and, with
    // deviation storage, the densities read below)
    pdl_wait();
    pdl_trigger();
    // frame origin: the droplet's centre of mass of the current state (its
    // float32 copy for the float32 kernels)
    C xc = C(0), yc = C(0), zc = C(0);
    if (g.frame) {
        if constexpr (std::is_same<C, float>::value) {
            xc = cp.frame[0];
            yc = cp.frame[1];
            zc = cp.frame[2];
        } else {
            xc = (C)cp.sum[4];
            yc = (C)cp.sum[5];
            zc = (C)cp.sum[6];
        }
    }
    // x faces: two threads per node (adjacent lanes), each writing half of
    // every padding sector, so that a warp writes 16 whole sectors per store
    const int face = blockIdx.z;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int half = face < 2 ? (a & 1) : -1;
    int x, y, z;
    if (!shell_node(L, face, face < 2 ? a >> 1 : a, blockIdx.y * blockDim.y + threadIdx.y, x, y, z)) return;
    if constexpr (is_dev_t<S>::value)
        ghost_node_dev<decltype(dev_tag(S{})), C>(f, L, g, xc, yc, zc, x, y, z, half, d_err);
    else
        ghost_node<S, C>(f, L, g, xc, yc, zc, x, y, z, half, d_err);
}

template <typename S, typename C, bool PER, bool MRT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, Layout L,
                                                          ModelC<C> m, int TX, int TY, int zchunk, CentreParts cp,
                                                          int* __restrict__ d_err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, L.Lz);
    C cm[4] = {C(0), C(0), C(0), C(0)};
    tile_march<S, C, PER, MRT>(src, dst, L, m, TX, TY, blockIdx.x * TX, blockIdx.y * TY, zc0, zc1,
                          reinterpret_cast<C*>(smem_raw), d_err, cm);
    __syncthreads();  // the ring is reused as reduction scratch
    centre_epilogue(cm, cp, reinterpret_cast<C*>(smem_raw));
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
        double ra = 0.0, rb = 0.0;
        if constexpr (is_dev_t<S>::value) {
            const float4 nb = reinterpret_cast<const float4*>(f)[L.dev_node(x, y, z)];
            ra = nb.x;
            rb = nb.y;
        } else {
            const long long b = L.at(0, 0, x, y, z);
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                ra += (double)f[b + (long long)i * L.pitch];
                rb += (double)f[b + (long long)(19 + i) * L.pitch];
            }
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
    for (int k = 0; k < 5; ++k) r.mrt[k] = (C)m.mrt_rates[k];
    return r;
}

template <typename S, typename C, bool PER, bool MRT, int MAXT>
void stream_collide_launch(const void* src, void* dst, const Layout& L, const ModelC<C>& mc, const Shape& sh,
                           CentreParts cp, int* d_err, cudaStream_t s) {
    auto k = k_stream_collide<S, C, PER, MRT, MAXT>;
    if (sh.smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    k<<<sh.grid, sh.threads, sh.smem, s>>>((const S*)src, (S*)dst, L, mc, sh.tx, sh.ty, sh.zchunk, cp, d_err);
}

template <typename S, typename C, int MAXT>
cudaError_t stream_collide_t(const void* src, void* dst, const Layout& L, const Model& m, const Shape& sh,
                             CentreParts cp, int* d_err, cudaStream_t s) {
    const ModelC<C> mc = model_c<C>(m);
    if (m.periodic) {
        if (m.mrt) stream_collide_launch<S, C, true, true, MAXT>(src, dst, L, mc, sh, cp, d_err, s);
        else stream_collide_launch<S, C, true, false, MAXT>(src, dst, L, mc, sh, cp, d_err, s);
    } else {
        if (m.mrt) stream_collide_launch<S, C, false, true, MAXT>(src, dst, L, mc, sh, cp, d_err, s);
        else stream_collide_launch<S, C, false, false, MAXT>(src, dst, L, mc, sh, cp, d_err, s);
    }
    return cudaGetLastError();
}

constexpr int kMaxThreadsF32 = 512;
constexpr int kMaxThreadsF64 = 256;

}  // namespace

Layout make_layout(int Lx, int Ly, int Lz, int prec) {
    Layout L;
    L.Lx = Lx; L.Ly = Ly; L.Lz = Lz;
    const int align = 32 / elem_bytes_of(prec);  // elements per 32-byte sector
    L.x0 = align;
    L.pitch = ((L.x0 + Lx + 1 + align - 1) / align) * align;
    L.ny = Ly + 2;
    L.nz = Lz + 2;
    // 16-bit deviation storage: 8 units of node block + 36 deviations per node
    // (pitch is a multiple of 16 units, so every float4 block stays 16-byte
    // aligned and row / 8 is whole)
    L.row = (is_dev(prec) ? 44LL : 38LL) * L.pitch;
    L.plane = (long long)L.ny * L.row;
    L.total = (long long)L.nz * L.plane;
    return L;
}

Shape choose_shape(const Layout& L, int prec, int periodic, int mrt, int ty_req, int zchunk_req, int variant_req,
                   int num_sms) {
    Shape sh;
    sh.rows = 0;
    sh.variant = kRowDirect;
    if (ty_req <= 0 && (!mrt || prec == kFP32) && rows_kernel_applies(L, prec, periodic)) {
        // One CTA per row.  MRT rows: direct loads only.  Automatic choice,
        // measured on GB300: shared-memory staging (at 128^3 fp32 129 us per
        // launch against 166 us for direct loads; at 256^3 fp16dev 734 us
        // against 801 us).
        const int automatic = kRowStaged;
        const int variant = mrt ? kRowDirect
                                : (variant_req == 1 ? kRowDirect
                                                    : (variant_req == 2 ? kRowStaged
                                                                        : (variant_req == 3 ? kRowWs : automatic)));
        const int resident = rows_kernel_resident_ctas(L, prec, variant, mrt);
        if (resident > 0) {
            // Chunks of about 43 planes: measured on GB300 at 128^3 (384 CTAs,
            // one wave) and 256^3 (1536 CTAs) against 8 to 64 planes.
            // Consecutive chunks march in opposite directions, so the two
            // planes a chunk boundary shares are read at the same time (at the
            // start or the end of both marches) and L2 serves the second
            // read.  Small boxes take more chunks (down to 8 planes) to reach
            // half the resident CTA count.
            int chunks = (L.Lz + 43) / 44;
            if (variant == kRowWs) {
                // long chunks, all CTAs resident at once when the rows fit
                // (a second, partial wave would leave SMs idle)
                if (resident >= L.Ly) chunks = resident / L.Ly;
                if (chunks > L.Lz / 8) chunks = L.Lz / 8;
            } else if (2 * chunks * L.Ly < resident) {
                chunks = resident / (2 * L.Ly);
                if (chunks > L.Lz / 8) chunks = L.Lz / 8;
            }
            // A grid that is one wave takes the most chunks that still fit in
            // one wave (measured at 128^3 with 16-bit storage, 4 resident CTAs
            // per SM: 4 chunks 107.6 us, 3 chunks 118.8 us per launch).
            if (variant != kRowWs && chunks * L.Ly <= resident)
                while ((chunks + 1) * L.Ly <= resident && chunks + 1 <= L.Lz / 8) ++chunks;
            if (zchunk_req > 0) chunks = (L.Lz + zchunk_req - 1) / zchunk_req;
            if (chunks < 1) chunks = 1;
            if (chunks > L.Lz) chunks = L.Lz;
            sh.rows = 1;
            sh.variant = variant;
            sh.tx = L.Lx;
            sh.ty = 1;
            sh.zchunk = (L.Lz + chunks - 1) / chunks;
            sh.grid = dim3(1, L.Ly, (L.Lz + sh.zchunk - 1) / sh.zchunk);
            sh.threads = L.Lx;
            sh.smem = 0;
            return sh;
        }
    }
    const int cbytes = prec == kFP64 ? 8 : 4;  // compute type of the density ring
    const int maxt = prec == kFP64 ? kMaxThreadsF64 : kMaxThreadsF32;
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
    sh.smem = (size_t)4 * 2 * (sh.tx + 2) * (sh.ty + 2) * cbytes;
    const size_t red = (size_t)((sh.threads + 31) / 32) * 4 * sizeof(double);
    if (sh.smem < red) sh.smem = red;
    return sh;
}

cudaError_t launch_init(int prec, void* f, const Layout& L, double R, double xi, double rho_hi, double rho_lo,
                        Grad A0, cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const int T = 256;
    const unsigned blocks = (unsigned)((N + T - 1) / T);
    if (prec == kFP64) k_init<double><<<blocks, T, 0, s>>>((double*)f, L, R, xi, rho_hi, rho_lo, A0);
    else if (prec == kFP32) k_init<float><<<blocks, T, 0, s>>>((float*)f, L, R, xi, rho_hi, rho_lo, A0);
    else if (prec == kFP16Dev) k_init_dev<__half><<<blocks, T, 0, s>>>((Dev<__half>*)f, L, R, xi, rho_hi, rho_lo, A0);
    else k_init_dev<__nv_bfloat16><<<blocks, T, 0, s>>>((Dev<__nv_bfloat16>*)f, L, R, xi, rho_hi, rho_lo, A0);
    return cudaGetLastError();
}

cudaError_t launch_ghost(int prec, void* f, const Layout& L, const Model& m, Grad A, CentreParts cp, int* d_err,
                         cudaStream_t s) {
    const int fast = (L.Lx > 2 * (L.Ly + 2) ? L.Lx : 2 * (L.Ly + 2));  // x faces: two threads per node
    const int slow = (L.Lz + 2 > L.Ly ? L.Lz + 2 : L.Ly);
    const dim3 block(32, 8, 1);
    const dim3 grid((fast + 31) / 32, (slow + 7) / 8, 6);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = s;
    cudaLaunchAttribute attr[1] = {pdl_attribute()};
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (prec == kFP64)
        return cudaLaunchKernelEx(&cfg, k_ghost<double, double>, (double*)f, L, ghost_params<double>(m, A.a), cp, d_err);
    const GhostParams<float> g = ghost_params<float>(m, A.a);
    if (prec == kFP32) return cudaLaunchKernelEx(&cfg, k_ghost<float, float>, (float*)f, L, g, cp, d_err);
    if (prec == kFP16Dev)
        return cudaLaunchKernelEx(&cfg, k_ghost<Dev<__half>, float>, (Dev<__half>*)f, L, g, cp, d_err);
    return cudaLaunchKernelEx(&cfg, k_ghost<Dev<__nv_bfloat16>, float>, (Dev<__nv_bfloat16>*)f, L, g, cp, d_err);
}

cudaError_t launch_centre(int prec, const void* f, const Layout& L, CentreParts cp, cudaStream_t s) {
    if (prec == kFP64) k_centre<double><<<cp.n, 256, 0, s>>>((const double*)f, L, cp);
    else if (prec == kFP32) k_centre<float><<<cp.n, 256, 0, s>>>((const float*)f, L, cp);
    else if (prec == kFP16Dev) k_centre<Dev<__half>><<<cp.n, 256, 0, s>>>((const Dev<__half>*)f, L, cp);
    else k_centre<Dev<__nv_bfloat16>><<<cp.n, 256, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, cp);
    return cudaGetLastError();
}

cudaError_t launch_stream_collide(int prec, const void* src, void* dst, const Layout& L, const Model& m,
                                  const Shape& sh, const Grad& A, CentreParts cp, int* d_err, cudaStream_t s) {
    if (sh.rows) return launch_stream_collide_rows(prec, sh.variant, src, dst, L, m, A, sh.zchunk, cp, d_err, s);
    if (prec == kFP64) return stream_collide_t<double, double, kMaxThreadsF64>(src, dst, L, m, sh, cp, d_err, s);
    if (prec == kFP32) return stream_collide_t<float, float, kMaxThreadsF32>(src, dst, L, m, sh, cp, d_err, s);
    if (prec == kFP16Dev) return stream_collide_t<Dev<__half>, float, kMaxThreadsF32>(src, dst, L, m, sh, cp, d_err, s);
    return stream_collide_t<Dev<__nv_bfloat16>, float, kMaxThreadsF32>(src, dst, L, m, sh, cp, d_err, s);
}

}  // namespace lbmgb
