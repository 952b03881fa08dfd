// Reductions and observables over the population field:
//
//   k_moments / k_moments_final -- the droplet's ten float64 moments of
//       w = max(phi, 0), phi = (rho_A - rho_B)/(rho_A + rho_B), reduced with
//       warp shuffles, then the central second-moment tensor, its eigenvalues
//       and eigenvectors (cyclic Jacobi, float64) and the deformation
//       D = (L - W)/(L + W) of Sec. 2, Eq. 4 with L, W proportional to
//       sqrt(lambda_max), sqrt(lambda_min) (a uniform ellipsoid has principal
//       second moments a_k^2 / 5);
//   k_fields    -- rho_A, rho_B and u of the stored populations (Eq. 6);
//   k_checksums -- float64 mass of each component and total momentum;
//   k_pack / k_unpack -- float64 host layout <-> padded device layout.
// Each reads float64, float32 or 16-bit deviation storage (lbm_dev.cuh); the
// latter rebuilds the populations it needs from rho* and the deviations.
//
// Reductions are deterministic: a fixed grid, a fixed in-block tree and a
// fixed-order final pass.

#include <cuda_runtime.h>

#include <type_traits>

#include "lbm_dev.cuh"
#include "lbm_eigen.cuh"
#include "lbm_internal.h"
#include "lbm_lattice.cuh"

namespace lbmgb {
namespace {

__host__ __device__ __forceinline__ constexpr int qx(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int qy(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int qz(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}

constexpr int kRedThreads = 256;

// What 16-bit deviation storage needs to rebuild populations that leave the box.
struct DevRef {
    float rho_b[2];
    int periodic;
};

DevRef dev_ref(const Model& m) {
    DevRef r;
    r.rho_b[0] = (float)m.rho_b[0];
    r.rho_b[1] = (float)m.rho_b[1];
    r.periodic = m.periodic;
    return r;
}

// Post-collision population (s, i) of fluid node (x, y, z).  Deviation
// storage: i = 0 is the stored rest population, i >= 1 is rebuilt as
// w_i rho*(x + c_i) + d_i in float32, the arithmetic of the stream-collide
// kernels (rho_b where x + c_i lies outside the box).
template <typename S>
__device__ __forceinline__ double population(const S* __restrict__ f, const Layout& L, const DevRef& r, int s, int i,
                                             int x, int y, int z) {
    if constexpr (is_dev_t<S>::value) {
        using T = decltype(dev_tag(S{}));
        const float4* nb = reinterpret_cast<const float4*>(f);
        if (i == 0) {
            const float4 o = nb[L.dev_node(x, y, z)];
            return (double)(s ? o.w : o.z);
        }
        int xd = x + qx(i), yd = y + qy(i), zd = z + qz(i);
        float rd = r.rho_b[s];
        if (r.periodic) {
            xd = (xd + L.Lx) % L.Lx; yd = (yd + L.Ly) % L.Ly; zd = (zd + L.Lz) % L.Lz;
        }
        if (xd >= 0 && xd < L.Lx && yd >= 0 && yd < L.Ly && zd >= 0 && zd < L.Lz) {
            const float4 o = nb[L.dev_node(xd, yd, zd)];
            rd = s ? o.y : o.x;
        }
        const unsigned short b = reinterpret_cast<const unsigned short*>(f)[L.dev_at(s, i, x, y, z)];
        return (double)(wgt<float>(i) * rd + dev_to_f<T>(b));
    } else {
        (void)r;
        return (double)f[L.at(s, i, x, y, z)];
    }
}

// hi + lo += v, exactly up to the rounding of lo: TwoSum (Knuth) gives the
// rounding error of hi + v, which lo gathers.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float vv = s - hi;
    const float e = (hi - (s - vv)) + (v - vv);
    hi = s;
    lo += e;
}

// Component densities of fluid node (x, y, z): the sum of its populations,
// or rho* of deviation storage (the same value up to float32 rounding).
template <typename S>
__device__ __forceinline__ void node_rho(const S* __restrict__ f, const Layout& L, int x, int y, int z, double& ra,
                                         double& rb) {
    if constexpr (is_dev_t<S>::value) {
        const float4 o = reinterpret_cast<const float4*>(f)[L.dev_node(x, y, z)];
        ra = o.x;
        rb = o.y;
    } else if constexpr (std::is_same<S, float>::value) {
        // float32 storage: each density as an unevaluated pair hi + lo of
        // float32 sums (Knuth's TwoSum per addition, its rounding errors
        // gathered in lo), so that the 36 additions run on the float32 pipe
        // (this GPU's FP64 pipe runs at 1/64 of its rate); hi + lo agrees
        // with a float64 sum to about 1e-14 relative.
        const long long b = L.at(0, 0, x, y, z);
        float ah = f[b], al = 0.f, bh = f[b + 19LL * L.pitch], bl = 0.f;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            two_sum_acc(ah, al, f[b + (long long)i * L.pitch]);
            two_sum_acc(bh, bl, f[b + (long long)(19 + i) * L.pitch]);
        }
        ra = (double)ah + (double)al;
        rb = (double)bh + (double)bl;
    } else {
        const long long b = L.at(0, 0, x, y, z);
        ra = 0.0;
        rb = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            ra += (double)f[b + (long long)i * L.pitch];
            rb += (double)f[b + (long long)(19 + i) * L.pitch];
        }
    }
}

// Block-wide sum of K doubles per thread; thread 0 writes them to out[0..K).
template <int K>
__device__ void block_sum(double (&v)[K], double* out) {
    __shared__ double part[kRedThreads / 32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double a = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        v[k] = a;
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) part[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = lane < kRedThreads / 32 ? part[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) out[k] = a;
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(kRedThreads) k_moments(const S* __restrict__ f, Layout L, double* __restrict__ partials) {
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const double cx = 0.5 * (L.Lx - 1), cy = 0.5 * (L.Ly - 1), cz = 0.5 * (L.Lz - 1);
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
        double ra, rb;
        node_rho(f, L, x, y, z, ra, rb);
        const double phi = (ra - rb) / (ra + rb);
        const double w = phi > 0.0 ? phi : 0.0;
        const double px = x - cx, py = y - cy, pz = z - cz;
        m[0] += w;
        m[1] += w * px; m[2] += w * py; m[3] += w * pz;
        m[4] += w * px * px; m[5] += w * px * py; m[6] += w * px * pz;
        m[7] += w * py * py; m[8] += w * py * pz; m[9] += w * pz * pz;
    }
    block_sum<10>(m, partials + 10LL * blockIdx.x);
}

// Sum the per-block partials in block order, then derive D and the axes.
__global__ void k_moments_final(const double* __restrict__ partials, int nblocks, double* __restrict__ result) {
    const int lane = threadIdx.x;  // 32 threads
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        double a = 0.0;
        for (int b = lane; b < nblocks; b += 32) a += partials[10LL * b + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        m[k] = a;
    }
    if (lane != 0) return;
    deformation_from_moments(m, result);
}

template <typename S>
__global__ void k_fields(const S* __restrict__ f, Layout L, DevRef dr, double* __restrict__ ra_out,
                         double* __restrict__ rb_out, double* __restrict__ u_out) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    double r[2] = {0.0, 0.0}, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double v = population(f, L, dr, s, i, x, y, z);
            r[s] += v;
            j[0] += qx(i) * v; j[1] += qy(i) * v; j[2] += qz(i) * v;
        }
    if (ra_out) ra_out[n] = r[0];
    if (rb_out) rb_out[n] = r[1];
    if (u_out) {
        const double tot = r[0] + r[1];
        u_out[3 * n + 0] = j[0] / tot;
        u_out[3 * n + 1] = j[1] / tot;
        u_out[3 * n + 2] = j[2] / tot;
    }
}

template <typename S>
__global__ void __launch_bounds__(kRedThreads) k_checksums(const S* __restrict__ f, Layout L, DevRef dr,
                                                           double* __restrict__ partials) {
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const double q = population(f, L, dr, s, i, x, y, z);
                v[s] += q;
                v[2] += qx(i) * q; v[3] += qy(i) * q; v[4] += qz(i) * q;
            }
    }
    block_sum<5>(v, partials + 5LL * blockIdx.x);
}

__global__ void k_checksums_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double a = 0.0;
        for (int b = lane; b < nblocks; b += 32) a += partials[5LL * b + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[k] = a;
    }
}

template <typename S>
__global__ void k_pack(const S* __restrict__ f, Layout L, DevRef dr, double* __restrict__ out) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 38 * N) return;
    const int si = (int)(e / N);
    const long long n = e - si * N;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    out[e] = population(f, L, dr, si / 19, si % 19, x, y, z);
}

// Deviation storage upload, pass 1: rho*_s = float32 of the float64 sum of
// node n's populations, into rho[s * N + n].
__global__ void k_unpack_dev_rho(Layout L, const double* __restrict__ in, float* __restrict__ rho) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        double a = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) a += in[(long long)(s * 19 + i) * N + n];
        rho[s * N + n] = (float)a;
    }
}

// Pass 2: deviations from w_i rho*(x + c_i), node block with the rest
// population closing the node's mass (the arithmetic of the kernels).
template <typename T>
__global__ void k_unpack_dev(Dev<T>* __restrict__ f, Layout L, DevRef dr, const double* __restrict__ in,
                             const float* __restrict__ rho) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    unsigned short* d = reinterpret_cast<unsigned short*>(f);
    float rest[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float others = 0.f;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            int xd = x + qx(i), yd = y + qy(i), zd = z + qz(i);
            if (dr.periodic) {
                xd = (xd + L.Lx) % L.Lx; yd = (yd + L.Ly) % L.Ly; zd = (zd + L.Lz) % L.Lz;
            }
            float rd = dr.rho_b[s];
            if (xd >= 0 && xd < L.Lx && yd >= 0 && yd < L.Ly && zd >= 0 && zd < L.Lz)
                rd = rho[s * N + ((long long)zd * L.Ly + yd) * L.Lx + xd];
            const float ref = wgt<float>(i) * rd;
            const unsigned short b = dev_from_f<T>((float)(in[(long long)(s * 19 + i) * N + n] - (double)ref));
            d[L.dev_at(s, i, x, y, z)] = b;
            others += ref + dev_to_f<T>(b);
        }
        rest[s] = rho[s * N + n] - others;
    }
    reinterpret_cast<float4*>(f)[L.dev_node(x, y, z)] = make_float4(rho[n], rho[N + n], rest[0], rest[1]);
}

template <typename S>
__global__ void k_unpack(S* __restrict__ f, Layout L, const double* __restrict__ in) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 38 * N) return;
    const int si = (int)(e / N);
    const long long n = e - si * N;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    f[L.at(si / 19, si % 19, x, y, z)] = (S)in[e];
}

// ---- connected components of the droplet phase (breakup detection) ----

// label[n] = n where phi > threshold (phi = (rho_A - rho_B) / (rho_A + rho_B)), -1 elsewhere;
// n = (z Ly + y) Lx + x.
template <typename S>
__global__ void k_cc_init(const S* __restrict__ f, Layout L, double threshold, int* __restrict__ label) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    double ra, rb;
    node_rho(f, L, x, y, z, ra, rb);
    label[n] = (ra - rb) / (ra + rb) > threshold ? (int)n : -1;
}

// One sweep of minimum-label propagation over the 6 face neighbours (wrapping
// in the periodic mode), with pointer jumping; sets *changed when a label
// decreased.  Labels only decrease and stay labels of the same component, so
// repeated sweeps converge to the smallest index of each component.
__global__ void k_cc_sweep(Layout L, int periodic, int* __restrict__ label, int* __restrict__ changed) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int own = label[n];
    if (own < 0) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    int m = own;
    const int dx[6] = {1, -1, 0, 0, 0, 0}, dy[6] = {0, 0, 1, -1, 0, 0}, dz[6] = {0, 0, 0, 0, 1, -1};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        int xn = x + dx[q], yn = y + dy[q], zn = z + dz[q];
        if (periodic) {
            xn = (xn + L.Lx) % L.Lx; yn = (yn + L.Ly) % L.Ly; zn = (zn + L.Lz) % L.Lz;
        } else if (xn < 0 || xn >= L.Lx || yn < 0 || yn >= L.Ly || zn < 0 || zn >= L.Lz) {
            continue;
        }
        const int v = label[((long long)zn * L.Ly + yn) * L.Lx + xn];
        if (v >= 0 && v < m) m = v;
    }
    const int jump = label[m];  // the label of the smallest label seen (pointer jumping)
    if (jump >= 0 && jump < m) m = jump;
    if (m < own) {
        label[n] = m;
        *changed = 1;
    }
}

// Component sizes: size[label[n]] += 1; then roots (label[n] == n) append
// (root, size) to out with an atomic counter.
__global__ void k_cc_sizes(Layout L, const int* __restrict__ label, int* __restrict__ size) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int v = label[n];
    if (v >= 0) atomicAdd(size + v, 1);
}

__global__ void k_cc_roots(Layout L, const int* __restrict__ label, const int* __restrict__ size,
                           int* __restrict__ count, long long* __restrict__ out, int cap) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if (label[n] != (int)n) return;
    const int k = atomicAdd(count, 1);
    if (k < cap) out[k] = size[n];
}

// ---- surface-area deformation (Eq. 17) and mass reinjection ----

// phi of every fluid node into phi[n] (n = (z Ly + y) Lx + x) and per-block
// {sum phi, min phi, max phi}.
template <typename S>
__global__ void __launch_bounds__(kRedThreads) k_phi(const S* __restrict__ f, Layout L, double* __restrict__ phi,
                                                     double* __restrict__ partials) {
    __shared__ double red[3][kRedThreads / 32];
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    double sum = 0.0, lo = 1e300, hi = -1e300;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
        double ra, rb;
        node_rho(f, L, x, y, z, ra, rb);
        const double p = (ra - rb) / (ra + rb);
        phi[n] = p;
        sum += p;
        lo = fmin(lo, p);
        hi = fmax(hi, p);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) { red[0][warp] = sum; red[1][warp] = lo; red[2][warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kRedThreads / 32; ++w) {
            red[0][0] += red[0][w];
            red[1][0] = fmin(red[1][0], red[1][w]);
            red[2][0] = fmax(red[2][0], red[2][w]);
        }
        double* out = partials + 4LL * blockIdx.x;
        out[0] = red[0][0]; out[1] = red[1][0]; out[2] = red[2][0];
    }
}

// Per-block sum of |grad phi| (central differences) over interior nodes into partials[4 b + 3].
__global__ void __launch_bounds__(kRedThreads) k_grad_phi(Layout L, const double* __restrict__ phi,
                                                          double* __restrict__ partials) {
    double v[1] = {0.0};
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long sx = 1, sy = L.Lx, sz = (long long)L.Lx * L.Ly;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
        if (x < 1 || x > L.Lx - 2 || y < 1 || y > L.Ly - 2 || z < 1 || z > L.Lz - 2) continue;
        const double gx = 0.5 * (phi[n + sx] - phi[n - sx]);
        const double gy = 0.5 * (phi[n + sy] - phi[n - sy]);
        const double gz = 0.5 * (phi[n + sz] - phi[n - sz]);
        v[0] += sqrt(gx * gx + gy * gy + gz * gz);
    }
    double out[1];
    block_sum<1>(v, out);
    if (threadIdx.x == 0) partials[4LL * blockIdx.x + 3] = out[0];
}

// Block order reduction of the partials: {sum phi, min, max, sum |grad phi|}.
__global__ void k_phi_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double sum = 0.0, lo = 1e300, hi = -1e300, g = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double* p = partials + 4LL * b;
        sum += p[0];
        lo = fmin(lo, p[1]);
        hi = fmax(hi, p[2]);
        g += p[3];
    }
    out[0] = sum; out[1] = lo; out[2] = hi; out[3] = g;
}

// Per-block {mass of A where phi > 0, mass of A elsewhere}.
template <typename S>
__global__ void __launch_bounds__(kRedThreads) k_mass_split(const S* __restrict__ f, Layout L,
                                                            double* __restrict__ partials) {
    double v[2] = {0.0, 0.0};
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
        double ra, rb;
        node_rho(f, L, x, y, z, ra, rb);
        v[(ra - rb) / (ra + rb) > 0.0 ? 0 : 1] += ra;
    }
    block_sum<2>(v, partials + 2LL * blockIdx.x);
}

__global__ void k_mass_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblocks; ++k) { a += partials[2LL * k]; b += partials[2LL * k + 1]; }
    out[0] = a; out[1] = b;
}

// f_A,i *= k at the nodes where phi > 0 (phi of the populations before scaling).
template <typename S>
__global__ void k_reinject(S* __restrict__ f, Layout L, double k) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
    double ra, rb;
    node_rho(f, L, x, y, z, ra, rb);
    if (!((ra - rb) / (ra + rb) > 0.0)) return;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        S* q = f + L.at(0, i, x, y, z);
        *q = (S)((double)*q * k);
    }
}

}  // namespace

int moments_blocks(const Layout& L, int num_sms) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    long long b = (N + kRedThreads - 1) / kRedThreads;
    const long long cap = 4LL * (num_sms > 0 ? num_sms : 152);
    return (int)(b < cap ? b : cap);
}

cudaError_t launch_moments(int prec, const void* f, const Layout& L, double* partials, int nblocks, double* result,
                           cudaStream_t s) {
    if (prec == kFP64) k_moments<double><<<nblocks, kRedThreads, 0, s>>>((const double*)f, L, partials);
    else if (prec == kFP32) k_moments<float><<<nblocks, kRedThreads, 0, s>>>((const float*)f, L, partials);
    else if (prec == kFP16Dev) k_moments<Dev<__half>><<<nblocks, kRedThreads, 0, s>>>((const Dev<__half>*)f, L, partials);
    else k_moments<Dev<__nv_bfloat16>><<<nblocks, kRedThreads, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, partials);
    k_moments_final<<<1, 32, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

cudaError_t launch_fields(int prec, const void* f, const Layout& L, const Model& m, double* ra, double* rb, double* u,
                          cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    const DevRef dr = dev_ref(m);
    if (prec == kFP64) k_fields<double><<<blocks, 256, 0, s>>>((const double*)f, L, dr, ra, rb, u);
    else if (prec == kFP32) k_fields<float><<<blocks, 256, 0, s>>>((const float*)f, L, dr, ra, rb, u);
    else if (prec == kFP16Dev) k_fields<Dev<__half>><<<blocks, 256, 0, s>>>((const Dev<__half>*)f, L, dr, ra, rb, u);
    else k_fields<Dev<__nv_bfloat16>><<<blocks, 256, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, dr, ra, rb, u);
    return cudaGetLastError();
}

cudaError_t launch_checksums(int prec, const void* f, const Layout& L, const Model& m, double* partials, int nblocks,
                             double* result5, cudaStream_t s) {
    const DevRef dr = dev_ref(m);
    if (prec == kFP64) k_checksums<double><<<nblocks, kRedThreads, 0, s>>>((const double*)f, L, dr, partials);
    else if (prec == kFP32) k_checksums<float><<<nblocks, kRedThreads, 0, s>>>((const float*)f, L, dr, partials);
    else if (prec == kFP16Dev)
        k_checksums<Dev<__half>><<<nblocks, kRedThreads, 0, s>>>((const Dev<__half>*)f, L, dr, partials);
    else k_checksums<Dev<__nv_bfloat16>><<<nblocks, kRedThreads, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, dr, partials);
    k_checksums_final<<<1, 32, 0, s>>>(partials, nblocks, result5);
    return cudaGetLastError();
}

cudaError_t launch_pack(int prec, const void* f, const Layout& L, const Model& m, double* out, cudaStream_t s) {
    const long long E = 38LL * L.Lx * L.Ly * L.Lz;
    const unsigned blocks = (unsigned)((E + 255) / 256);
    const DevRef dr = dev_ref(m);
    if (prec == kFP64) k_pack<double><<<blocks, 256, 0, s>>>((const double*)f, L, dr, out);
    else if (prec == kFP32) k_pack<float><<<blocks, 256, 0, s>>>((const float*)f, L, dr, out);
    else if (prec == kFP16Dev) k_pack<Dev<__half>><<<blocks, 256, 0, s>>>((const Dev<__half>*)f, L, dr, out);
    else k_pack<Dev<__nv_bfloat16>><<<blocks, 256, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, dr, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int prec, void* f, const Layout& L, const Model& m, const double* in, float* scratch,
                          cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    if (is_dev(prec)) {
        if (!scratch) return cudaErrorInvalidValue;
        const unsigned blocks = (unsigned)((N + 255) / 256);
        const DevRef dr = dev_ref(m);
        k_unpack_dev_rho<<<blocks, 256, 0, s>>>(L, in, scratch);
        if (prec == kFP16Dev) k_unpack_dev<__half><<<blocks, 256, 0, s>>>((Dev<__half>*)f, L, dr, in, scratch);
        else k_unpack_dev<__nv_bfloat16><<<blocks, 256, 0, s>>>((Dev<__nv_bfloat16>*)f, L, dr, in, scratch);
        return cudaGetLastError();
    }
    const long long E = 38LL * N;
    const unsigned blocks = (unsigned)((E + 255) / 256);
    if (prec == kFP64) k_unpack<double><<<blocks, 256, 0, s>>>((double*)f, L, in);
    else k_unpack<float><<<blocks, 256, 0, s>>>((float*)f, L, in);
    return cudaGetLastError();
}

}  // namespace lbmgb

namespace lbmgb {

cudaError_t launch_cc_init(int prec, const void* f, const Layout& L, double threshold, int* label, cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (prec == kFP64) k_cc_init<double><<<blocks, 256, 0, s>>>((const double*)f, L, threshold, label);
    else if (prec == kFP32) k_cc_init<float><<<blocks, 256, 0, s>>>((const float*)f, L, threshold, label);
    else if (prec == kFP16Dev) k_cc_init<Dev<__half>><<<blocks, 256, 0, s>>>((const Dev<__half>*)f, L, threshold, label);
    else k_cc_init<Dev<__nv_bfloat16>><<<blocks, 256, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, threshold, label);
    return cudaGetLastError();
}

cudaError_t launch_cc_sweep(const Layout& L, int periodic, int* label, int* changed, cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    k_cc_sweep<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(L, periodic, label, changed);
    return cudaGetLastError();
}

cudaError_t launch_cc_sizes(const Layout& L, const int* label, int* size, int* count, long long* out, int cap,
                            cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    k_cc_sizes<<<blocks, 256, 0, s>>>(L, label, size);
    k_cc_roots<<<blocks, 256, 0, s>>>(L, label, size, count, out, cap);
    return cudaGetLastError();
}

}  // namespace lbmgb

namespace lbmgb {

// out[0..3] = {sum phi, min phi, max phi, sum |grad phi| over interior nodes};
// scratch: N doubles (phi) and 4 nblocks doubles.
cudaError_t launch_surface_stats(int prec, const void* f, const Layout& L, double* phi, double* partials, int nblocks,
                                 double* out, cudaStream_t s) {
    if (prec == kFP64) k_phi<double><<<nblocks, kRedThreads, 0, s>>>((const double*)f, L, phi, partials);
    else if (prec == kFP32) k_phi<float><<<nblocks, kRedThreads, 0, s>>>((const float*)f, L, phi, partials);
    else if (prec == kFP16Dev) k_phi<Dev<__half>><<<nblocks, kRedThreads, 0, s>>>((const Dev<__half>*)f, L, phi, partials);
    else k_phi<Dev<__nv_bfloat16>><<<nblocks, kRedThreads, 0, s>>>((const Dev<__nv_bfloat16>*)f, L, phi, partials);
    k_grad_phi<<<nblocks, kRedThreads, 0, s>>>(L, phi, partials);
    k_phi_final<<<1, 32, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

// out[0..1] = {mass of A where phi > 0, elsewhere}; partials: 2 nblocks doubles.
cudaError_t launch_mass_split(int prec, const void* f, const Layout& L, double* partials, int nblocks, double* out,
                              cudaStream_t s) {
    if (prec == kFP64) k_mass_split<double><<<nblocks, kRedThreads, 0, s>>>((const double*)f, L, partials);
    else if (prec == kFP32) k_mass_split<float><<<nblocks, kRedThreads, 0, s>>>((const float*)f, L, partials);
    else return cudaErrorInvalidValue;
    k_mass_final<<<1, 32, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_reinject(int prec, void* f, const Layout& L, double k, cudaStream_t s) {
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (prec == kFP64) k_reinject<double><<<blocks, 256, 0, s>>>((double*)f, L, k);
    else if (prec == kFP32) k_reinject<float><<<blocks, 256, 0, s>>>((float*)f, L, k);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace lbmgb
