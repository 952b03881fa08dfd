// Allocation-free droplet moments: lbm_moments_static (declared in lbm.h).
//
// Some callers cannot allocate device memory at the moment they need the
// droplet's shape: code running inside a stream that is being captured into a
// CUDA graph (where cudaMalloc is not permitted), real-time loops that must
// not touch the allocator, or hosts that hand this library a fixed memory
// budget.  This entry point serves them.  It reads populations the caller
// already holds on the device and writes the result to a device buffer the
// caller provides; the per-block partial sums it needs live in one
// file-scope device array of fixed size, so the call performs no allocation
// of any kind.
//
// The scratch array is a static __device__ symbol: every GPU that loads the
// library holds it (kStaticBlocks * 10 doubles = 80 KB) until the process
// exits.  In host code its name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, once per device, on the
// first call made while that device is current.  Make that first call before
// any stream capture begins.  All calls share the one array: two calls whose
// kernels overlap on the GPU (different streams, no ordering between them)
// race on it and give wrong results; calls on one stream are ordered and safe.
// Every block overwrites its own slot of partial sums before the final
// reduction reads it, so no part of the array has to start at zero.

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/lbm.h"

namespace {

constexpr int kStaticBlocks = 1024;  // partial-sum slots in the scratch array
constexpr int kStaticThreads = 256;

static __device__ __align__(256) double g_moment_scratch[kStaticBlocks * 10];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[128] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    if (dev < 0 || dev >= 128) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_moment_scratch) != cudaSuccess || !p) return LBM_ECUDA;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

// Per-block sums of the ten moments of w = max(phi, 0) over a dense
// [2][19][Lz][Ly][Lx] population array (x fastest).
template <typename S>
__global__ void __launch_bounds__(kStaticThreads) k_moments_dense(const S* __restrict__ f, int Lx, int Ly, int Lz,
                                                                  double* __restrict__ partials) {
    const long long N = (long long)Lx * Ly * Lz;
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    const double cx = 0.5 * (Lx - 1), cy = 0.5 * (Ly - 1), cz = 0.5 * (Lz - 1);
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        double ra = 0.0, rb = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            ra += (double)f[(long long)i * N + n];
            rb += (double)f[(long long)(19 + i) * N + n];
        }
        const double phi = (ra - rb) / (ra + rb);
        const double w = phi > 0.0 ? phi : 0.0;
        const double px = (double)(n % Lx) - cx;
        const double py = (double)((n / Lx) % Ly) - cy;
        const double pz = (double)(n / ((long long)Lx * Ly)) - cz;
        m[0] += w;
        m[1] += w * px; m[2] += w * py; m[3] += w * pz;
        m[4] += w * px * px; m[5] += w * px * py; m[6] += w * px * pz;
        m[7] += w * py * py; m[8] += w * py * pz; m[9] += w * pz * pz;
    }
    __shared__ double part[kStaticThreads / 32][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        double a = m[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) part[warp][k] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            double a = lane < kStaticThreads / 32 ? part[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) partials[10LL * blockIdx.x + k] = a;
        }
    }
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations.
__device__ void jacobi3_static(double a[3][3], double lam[3], double v[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        const double scale = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off <= 1e-300 || off <= 1e-17 * scale) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int k = 0; k < 3; ++k) lam[k] = a[k][k];
}

// Sum the partials in block order; moments, D, axes, eigenvalues and centre
// in the result layout of lbm_moments_static.
__global__ void k_moments_dense_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    const int lane = threadIdx.x;
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
    for (int k = 0; k < 10; ++k) out[k] = m[k];
    const double mass = m[0];
    const double c[3] = {m[1] / mass, m[2] / mass, m[3] / mass};
    double I[3][3];
    I[0][0] = m[4] / mass - c[0] * c[0];
    I[0][1] = I[1][0] = m[5] / mass - c[0] * c[1];
    I[0][2] = I[2][0] = m[6] / mass - c[0] * c[2];
    I[1][1] = m[7] / mass - c[1] * c[1];
    I[1][2] = I[2][1] = m[8] / mass - c[1] * c[2];
    I[2][2] = m[9] / mass - c[2] * c[2];
    double lam[3], v[3][3];
    jacobi3_static(I, lam, v);
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[ord[j]] > lam[ord[i]]) { const int tmp = ord[i]; ord[i] = ord[j]; ord[j] = tmp; }
    for (int k = 0; k < 3; ++k) {
        const int col = ord[k];
        int big = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(v[a][col]) > fabs(v[big][col])) big = a;
        const double sgn = v[big][col] < 0.0 ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) out[11 + 3 * a + k] = sgn * v[a][col];
        out[20 + k] = lam[col];
        out[23 + k] = c[k];
    }
    const double a1 = sqrt(fmax(lam[ord[0]], 0.0)), a3 = sqrt(fmax(lam[ord[2]], 0.0));
    out[10] = (a1 - a3) / (a1 + a3);
}

}  // namespace

extern "C" int lbm_moments_static(const void* f, int32_t precision, const int32_t box[3], double* out,
                                  void* cuda_stream) {
    if (!f || !out || !box) return LBM_EINVAL;
    if (precision != LBM_FP64 && precision != LBM_FP32) return LBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (box[a] < 1) return LBM_EINVAL;
    const long long N = (long long)box[0] * box[1] * box[2];
    // largest box this entry point accepts: 38 N population elements must be
    // addressable, and the partial sums of at most kStaticBlocks blocks fit
    // the scratch array whatever N is
    if (N > (1LL << 31) / 38) return LBM_EINVAL;
    double* scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long nb = (N + kStaticThreads - 1) / kStaticThreads;
    const int blocks = (int)(nb < kStaticBlocks ? nb : kStaticBlocks);
    if (precision == LBM_FP64)
        k_moments_dense<double><<<blocks, kStaticThreads, 0, s>>>((const double*)f, box[0], box[1], box[2], scratch);
    else
        k_moments_dense<float><<<blocks, kStaticThreads, 0, s>>>((const float*)f, box[0], box[1], box[2], scratch);
    k_moments_dense_final<<<1, 32, 0, s>>>(scratch, blocks, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
