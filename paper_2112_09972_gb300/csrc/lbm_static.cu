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
// any stream capture begins.  The cached address belongs to the device's
// current primary context: after cudaDeviceReset (which discards that
// context and the array with it) the cache is stale, so a process that resets
// a device must not call this entry point on it again.  A launch that fails
// drops the cached address of the device, so the next call looks it up anew.
// All calls share the one array: two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it and give wrong
// results; calls on one stream are ordered and safe.  Every block overwrites
// its own slot of partial sums before the final reduction reads it, so no
// part of the array has to start at zero.
//
// The call's status is that of its own two launches (the return codes of
// cudaLaunchKernel), not the thread's last-error state, so an error left by
// an earlier, unrelated call is neither reported here nor cleared.

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_eigen.cuh"

namespace {

constexpr int kStaticBlocks = 1024;  // partial-sum slots in the scratch array
constexpr int kStaticThreads = 256;

static __device__ __align__(256) double g_moment_scratch[kStaticBlocks * 10];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[128] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; *dev_out receives the device index).
int scratch_for_current_device(double** out, int* dev_out) {
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
    *dev_out = dev;
    return LBM_OK;
}

// Forget the cached address of device dev (after a failed launch).
void drop_scratch(int dev) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    g_scratch_ptr[dev] = nullptr;
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

// Sum the partials (each lane a strided subset of the blocks, then a warp
// shuffle tree: a fixed order, so the result is deterministic) and derive the
// moments, D, axes, eigenvalues and centre in the result layout of
// lbm_deformation, with the same eigen-solver as the context-based path.
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
    if (lane == 0) lbmgb::deformation_from_moments(m, out);
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
    int dev = 0;
    int st = scratch_for_current_device(&scratch, &dev);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long nb = (N + kStaticThreads - 1) / kStaticThreads;
    int blocks = (int)(nb < kStaticBlocks ? nb : kStaticBlocks);
    int Lx = box[0], Ly = box[1], Lz = box[2];
    void* args[] = {(void*)&f, &Lx, &Ly, &Lz, &scratch};
    const void* k = precision == LBM_FP64 ? (const void*)k_moments_dense<double> : (const void*)k_moments_dense<float>;
    cudaError_t e = cudaLaunchKernel(k, dim3(blocks), dim3(kStaticThreads), args, 0, s);
    if (e == cudaSuccess) {
        void* fargs[] = {&scratch, &blocks, &out};
        e = cudaLaunchKernel((const void*)k_moments_dense_final, dim3(1), dim3(32), fargs, 0, s);
    }
    if (e != cudaSuccess) {
        drop_scratch(dev);
        return LBM_ECUDA;
    }
    return LBM_OK;
}
