// Batched ensemble of independent droplet boxes (the statistics over many
// tracer trajectories that the paper's conclusion, Sec. 6, calls for).
//
// Every box is a full copy of the single-box method (ghost boundary, fused
// stream + Shan-Chen force + collision, droplet frame), with its own size,
// radius and per-step velocity-gradient history.  One time step of the whole
// ensemble is two launches:
//
//   k_batch_ghost           -- ghost shells of all boxes, A(t) of each box from
//                              a device table indexed by the device step counter;
//   k_batch_stream_collide  -- a persistent kernel (grid sized to the resident
//                              CTA slots) whose CTAs walk a work list of
//                              (box, x-y tile, z chunk) items, the largest
//                              first, each with the tile march of the
//                              single-box generic kernel; the last item of a
//                              box reduces that box's droplet centre of mass
//                              (next step's frame origin), and the last CTA
//                              advances the device step counter.
//
// Because the step counter and the gradient table live on the device, a
// captured CUDA graph of two steps (both ping-pong parities) replays any
// number of steps.  The work-list shape (z chunk and CTAs per SM) is chosen
// by lbm_batch_autotune from timed trial steps.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_eigen.cuh"
#include "lbm_internal.h"
#include "lbm_lattice.cuh"
#include "lbm_tile.cuh"

using namespace lbmgb;

namespace lbmgb_batch {

struct BatchBox {
    Layout L;
    float* f[2];  // ping-pong population buffers (padded row-interleaved layout)
};

struct BatchItem {
    int box, x0, y0, zc0, zc1, tx, ty;
};

constexpr int kBatchThreads = 256;

// ---- kernels ----------------------------------------------------------------

__global__ void __launch_bounds__(256)
    k_batch_ghost(const BatchBox* __restrict__ boxes, int parity, GhostParams<float> g, const float* __restrict__ A_table,
                  long long table_steps, int nbox, const float* __restrict__ box_frame,
                  const long long* __restrict__ d_step, int* __restrict__ d_err) {
    const int box = blockIdx.z / 6, face = blockIdx.z % 6;
    const BatchBox b = boxes[box];
    // x faces: two threads per node, each writing half of every padding sector
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int half = face < 2 ? (a & 1) : -1;
    int x, y, z;
    if (!shell_node(b.L, face, face < 2 ? a >> 1 : a, blockIdx.y * blockDim.y + threadIdx.y, x, y, z)) return;
    long long step = *d_step;
    if (step >= table_steps) step = table_steps - 1;
    if (table_steps > 0) {
        const float* a = A_table + (step * nbox + box) * 9;
#pragma unroll
        for (int j = 0; j < 9; ++j) g.A[j] = a[j];
    } else {
#pragma unroll
        for (int j = 0; j < 9; ++j) g.A[j] = 0.f;
    }
    float xc = 0.f, yc = 0.f, zc = 0.f;
    if (g.frame) {
        xc = box_frame[4 * box + 0];
        yc = box_frame[4 * box + 1];
        zc = box_frame[4 * box + 2];
    }
    ghost_node<float, float>(b.f[parity], b.L, g, xc, yc, zc, x, y, z, half, d_err);
}

__global__ void __launch_bounds__(kBatchThreads)
    k_batch_stream_collide(const BatchBox* __restrict__ boxes, const BatchItem* __restrict__ items, int nitems,
                           const int* __restrict__ box_first, const int* __restrict__ box_nitems, int parity,
                           ModelC<float> m, float* __restrict__ item_parts, double* __restrict__ box_sums,
                           float* __restrict__ box_frame, unsigned* __restrict__ box_done, unsigned* __restrict__ ctas_done,
                           long long* __restrict__ d_step, int* __restrict__ d_err) {
    extern __shared__ __align__(16) float ring[];
    // (float32 reductions: this GPU's FP64 pipe runs at 1/64 of the float32 rate)
    __shared__ float red[4 * (kBatchThreads / 32)];
    __shared__ unsigned last_item, last_cta;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchBox b = boxes[w.box];
        float cm[4] = {0.f, 0.f, 0.f, 0.f};
        tile_march<float, float, false>(b.f[parity], b.f[1 - parity], b.L, m, w.tx, w.ty, w.x0, w.y0, w.zc0, w.zc1,
                                        ring, d_err, cm);
        // per-item partial sums of the droplet moments (fixed order)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float a = cm[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[4 * warp + q] = a;
        }
        __syncthreads();  // also: the ring is free for the next item
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float a = lane < kBatchThreads / 32 ? red[4 * lane + q] : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
                if (lane == 0) item_parts[4LL * it + q] = a;
            }
            if (lane == 0) {
                __threadfence();
                last_item = atomicAdd(box_done + w.box, 1u) == (unsigned)box_nitems[w.box] - 1u ? 1u : 0u;
            }
        }
        __syncthreads();
        if (last_item && warp == 0) {
            // the box's frame origin: its items' partials summed in item order
            __threadfence();
            const int first = box_first[w.box], n = box_nitems[w.box];
            float s4[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = lane; k < n; k += 32)
#pragma unroll
                for (int q = 0; q < 4; ++q) s4[q] += __ldcg(item_parts + 4LL * (first + k) + q);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s4[q] += __shfl_down_sync(0xffffffffu, s4[q], o);
            if (lane == 0) {
                double* bs = box_sums + 8LL * w.box;
#pragma unroll
                for (int q = 0; q < 4; ++q) bs[q] = (double)s4[q];
                const bool have = s4[0] > 0.f;
                for (int q = 0; q < 3; ++q) {
                    const float xc = have ? s4[1 + q] / s4[0] : 0.f;
                    bs[4 + q] = (double)xc;
                    box_frame[4LL * w.box + q] = xc;
                }
                box_done[w.box] = 0u;
            }
        }
        __syncthreads();
    }
    // the last CTA to finish advances the step counter
    if (t == 0) {
        __threadfence();
        last_cta = atomicAdd(ctas_done, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (last_cta && t == 0) {
        *d_step += 1;
        *ctas_done = 0u;
    }
}

// Ten moments of w = max(phi, 0) per box: blockIdx.y = box, partials
// [box][block][10].
__global__ void __launch_bounds__(256) k_batch_moments(const BatchBox* __restrict__ boxes, int parity,
                                                       double* __restrict__ partials) {
    const BatchBox b = boxes[blockIdx.y];
    const Layout& L = b.L;
    const float* f = b.f[parity];
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    const long long N = (long long)L.Lx * L.Ly * L.Lz;
    const double cx = 0.5 * (L.Lx - 1), cy = 0.5 * (L.Ly - 1), cz = 0.5 * (L.Lz - 1);
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.Lx), y = (int)((n / L.Lx) % L.Ly), z = (int)(n / ((long long)L.Lx * L.Ly));
        const long long base = L.at(0, 0, x, y, z);
        float ra = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            ra += f[base + (long long)i * L.pitch];
            rb += f[base + (long long)(19 + i) * L.pitch];
        }
        const float phi = (ra - rb) / (ra + rb);
        const double w = phi > 0.f ? (double)phi : 0.0;
        const double px = x - cx, py = y - cy, pz = z - cz;
        m[0] += w;
        m[1] += w * px; m[2] += w * py; m[3] += w * pz;
        m[4] += w * px * px; m[5] += w * px * py; m[6] += w * px * pz;
        m[7] += w * py * py; m[8] += w * py * pz; m[9] += w * pz * pz;
    }
    __shared__ double part[8][10];
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
            double a = lane < 8 ? part[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) partials[(10LL * gridDim.x) * blockIdx.y + 10LL * blockIdx.x + k] = a;
        }
    }
}

// Per box (blockIdx.x): moments, D, axes, eigenvalues, centre -> result[box][26];
// optionally also the frame origin into box_sums.
__global__ void k_batch_moments_final(const double* __restrict__ partials, int nblocks, double* __restrict__ result,
                                      double* __restrict__ box_sums, float* __restrict__ box_frame) {
    const int lane = threadIdx.x;
    const double* p = partials + 10LL * nblocks * blockIdx.x;
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        double a = 0.0;
        for (int b = lane; b < nblocks; b += 32) a += p[10LL * b + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        m[k] = a;
    }
    if (lane != 0) return;
    double* r = result + 26LL * blockIdx.x;
    deformation_from_moments(m, r);
    if (box_sums) {
        double* bs = box_sums + 8LL * blockIdx.x;
        for (int q = 0; q < 4; ++q) bs[q] = m[q];
        const bool have = m[0] > 0.0;
        for (int q = 0; q < 3; ++q) {
            bs[4 + q] = have ? m[1 + q] / m[0] : 0.0;
            box_frame[4LL * blockIdx.x + q] = (float)bs[4 + q];
        }
    }
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (e == cudaErrorMemoryAllocation) return LBM_ENOMEM;
    return LBM_ECUDA;
}

#define BATCH_TRY(expr)                                \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

}  // namespace lbmgb_batch

using namespace lbmgb_batch;

// ---- host side ----------------------------------------------------------------

struct lbm_batch {
    int nbox;
    std::vector<BatchBox> boxes;  // host copies (device pointers inside)
    std::vector<double> R;
    double xi, rho_hi, rho_lo;
    Model model;
    int device, num_sms;
    cudaStream_t stream;
    bool own_stream;
    int parity;
    bool initialised;
    int64_t step;
    // device tables
    BatchBox* d_boxes;
    BatchItem* d_items;
    int* d_box_first;
    int* d_box_nitems;
    double* d_item_parts;
    double* d_box_sums;   // [nbox][8]
    float* d_box_frame;   // [nbox][4]: the frame origin in float32 (read by the ghost kernel)
    unsigned* d_box_done; // [nbox]
    unsigned* d_ctas_done;
    long long* d_step;
    int* d_err;
    int* h_err;
    int latched;
    float* d_A;
    long long A_steps;
    // work list
    std::vector<BatchItem> items;
    int zchunk, ctas_per_sm, grid;
    size_t smem;
    int item_cap;
    bool prepared;  // the launch tables match zchunk / ctas_per_sm
    // row-kernel mode (every box fits the padded row geometry): row-group
    // table, per-box descriptors and centre partials of the batched row launch
    bool rows;
    int4* d_groups;
    RowsBatchBox* d_rbox;
    float* d_rparts;
    int rgroups, rmax_chunks;
    // moments
    double* d_mparts;
    double* d_result;
    double* h_result;
    int mblocks;
    // graphs of two steps, one per starting parity
    cudaGraphExec_t graph[2];
};

namespace lbmgb_batch {

// Work list for the current z chunk: the items of every box, largest boxes
// first, each box's items contiguous (its reduction sums a contiguous range of
// per-item partials).  CTA k walks items k, k + grid, k + 2 grid, ...
void build_items(lbm_batch* b, std::vector<int>& first, std::vector<int>& count) {
    b->items.clear();
    std::vector<std::pair<long long, int>> order;
    for (int k = 0; k < b->nbox; ++k)
        order.push_back({(long long)b->boxes[k].L.Lx * b->boxes[k].L.Ly * b->boxes[k].L.Lz, k});
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<long long, int>& a, const std::pair<long long, int>& c) { return a.first > c.first; });
    first.assign(b->nbox, 0);
    count.assign(b->nbox, 0);
    size_t smem = 0;
    for (auto& o : order) {
        const int k = o.second;
        const Layout& L = b->boxes[k].L;
        const int tx = std::min(L.Lx, kBatchThreads);
        const int ty = std::max(1, std::min(kBatchThreads / tx, L.Ly));
        const int zc = std::max(1, std::min(b->zchunk, L.Lz));
        first[k] = (int)b->items.size();
        for (int z0 = 0; z0 < L.Lz; z0 += zc)
            for (int y0 = 0; y0 < L.Ly; y0 += ty)
                for (int x0 = 0; x0 < L.Lx; x0 += tx)
                    b->items.push_back(BatchItem{k, x0, y0, z0, std::min(z0 + zc, L.Lz), tx, ty});
        count[k] = (int)b->items.size() - first[k];
        smem = std::max(smem, (size_t)4 * 2 * (tx + 2) * (ty + 2) * sizeof(float));
    }
    b->smem = smem;
}

}  // namespace lbmgb_batch

extern "C" {

int lbm_batch_create(lbm_batch** out, int32_t nbox, const int32_t* boxes, const double* R, const double visc[2],
                     double G, const lbm_opts* opts) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (nbox < 1 || nbox > (1 << 20) || !boxes || !R || !visc) return LBM_EINVAL;
    lbm_opts o;
    lbm_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != LBM_FP32 || o.bc != LBM_BC_GHOST_LINEAR) return LBM_EINVAL;
    if (o.frame != LBM_FRAME_DROPLET && o.frame != LBM_FRAME_BOX) return LBM_EINVAL;
    if (!(visc[0] > 0.0) || !(visc[1] > 0.0) || !std::isfinite(visc[0]) || !std::isfinite(visc[1])) return LBM_EINVAL;
    if (!(G >= 0.0) || !std::isfinite(G)) return LBM_EINVAL;
    for (int k = 0; k < nbox; ++k) {
        for (int a = 0; a < 3; ++a)
            if (boxes[3 * k + a] < 4 || boxes[3 * k + a] > 1024) return LBM_EINVAL;
        const int mn = std::min(boxes[3 * k], std::min(boxes[3 * k + 1], boxes[3 * k + 2]));
        if (!(R[k] >= 0.0) || !std::isfinite(R[k]) || 2.0 * R[k] > mn - 2) return LBM_EINVAL;
    }
    const double hi = o.rho_hi > 0.0 ? o.rho_hi : 1.0;
    double lo = o.rho_lo;
    if (!(lo > 0.0)) return LBM_EINVAL;  // the ensemble takes the minority density explicitly
    if (!(lo <= hi)) return LBM_EINVAL;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete b; return LBM_ECUDA; }
    if (cudaSetDevice(dev) != cudaSuccess) { delete b; return LBM_ECUDA; }
    b->device = dev;
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    b->nbox = nbox;
    b->R.assign(R, R + nbox);
    b->xi = o.xi > 0.0 ? o.xi : 1.0;
    b->rho_hi = hi;
    b->rho_lo = lo;
    const double mach = o.mach_limit > 0.0 ? o.mach_limit : 0.9;
    b->model.tau[0] = 3.0 * visc[0] + 0.5;
    b->model.tau[1] = 3.0 * visc[1] + 0.5;
    b->model.G = G;
    b->model.rho_b[0] = lo;
    b->model.rho_b[1] = hi;
    b->model.periodic = 0;
    b->model.mach2 = mach * mach / 3.0;
    b->model.droplet_frame = o.frame == LBM_FRAME_DROPLET;
    b->stream = (cudaStream_t)o.cuda_stream;
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return LBM_ECUDA; }
        b->own_stream = true;
    }
    b->ctas_per_sm = 0;  // 0: as many as fit
    // the row kernel when every box fits its padded rows (and the tile shape
    // is left to the library), else the generic tile march
    b->rows = o.tile_y <= 0;
    long long rows_total = 0;
    for (int k = 0; k < nbox; ++k) {
        b->rows = b->rows && rows_batch_applies(boxes[3 * k], boxes[3 * k + 1], boxes[3 * k + 2]);
        rows_total += boxes[3 * k + 1];
    }
    b->rows = b->rows && rows_total <= 65535;
    b->zchunk = o.z_chunk > 0 ? o.z_chunk : (b->rows ? 32 : 16);
    b->boxes.resize(nbox);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < nbox && e == cudaSuccess; ++k) {
        b->boxes[k].L = b->rows ? make_layout_rows(boxes[3 * k], boxes[3 * k + 1], boxes[3 * k + 2])
                                : make_layout(boxes[3 * k], boxes[3 * k + 1], boxes[3 * k + 2], kFP32);
        const size_t bytes = (size_t)b->boxes[k].L.total * sizeof(float);
        for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
            e = cudaMalloc(&b->boxes[k].f[q], bytes);
            if (e == cudaSuccess) e = cudaMemsetAsync(b->boxes[k].f[q], 0, bytes, b->stream);
        }
    }
    b->mblocks = 64;
    if (e == cudaSuccess) e = cudaMalloc(&b->d_boxes, sizeof(BatchBox) * nbox);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_boxes, b->boxes.data(), sizeof(BatchBox) * nbox, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_box_sums, sizeof(double) * 8 * nbox);
    if (e == cudaSuccess) e = cudaMemset(b->d_box_sums, 0, sizeof(double) * 8 * nbox);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_box_frame, sizeof(float) * 4 * nbox);
    if (e == cudaSuccess) e = cudaMemset(b->d_box_frame, 0, sizeof(float) * 4 * nbox);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_box_done, sizeof(unsigned) * nbox);
    if (e == cudaSuccess) e = cudaMemset(b->d_box_done, 0, sizeof(unsigned) * nbox);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_box_first, sizeof(int) * nbox);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_box_nitems, sizeof(int) * nbox);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctas_done, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_ctas_done, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_step, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_step, 0, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_mparts, sizeof(double) * 10 * b->mblocks * nbox);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_result, sizeof(double) * 26 * nbox);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_result, sizeof(double) * 26 * nbox);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        const int st = cuda_status(e);
        lbm_batch_destroy(b);
        return st;
    }
    *b->h_err = 0;
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& bx : b->boxes) {
        cudaFree(bx.f[0]);
        cudaFree(bx.f[1]);
    }
    for (int q = 0; q < 2; ++q)
        if (b->graph[q]) cudaGraphExecDestroy(b->graph[q]);
    cudaFree(b->d_boxes);
    cudaFree(b->d_items);
    cudaFree(b->d_box_first);
    cudaFree(b->d_box_nitems);
    cudaFree(b->d_item_parts);
    cudaFree(b->d_box_sums);
    cudaFree(b->d_box_frame);
    cudaFree(b->d_groups);
    cudaFree(b->d_rbox);
    cudaFree(b->d_rparts);
    cudaFree(b->d_box_done);
    cudaFree(b->d_ctas_done);
    cudaFree(b->d_step);
    cudaFree(b->d_err);
    cudaFree(b->d_A);
    cudaFree(b->d_mparts);
    cudaFree(b->d_result);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->h_result) cudaFreeHost(b->h_result);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

namespace lbmgb_batch {

void drop_graphs(lbm_batch* b) {
    for (int q = 0; q < 2; ++q)
        if (b->graph[q]) {
            cudaGraphExecDestroy(b->graph[q]);
            b->graph[q] = nullptr;
        }
}

// (Re)build the work list for the current z chunk and CTAs per SM, upload it.
int prepare_rows(lbm_batch* b);

int prepare_items(lbm_batch* b) {
    BATCH_TRY(cudaStreamSynchronize(b->stream));
    if (b->rows) return prepare_rows(b);
    std::vector<int> first, count;
    build_items(b, first, count);
    const int n = (int)b->items.size();
    cudaFree(b->d_items);
    cudaFree(b->d_item_parts);
    b->d_items = nullptr;
    b->d_item_parts = nullptr;
    BATCH_TRY(cudaMalloc(&b->d_items, sizeof(BatchItem) * n));
    BATCH_TRY(cudaMalloc(&b->d_item_parts, sizeof(double) * 4 * n));
    BATCH_TRY(cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice));
    BATCH_TRY(cudaMemcpy(b->d_box_first, first.data(), sizeof(int) * b->nbox, cudaMemcpyHostToDevice));
    BATCH_TRY(cudaMemcpy(b->d_box_nitems, count.data(), sizeof(int) * b->nbox, cudaMemcpyHostToDevice));
    // persistent grid: the resident CTA slots (or the requested CTAs per SM),
    // at most one CTA per item
    auto k = k_batch_stream_collide;
    BATCH_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    int per_sm = 0;
    BATCH_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBatchThreads, b->smem));
    if (per_sm < 1) return LBM_ECUDA;
    if (b->ctas_per_sm > 0) per_sm = std::min(per_sm, b->ctas_per_sm);
    b->grid = std::max(1, std::min(n, per_sm * b->num_sms));
    drop_graphs(b);
    b->prepared = true;
    return LBM_OK;
}

// Row-kernel mode: the row groups of every box (largest boxes first, each
// box's groups contiguous), the boxes' descriptors and their centre-partial
// slots for the current z chunk.
int prepare_rows(lbm_batch* b) {
    const int zc = std::max(1, b->zchunk);
    std::vector<int> order(b->nbox);
    for (int k = 0; k < b->nbox; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const Layout &La = b->boxes[a].L, &Lc = b->boxes[c].L;
        return (long long)La.Lx * La.Ly * La.Lz > (long long)Lc.Lx * Lc.Ly * Lc.Lz;
    });
    std::vector<int4> groups;
    std::vector<RowsBatchBox> rbox(b->nbox);
    int part = 0, max_chunks = 1;
    for (int k : order) {
        const Layout& L = b->boxes[k].L;
        const int chunks = (L.Lz + zc - 1) / zc;
        max_chunks = std::max(max_chunks, chunks);
        rbox[k].f[0] = b->boxes[k].f[0];
        rbox[k].f[1] = b->boxes[k].f[1];
        rbox[k].L = L;
        rbox[k].ctas = L.Ly * chunks;
        rbox[k].part0 = part;
        part += rbox[k].ctas;
        for (int y0 = 0; y0 < L.Ly; y0 += kRowClusterRows) groups.push_back(make_int4(k, y0, chunks, 0));
    }
    cudaFree(b->d_groups);
    cudaFree(b->d_rbox);
    cudaFree(b->d_rparts);
    b->d_groups = nullptr;
    b->d_rbox = nullptr;
    b->d_rparts = nullptr;
    BATCH_TRY(cudaMalloc(&b->d_groups, sizeof(int4) * groups.size()));
    BATCH_TRY(cudaMalloc(&b->d_rbox, sizeof(RowsBatchBox) * b->nbox));
    BATCH_TRY(cudaMalloc(&b->d_rparts, sizeof(float) * 4 * (size_t)part));
    BATCH_TRY(cudaMemcpy(b->d_groups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice));
    BATCH_TRY(cudaMemcpy(b->d_rbox, rbox.data(), sizeof(RowsBatchBox) * b->nbox, cudaMemcpyHostToDevice));
    b->rgroups = (int)groups.size();
    b->rmax_chunks = max_chunks;
    b->grid = b->rgroups * kRowClusterRows * max_chunks;
    b->smem = rows_batch_smem();
    drop_graphs(b);
    b->prepared = true;
    return LBM_OK;
}

int batch_init(lbm_batch* b) {
    if (b->initialised) return LBM_OK;
    if (!b->prepared) {
        const int st = prepare_items(b);
        if (st) return st;
    }
    // initial state of every box: tanh droplet in u = A_box(0) x
    std::vector<float> A0(9 * (size_t)b->nbox, 0.f);
    if (b->A_steps > 0) BATCH_TRY(cudaMemcpy(A0.data(), b->d_A, sizeof(float) * 9 * b->nbox, cudaMemcpyDeviceToHost));
    for (int k = 0; k < b->nbox; ++k) {
        Grad g;
        for (int j = 0; j < 9; ++j) g.a[j] = (double)A0[9 * k + j];
        BATCH_TRY(launch_init(1, b->boxes[k].f[b->parity], b->boxes[k].L, b->R[k], b->xi, b->rho_hi, b->rho_lo, g,
                              b->stream));
    }
    // first frame origins from the initial populations
    k_batch_moments<<<dim3(b->mblocks, b->nbox), 256, 0, b->stream>>>(b->d_boxes, b->parity, b->d_mparts);
    k_batch_moments_final<<<b->nbox, 32, 0, b->stream>>>(b->d_mparts, b->mblocks, b->d_result, b->d_box_sums,
                                                         b->d_box_frame);
    BATCH_TRY(cudaGetLastError());
    b->initialised = true;
    return LBM_OK;
}

cudaError_t enqueue_step(lbm_batch* b, int parity) {
    int fast = 0, slow = 0;
    for (const auto& bx : b->boxes) {
        fast = std::max(fast, std::max(bx.L.Lx, 2 * (bx.L.Ly + 2)));  // x faces: two threads per node
        slow = std::max(slow, std::max(bx.L.Lz + 2, bx.L.Ly));
    }
    const dim3 gblock(32, 8, 1);
    const dim3 ggrid((fast + 31) / 32, (slow + 7) / 8, 6 * b->nbox);
    const double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // A comes from the table
    k_batch_ghost<<<ggrid, gblock, 0, b->stream>>>(b->d_boxes, parity, ghost_params<float>(b->model, zero), b->d_A,
                                                   b->A_steps, b->nbox, b->d_box_frame, b->d_step, b->d_err);
    if (b->rows) {
        RowsBatch rb;
        rb.group = b->d_groups;
        rb.box = b->d_rbox;
        rb.parts = b->d_rparts;
        rb.box_done = b->d_box_done;
        rb.box_sums = b->d_box_sums;
        rb.box_frame = b->d_box_frame;
        rb.ctas_done = b->d_ctas_done;
        rb.d_step = b->d_step;
        rb.parity = parity;
        return launch_rows_batch(rb, b->rgroups, b->rmax_chunks, b->zchunk, b->model, b->d_err, b->stream);
    }
    ModelC<float> mc;
    for (int s = 0; s < 2; ++s) {
        mc.tau[s] = (float)b->model.tau[s];
        mc.inv_tau[s] = (float)(1.0 / b->model.tau[s]);
        mc.rho_b[s] = (float)b->model.rho_b[s];
    }
    mc.G = (float)b->model.G;
    k_batch_stream_collide<<<b->grid, kBatchThreads, b->smem, b->stream>>>(
        b->d_boxes, b->d_items, (int)b->items.size(), b->d_box_first, b->d_box_nitems, parity, mc,
        reinterpret_cast<float*>(b->d_item_parts), b->d_box_sums, b->d_box_frame, b->d_box_done, b->d_ctas_done,
        b->d_step, b->d_err);
    return cudaGetLastError();
}

int batch_sync(lbm_batch* b) {
    BATCH_TRY(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BATCH_TRY(cudaStreamSynchronize(b->stream));
    if (!b->latched) {
        const int bits = *b->h_err;
        if (bits & 4) b->latched = LBM_ETIMEOUT;
        else if (bits & 2) b->latched = LBM_EMACH;
        else if (bits & 1) b->latched = LBM_ENONFINITE;
    }
    return b->latched;
}

}  // namespace lbmgb_batch

extern "C" {

int lbm_batch_set_gradients(lbm_batch* b, int64_t nsteps, const double* A) {
    if (!b || nsteps < 0 || (nsteps > 0 && !A)) return LBM_EINVAL;
    const size_t n = (size_t)nsteps * b->nbox * 9;
    for (size_t k = 0; k < (size_t)nsteps * b->nbox; ++k) {
        const double* a = A + 9 * k;
        double mx = 1.0;
        for (int j = 0; j < 9; ++j) {
            if (!std::isfinite(a[j])) return LBM_EINVAL;
            mx = std::max(mx, std::fabs(a[j]));
        }
        if (std::fabs(a[0] + a[4] + a[8]) > 1e-12 * mx) return LBM_EINVAL;
    }
    cudaSetDevice(b->device);
    BATCH_TRY(cudaStreamSynchronize(b->stream));
    std::vector<float> Af(n);
    for (size_t k = 0; k < n; ++k) Af[k] = (float)A[k];
    cudaFree(b->d_A);
    b->d_A = nullptr;
    b->A_steps = 0;
    if (n) {
        BATCH_TRY(cudaMalloc(&b->d_A, sizeof(float) * n));
        BATCH_TRY(cudaMemcpy(b->d_A, Af.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    b->A_steps = nsteps;
    drop_graphs(b);
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t n) {
    if (!b || n < 0) return LBM_EINVAL;
    if (b->latched) return b->latched;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ECUDA;
    int st = batch_init(b);
    if (st) return st;
    int64_t k = 0;
    // pairs of steps from a captured graph (both parities), then a single step
    while (n - k >= 2) {
        const int p = b->parity;
        if (!b->graph[p]) {
            cudaGraph_t g = nullptr;
            BATCH_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = enqueue_step(b, p);
            cudaError_t e2 = enqueue_step(b, 1 - p);
            cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return LBM_ECUDA;
            }
            cudaError_t e4 = cudaGraphInstantiate(&b->graph[p], g, 0);
            cudaGraphDestroy(g);
            if (e4 != cudaSuccess) return LBM_ECUDA;
        }
        BATCH_TRY(cudaGraphLaunch(b->graph[p], b->stream));
        k += 2;
        b->step += 2;
    }
    if (k < n) {
        BATCH_TRY(enqueue_step(b, b->parity));
        b->parity = 1 - b->parity;
        b->step += 1;
    }
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_EINVAL;
    cudaSetDevice(b->device);
    return batch_sync(b);
}

int lbm_batch_deformation(lbm_batch* b, double* D, double* axes, double* centre) {
    if (!b || !D) return LBM_EINVAL;
    cudaSetDevice(b->device);
    int st = batch_init(b);
    if (st) return st;
    k_batch_moments<<<dim3(b->mblocks, b->nbox), 256, 0, b->stream>>>(b->d_boxes, b->parity, b->d_mparts);
    k_batch_moments_final<<<b->nbox, 32, 0, b->stream>>>(b->d_mparts, b->mblocks, b->d_result, nullptr, nullptr);
    BATCH_TRY(cudaGetLastError());
    BATCH_TRY(cudaMemcpyAsync(b->h_result, b->d_result, sizeof(double) * 26 * b->nbox, cudaMemcpyDeviceToHost,
                              b->stream));
    if ((st = batch_sync(b))) return st;
    for (int k = 0; k < b->nbox; ++k) {
        const double* r = b->h_result + 26 * k;
        D[k] = r[10];
        if (axes) memcpy(axes + 9 * k, r + 11, sizeof(double) * 9);
        if (centre) memcpy(centre + 3 * k, r + 23, sizeof(double) * 3);
    }
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch* b, double* m) {
    if (!b || !m) return LBM_EINVAL;
    cudaSetDevice(b->device);
    int st = batch_init(b);
    if (st) return st;
    k_batch_moments<<<dim3(b->mblocks, b->nbox), 256, 0, b->stream>>>(b->d_boxes, b->parity, b->d_mparts);
    k_batch_moments_final<<<b->nbox, 32, 0, b->stream>>>(b->d_mparts, b->mblocks, b->d_result, nullptr, nullptr);
    BATCH_TRY(cudaGetLastError());
    BATCH_TRY(cudaMemcpyAsync(b->h_result, b->d_result, sizeof(double) * 26 * b->nbox, cudaMemcpyDeviceToHost,
                              b->stream));
    if ((st = batch_sync(b))) return st;
    for (int k = 0; k < b->nbox; ++k) memcpy(m + 10 * k, b->h_result + 26 * k, sizeof(double) * 10);
    return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch* b, int32_t box, double* f) {
    if (!b || !f || box < 0 || box >= b->nbox) return LBM_EINVAL;
    cudaSetDevice(b->device);
    int st = batch_init(b);
    if (st) return st;
    const Layout& L = b->boxes[box].L;
    const size_t E = 38ull * L.Lx * L.Ly * L.Lz;
    double* d = nullptr;
    BATCH_TRY(cudaMallocAsync(&d, sizeof(double) * E, b->stream));
    cudaError_t e = launch_pack(kFP32, b->boxes[box].f[b->parity], L, b->model, d, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, sizeof(double) * E, cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(d, b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return batch_sync(b);
}

int lbm_batch_set_populations(lbm_batch* b, int32_t box, const double* f) {
    if (!b || !f || box < 0 || box >= b->nbox) return LBM_EINVAL;
    cudaSetDevice(b->device);
    int st = batch_init(b);
    if (st) return st;
    const Layout& L = b->boxes[box].L;
    const size_t E = 38ull * L.Lx * L.Ly * L.Lz;
    for (size_t k = 0; k < E; ++k)
        if (!std::isfinite(f[k])) return LBM_EINVAL;
    double* d = nullptr;
    BATCH_TRY(cudaMallocAsync(&d, sizeof(double) * E, b->stream));
    cudaError_t e = cudaMemcpyAsync(d, f, sizeof(double) * E, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_unpack(kFP32, b->boxes[box].f[b->parity], L, b->model, d, nullptr, b->stream);
    cudaFreeAsync(d, b->stream);
    // refresh every box's frame origin from the stored populations
    if (e == cudaSuccess) {
        k_batch_moments<<<dim3(b->mblocks, b->nbox), 256, 0, b->stream>>>(b->d_boxes, b->parity, b->d_mparts);
        k_batch_moments_final<<<b->nbox, 32, 0, b->stream>>>(b->d_mparts, b->mblocks, b->d_result, b->d_box_sums,
                                                         b->d_box_frame);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return cuda_status(e);
}

int lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, int32_t* zchunk, int32_t* ctas_per_sm) {
    if (!b || trial_steps < 1 || b->step != 0) return LBM_EINVAL;
    cudaSetDevice(b->device);
    // row-kernel mode: z chunks only (one CTA per row and chunk)
    const std::vector<int> zcs = b->rows ? std::vector<int>{16, 22, 32, 43, 64} : std::vector<int>{8, 16, 32, 64};
    const std::vector<int> per = b->rows ? std::vector<int>{0} : std::vector<int>{0, 2, 4};
    float best = 1e30f;
    int bz = b->zchunk, bp = b->ctas_per_sm;
    cudaEvent_t e0, e1;
    BATCH_TRY(cudaEventCreate(&e0));
    BATCH_TRY(cudaEventCreate(&e1));
    for (int zc : zcs)
        for (int pp : per) {
            b->zchunk = zc;
            b->ctas_per_sm = pp;
            int st = prepare_items(b);
            if (st) return st;
            b->initialised = false;
            if ((st = batch_init(b))) return st;
            BATCH_TRY(cudaEventRecord(e0, b->stream));
            for (int k = 0; k < trial_steps; ++k) {
                BATCH_TRY(enqueue_step(b, b->parity));
                b->parity = 1 - b->parity;
            }
            BATCH_TRY(cudaEventRecord(e1, b->stream));
            BATCH_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            BATCH_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bz = zc;
                bp = pp;
            }
            // rewind the step counter for the next trial
            BATCH_TRY(cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream));
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->zchunk = bz;
    b->ctas_per_sm = bp;
    int st = prepare_items(b);
    if (st) return st;
    // start again from the initial state
    b->initialised = false;
    b->parity = 0;
    BATCH_TRY(cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream));
    BATCH_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
    if ((st = batch_init(b))) return st;
    if ((st = batch_sync(b))) return st;
    if (zchunk) *zchunk = bz;
    if (ctas_per_sm) *ctas_per_sm = bp;
    return LBM_OK;
}

int lbm_batch_launch_kind(lbm_batch* b, int32_t* kind) {
    if (!b || !kind) return LBM_EINVAL;
    *kind = b->rows ? 1 : 0;
    return LBM_OK;
}

int lbm_batch_shape(lbm_batch* b, int32_t* zchunk, int32_t* ctas, int32_t* items) {
    if (!b) return LBM_EINVAL;
    if (!b->prepared) {
        cudaSetDevice(b->device);
        const int st = prepare_items(b);
        if (st) return st;
    }
    if (zchunk) *zchunk = b->zchunk;
    if (ctas) *ctas = b->grid;
    // work items: the generic march's (box, tile, z chunk) items, or the row
    // kernel's row groups
    if (items) *items = b->rows ? (int32_t)b->rgroups : (int32_t)b->items.size();
    return LBM_OK;
}

}  // extern "C"
