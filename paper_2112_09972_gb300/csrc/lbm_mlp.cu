// Learned surrogate of the droplet's conformation tensor (an addition of this
// library beside the paper's method): a multilayer perceptron that maps a
// window of the velocity gradient A(t) to the six entries of the droplet's
// conformation tensor M = I / det(I)^(1/3) (I the second-moment tensor of
// Sec. 2, Eq. 4; M = identity for a sphere, the Maffettone-Minale tensor of
// Eqs. 1, 2).  Forward pass, backward pass and Adam run on the GPU:
//
//   k_gemm_nt   -- C = A B^T on bfloat16 tensor cores (mma.sync m16n8k16,
//                  float32 accumulation), A [M, K] and B [N, K] with K
//                  contiguous, fused epilogues (bias + ReLU to bfloat16,
//                  ReLU-derivative mask to bfloat16, float32 output)
//   k_transpose -- bfloat16 tile transpose (operands of the weight gradients)
//   k_prep, k_loss_grad, k_colsum, k_adam, k_weights, k_output,
//   k_deform_from_m -- input normalisation, mean-square loss and its
//                  gradient, bias gradients, Adam, bfloat16 weight copies,
//                  output scaling, and D of a predicted M (Eq. 4).
//
// Layers: z_l = h_{l-1} W_l^T + b_l, h_l = max(z_l, 0), last layer linear;
// inputs normalised as (x - x_mean) x_scale, outputs y = y_hat / y_scale +
// y_mean, loss = mean over samples and outputs of (y_hat - t_hat)^2.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <new>
#include <random>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_eigen.cuh"

namespace lbmgb_mlp {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 64, BK = 32;  // CTA tile of the GEMM
constexpr int kGemmThreads = 128;         // 4 warps, each a 32 x 32 sub-tile
constexpr int SROW = BK + 8;              // shared row (bfloat16) padded against bank conflicts

enum Epilogue { kStoreF32 = 0, kBiasF32 = 1, kBiasReluBf16 = 2, kMaskBf16 = 3 };

struct GemmArgs {
    const bf16* A;  // [M, K], row stride lda
    const bf16* B;  // [N, K], row stride ldb
    int lda, ldb, M, N, K;
    int epi;
    const float* bias;  // [N] (kBiasF32, kBiasReluBf16)
    const bf16* mask;   // [M, N], row stride ldm (kMaskBf16: keep where mask > 0)
    int ldm;
    float* Cf;  // float32 output, row stride ldc
    bf16* Cb;   // bfloat16 output, row stride ldc
    int ldc;
};

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// d += a b for one 16 x 8 x 16 tile (a row-major 16 x 16, b column-major 16 x 8).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C = A B^T for a BM x BN tile per CTA.  K is a multiple of BK; the strides
// and base addresses are multiples of 8 elements (16 bytes).  Rows of A or B
// beyond M or N read as zero and are not stored.
__global__ void __launch_bounds__(kGemmThreads) k_gemm_nt(GemmArgs g) {
    __shared__ __align__(16) bf16 sA[2][BM][SROW];
    __shared__ __align__(16) bf16 sB[2][BN][SROW];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

    // Each operand tile is 64 rows of 64 bytes: 256 chunks of 16 bytes, two per thread.
    uint4 ra[2], rb[2];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = t + q * kGemmThreads, row = c >> 2, col = (c & 3) * 8;
            const int m = m0 + row, n = n0 + row;
            ra[q] = m < g.M ? *reinterpret_cast<const uint4*>(g.A + (long long)m * g.lda + k0 + col)
                            : make_uint4(0u, 0u, 0u, 0u);
            rb[q] = n < g.N ? *reinterpret_cast<const uint4*>(g.B + (long long)n * g.ldb + k0 + col)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    auto stash = [&](int st) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = t + q * kGemmThreads, row = c >> 2, col = (c & 3) * 8;
            *reinterpret_cast<uint4*>(&sA[st][row][col]) = ra[q];
            *reinterpret_cast<uint4*>(&sB[st][row][col]) = rb[q];
        }
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    const int nk = g.K / BK;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) fetch((kt + 1) * BK);  // next tile in flight during the products
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i)  // rows 0-15 of the m16 tile, k halves by lane / 16
                ldmatrix_x4(af[i], &sA[st][wm + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int j = 0; j < 4; j += 2) {  // two n8 tiles: n by lane & 7 (+8 for lanes 16-31), k halves by bit 3
                unsigned r[4];
                ldmatrix_x4(r, &sB[st][wn + j * 8 + (lane & 7) + ((lane >> 4) << 3)][kk + ((lane >> 3) & 1) * 8]);
                bfr[j][0] = r[0];
                bfr[j][1] = r[1];
                bfr[j + 1][0] = r[2];
                bfr[j + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j][0], bfr[j][1]);
        }
        if (kt + 1 < nk) {
            stash(st ^ 1);  // the other stage: last read two iterations ago
            __syncthreads();
        }
    }

    // accumulator e of tile (i, j): row groupID (+8 for e >= 2), column 2 tig (+1 for odd e)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + i * 16 + (lane >> 2) + (e >> 1) * 8;
                const int n = n0 + wn + j * 8 + (lane & 3) * 2 + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][e];
                const long long o = (long long)m * g.ldc + n;
                switch (g.epi) {
                    case kStoreF32: g.Cf[o] = v; break;
                    case kBiasF32: g.Cf[o] = v + g.bias[n]; break;
                    case kBiasReluBf16: g.Cb[o] = __float2bfloat16_rn(fmaxf(v + g.bias[n], 0.f)); break;
                    default:
                        g.Cb[o] = __float2bfloat16_rn(__bfloat162float(g.mask[(long long)m * g.ldm + n]) > 0.f ? v : 0.f);
                }
            }
}

namespace {

// Normalised input in bfloat16: xb[r, c] = (x[r, c] - mean[c]) scale[c].
__global__ void k_prep(const float* __restrict__ x, long long n, int d0, const float* __restrict__ mean,
                       const float* __restrict__ scale, bf16* __restrict__ xb) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d0) return;
    const int c = (int)(e % d0);
    xb[e] = __float2bfloat16_rn((x[e] - mean[c]) * scale[c]);
}

// out[c, r] = in[r, c] for an R x C matrix (32 x 32 tiles through shared memory).
__global__ void k_transpose(const bf16* __restrict__ in, int R, int C, int ldi, bf16* __restrict__ out, int ldo) {
    __shared__ bf16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[k][threadIdx.x] = in[(long long)r * ldi + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(long long)c * ldo + r] = tile[threadIdx.x][k];
    }
}

// Output-layer gradient g = 2 (y_hat - t_hat) / (n dL) in bfloat16 (zero in
// the padding columns dL .. ldg-1) and per-block partial sums of the squared
// error (float64).
constexpr int kLossThreads = 256;
__global__ void __launch_bounds__(kLossThreads) k_loss_grad(const float* __restrict__ yhat, int ldy,
                                                            const float* __restrict__ tgt, int n, int dL, int ldg,
                                                            const float* __restrict__ ymean,
                                                            const float* __restrict__ yscale, bf16* __restrict__ g,
                                                            double* __restrict__ parts) {
    __shared__ double red[kLossThreads / 32];
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (e < (long long)n * ldg) {
        const int r = (int)(e / ldg), c = (int)(e % ldg);
        float gv = 0.f;
        if (c < dL) {
            const float th = (tgt[(long long)r * dL + c] - ymean[c]) * yscale[c];
            const float d = yhat[(long long)r * ldy + c] - th;
            sq = (double)d * (double)d;
            gv = 2.f * d / (float)((long long)n * dL);
        }
        g[e] = __float2bfloat16_rn(gv);
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kLossThreads / 32; ++w) s += red[w];
        parts[blockIdx.x] = s;
    }
}

// Sum of the partials in block order, divided by count: the mean loss.
__global__ void k_loss_final(const double* __restrict__ parts, int nparts, double count, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += parts[b];
    *out = s / count;
}

// Bias gradient: column sums db[c] = sum_r g[r, c] of a bfloat16 [n, C] matrix.
__global__ void k_colsum(const bf16* __restrict__ g, int n, int C, int ldg, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int r = 0; r < n; ++r) s += __bfloat162float(g[(long long)r * ldg + c]);
    db[c] = s;
}

// Adam on float32 parameters (bias-corrected moments).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
}

// bfloat16 copies of a float32 weight matrix W [R, C]: Wb = W and WTb = W^T.
__global__ void k_weights(const float* __restrict__ W, int R, int C, bf16* __restrict__ Wb,
                          bf16* __restrict__ WTb) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)R * C) return;
    const int r = (int)(e / C), c = (int)(e % C);
    const bf16 b = __float2bfloat16_rn(W[e]);
    Wb[e] = b;
    WTb[(long long)c * R + r] = b;
}

// Outputs in physical units: y[r, c] = y_hat[r, c] / scale[c] + mean[c].
__global__ void k_output(const float* __restrict__ yhat, int ldy, long long n, int dL,
                         const float* __restrict__ mean, const float* __restrict__ scale, float* __restrict__ y) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * dL) return;
    const long long r = e / dL;
    const int c = (int)(e % dL);
    y[e] = yhat[r * ldy + c] / scale[c] + mean[c];
}

// D of Sec. 2, Eq. 4 from a predicted conformation tensor M (entries xx, xy,
// xz, yy, yz, zz): D = (sqrt(l1) - sqrt(l3)) / (sqrt(l1) + sqrt(l3)) of its
// eigenvalues (D does not depend on the normalisation of M).
__global__ void k_deform_from_m(const float* __restrict__ m6, long long n, double* __restrict__ D) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float* q = m6 + 6 * r;
    double a[3][3] = {{q[0], q[1], q[2]}, {q[1], q[3], q[4]}, {q[2], q[4], q[5]}};
    double lam[3], v[3][3];
    lbmgb::jacobi3(a, lam, v);
    double hi = fmax(lam[0], fmax(lam[1], lam[2])), lo = fmin(lam[0], fmin(lam[1], lam[2]));
    hi = sqrt(fmax(hi, 0.0));
    lo = sqrt(fmax(lo, 0.0));
    D[r] = hi + lo > 0.0 ? (hi - lo) / (hi + lo) : 0.0;
}

}  // namespace
}  // namespace lbmgb_mlp

using namespace lbmgb_mlp;

struct lbm_mlp {
    int device;
    cudaStream_t stream;
    bool own_stream;
    int L;                  // layers
    std::vector<int> d;     // sizes d_0 .. d_L
    std::vector<int> dp;    // stored sizes: d_L padded to 32, the others as given
    int max_batch;
    int64_t step;           // Adam steps taken
    // float32 parameters, gradients and Adam moments: one flat array each,
    // W_l [dp_l, d_{l-1}] then b_l [dp_l] per layer (padding rows stay zero)
    std::vector<long long> offW, offb;
    long long nparam;
    float *p, *g, *m, *v;
    std::vector<bf16*> Wb, WTb;  // bfloat16 W_l [dp_l, d_{l-1}] and W_l^T [d_{l-1}, dp_l]
    float *x_mean, *x_scale, *y_mean, *y_scale;
    // activations and workspace for max_batch samples
    std::vector<bf16*> H;        // H[0] the normalised input, H[l] hidden layer l
    float* yhat;                 // [max_batch, dp_L]
    std::vector<bf16*> G;        // G[l] gradient with respect to z_l, [max_batch, dp_l]
    bf16 *T1, *T2;               // transposes for the weight gradients
    double *loss_parts, *loss;
    int loss_blocks;
    double* h_loss;              // pinned
};

namespace {

int mlp_status(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (e == cudaErrorMemoryAllocation) return LBM_ENOMEM;
    return LBM_ECUDA;
}

#define MLP_TRY(expr)                                   \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return mlp_status(e_);   \
    } while (0)

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t gemm(lbm_mlp* c, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int epi,
                 const float* bias, const bf16* mask, int ldm, float* Cf, bf16* Cb, int ldc) {
    GemmArgs a;
    a.A = A; a.B = B; a.lda = lda; a.ldb = ldb; a.M = M; a.N = N; a.K = K; a.epi = epi;
    a.bias = bias; a.mask = mask; a.ldm = ldm; a.Cf = Cf; a.Cb = Cb; a.ldc = ldc;
    const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm_nt<<<grid, kGemmThreads, 0, c->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t transpose(lbm_mlp* c, const bf16* in, int R, int C, int ldi, bf16* out, int ldo) {
    const dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, c->stream>>>(in, R, C, ldi, out, ldo);
    return cudaGetLastError();
}

cudaError_t refresh_weights(lbm_mlp* c) {
    for (int l = 1; l <= c->L; ++l) {
        const long long n = (long long)c->dp[l] * c->d[l - 1];
        k_weights<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->p + c->offW[l], c->dp[l], c->d[l - 1], c->Wb[l],
                                                           c->WTb[l]);
    }
    return cudaGetLastError();
}

// Forward pass of n <= max_batch samples (inputs x on the device, float32
// [n, d0]): activations into H, normalised outputs into yhat.
cudaError_t forward(lbm_mlp* c, const float* x, int n) {
    const int d0 = c->d[0];
    k_prep<<<blocks_for((long long)n * d0, 256), 256, 0, c->stream>>>(x, n, d0, c->x_mean, c->x_scale, c->H[0]);
    cudaError_t e = cudaGetLastError();
    for (int l = 1; l <= c->L && e == cudaSuccess; ++l) {
        const bool last = l == c->L;
        e = gemm(c, c->H[l - 1], c->d[l - 1], c->Wb[l], c->d[l - 1], n, c->dp[l], c->d[l - 1],
                 last ? kBiasF32 : kBiasReluBf16, c->p + c->offb[l], nullptr, 0, last ? c->yhat : nullptr,
                 last ? nullptr : c->H[l], c->dp[l]);
    }
    return e;
}

// Loss and parameter gradients of n samples (targets t on the device, float32 [n, dL]).
cudaError_t backward(lbm_mlp* c, const float* t, int n) {
    const int L = c->L, dL = c->d[L], dLp = c->dp[L];
    const long long ne = (long long)n * dLp;
    const int nb = (int)blocks_for(ne, kLossThreads);
    k_loss_grad<<<nb, kLossThreads, 0, c->stream>>>(c->yhat, dLp, t, n, dL, dLp, c->y_mean, c->y_scale, c->G[L],
                                                    c->loss_parts);
    k_loss_final<<<1, 32, 0, c->stream>>>(c->loss_parts, nb, (double)n * dL, c->loss);
    cudaError_t e = cudaGetLastError();
    for (int l = L; l >= 1 && e == cudaSuccess; --l) {
        const int dout = c->dp[l], din = c->d[l - 1];
        // dW_l = G_l^T H_{l-1}: operands with the batch index contiguous
        e = transpose(c, c->G[l], n, dout, dout, c->T1, n);
        if (e == cudaSuccess) e = transpose(c, c->H[l - 1], n, din, din, c->T2, n);
        if (e == cudaSuccess)
            e = gemm(c, c->T1, n, c->T2, n, dout, din, n, kStoreF32, nullptr, nullptr, 0, c->g + c->offW[l], nullptr,
                     din);
        if (e == cudaSuccess) {
            k_colsum<<<blocks_for(dout, 128), 128, 0, c->stream>>>(c->G[l], n, dout, dout, c->g + c->offb[l]);
            e = cudaGetLastError();
        }
        // G_{l-1} = (G_l W_l) masked by h_{l-1} > 0
        if (l > 1 && e == cudaSuccess)
            e = gemm(c, c->G[l], dout, c->WTb[l], dout, n, din, dout, kMaskBf16, nullptr, c->H[l - 1], din, nullptr,
                     c->G[l - 1], din);
    }
    return e;
}

}  // namespace

extern "C" {

int lbm_mlp_create(lbm_mlp** out, int32_t nlayers, const int32_t* sizes, int32_t max_batch, uint64_t seed,
                   void* cuda_stream, int32_t device) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!sizes || nlayers < 1 || nlayers > 16 || max_batch < 32 || max_batch % 32 != 0 || max_batch > (1 << 22))
        return LBM_EINVAL;
    for (int l = 0; l <= nlayers; ++l)
        if (sizes[l] < 1 || sizes[l] > 8192) return LBM_EINVAL;
    for (int l = 0; l < nlayers; ++l)
        if (sizes[l] % 32 != 0) return LBM_EINVAL;  // input and hidden widths: multiples of 32
    if (sizes[nlayers] > 32) return LBM_EINVAL;
    lbm_mlp* c = new (std::nothrow) lbm_mlp();
    if (!c) return LBM_ENOMEM;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete c; return LBM_ECUDA; }
    c->device = dev;
    if (cudaSetDevice(dev) != cudaSuccess) { delete c; return LBM_ECUDA; }
    c->L = nlayers;
    c->d.assign(sizes, sizes + nlayers + 1);
    c->dp = c->d;
    c->dp[nlayers] = 32;
    c->max_batch = max_batch;
    c->step = 0;
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
    if (!c->stream) {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return LBM_ECUDA; }
        c->own_stream = true;
    }
    c->offW.assign(nlayers + 1, 0);
    c->offb.assign(nlayers + 1, 0);
    long long off = 0;
    for (int l = 1; l <= nlayers; ++l) {
        c->offW[l] = off;
        off += (long long)c->dp[l] * c->d[l - 1];
        c->offb[l] = off;
        off += c->dp[l];
    }
    c->nparam = off;
    // He-normal weights (seeded), zero biases and zero padding rows
    std::vector<float> init((size_t)off, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 1; l <= nlayers; ++l) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / c->d[l - 1]));
        for (int r = 0; r < c->d[l]; ++r)
            for (int k = 0; k < c->d[l - 1]; ++k) init[(size_t)(c->offW[l] + (long long)r * c->d[l - 1] + k)] = (float)nd(rng);
    }
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(*ptr, 0, bytes, c->stream);
    };
    alloc((void**)&c->p, sizeof(float) * off);
    alloc((void**)&c->g, sizeof(float) * off);
    alloc((void**)&c->m, sizeof(float) * off);
    alloc((void**)&c->v, sizeof(float) * off);
    c->Wb.assign(nlayers + 1, nullptr);
    c->WTb.assign(nlayers + 1, nullptr);
    c->G.assign(nlayers + 1, nullptr);
    c->H.assign(nlayers, nullptr);
    int widest = 0;
    for (int l = 0; l <= nlayers; ++l) widest = std::max(widest, c->dp[l]);
    for (int l = 1; l <= nlayers; ++l) {
        alloc((void**)&c->Wb[l], sizeof(bf16) * c->dp[l] * c->d[l - 1]);
        alloc((void**)&c->WTb[l], sizeof(bf16) * c->dp[l] * c->d[l - 1]);
        alloc((void**)&c->G[l], sizeof(bf16) * (size_t)max_batch * c->dp[l]);
    }
    for (int l = 0; l < nlayers; ++l) alloc((void**)&c->H[l], sizeof(bf16) * (size_t)max_batch * c->d[l]);
    alloc((void**)&c->yhat, sizeof(float) * (size_t)max_batch * 32);
    alloc((void**)&c->T1, sizeof(bf16) * (size_t)max_batch * widest);
    alloc((void**)&c->T2, sizeof(bf16) * (size_t)max_batch * widest);
    c->loss_blocks = (int)blocks_for((long long)max_batch * 32, kLossThreads);
    alloc((void**)&c->loss_parts, sizeof(double) * c->loss_blocks);
    alloc((void**)&c->loss, sizeof(double));
    alloc((void**)&c->x_mean, sizeof(float) * c->d[0]);
    alloc((void**)&c->x_scale, sizeof(float) * c->d[0]);
    alloc((void**)&c->y_mean, sizeof(float) * 32);
    alloc((void**)&c->y_scale, sizeof(float) * 32);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->p, init.data(), sizeof(float) * off, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        // identity normalisation until set
        std::vector<float> ones(std::max(c->d[0], 32), 1.f);
        e = cudaMemcpyAsync(c->x_scale, ones.data(), sizeof(float) * c->d[0], cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->y_scale, ones.data(), sizeof(float) * 32, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = refresh_weights(c);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        const int st = mlp_status(e);
        lbm_mlp_destroy(c);
        return st;
    }
    *out = c;
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->p); cudaFree(c->g); cudaFree(c->m); cudaFree(c->v);
    for (bf16* q : c->Wb) cudaFree(q);
    for (bf16* q : c->WTb) cudaFree(q);
    for (bf16* q : c->G) cudaFree(q);
    for (bf16* q : c->H) cudaFree(q);
    cudaFree(c->yhat); cudaFree(c->T1); cudaFree(c->T2);
    cudaFree(c->loss_parts); cudaFree(c->loss);
    cudaFree(c->x_mean); cudaFree(c->x_scale); cudaFree(c->y_mean); cudaFree(c->y_scale);
    if (c->h_loss) cudaFreeHost(c->h_loss);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbm_mlp_set_normalisation(lbm_mlp* c, const float* x_mean, const float* x_scale, const float* y_mean,
                              const float* y_scale) {
    if (!c || !x_mean || !x_scale || !y_mean || !y_scale) return LBM_EINVAL;
    const int d0 = c->d[0], dL = c->d[c->L];
    for (int k = 0; k < d0; ++k)
        if (!std::isfinite(x_mean[k]) || !std::isfinite(x_scale[k])) return LBM_EINVAL;
    for (int k = 0; k < dL; ++k)
        if (!std::isfinite(y_mean[k]) || !std::isfinite(y_scale[k]) || y_scale[k] == 0.f) return LBM_EINVAL;
    cudaSetDevice(c->device);
    std::vector<float> ym(32, 0.f), ys(32, 1.f);
    for (int k = 0; k < dL; ++k) { ym[k] = y_mean[k]; ys[k] = y_scale[k]; }
    MLP_TRY(cudaMemcpyAsync(c->x_mean, x_mean, sizeof(float) * d0, cudaMemcpyHostToDevice, c->stream));
    MLP_TRY(cudaMemcpyAsync(c->x_scale, x_scale, sizeof(float) * d0, cudaMemcpyHostToDevice, c->stream));
    MLP_TRY(cudaMemcpyAsync(c->y_mean, ym.data(), sizeof(float) * 32, cudaMemcpyHostToDevice, c->stream));
    MLP_TRY(cudaMemcpyAsync(c->y_scale, ys.data(), sizeof(float) * 32, cudaMemcpyHostToDevice, c->stream));
    MLP_TRY(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_mlp_param_count(lbm_mlp* c, int64_t* n) {
    if (!c || !n) return LBM_EINVAL;
    long long s = 0;
    for (int l = 1; l <= c->L; ++l) s += (long long)c->d[l] * c->d[l - 1] + c->d[l];
    *n = s;
    return LBM_OK;
}

namespace {

// Copy between the padded device layout and the flat host layout
// W_1 [d_1, d_0], b_1, W_2, b_2, ... (to_host: device -> host).
int copy_params(lbm_mlp* c, float* dev, float* host, bool to_host) {
    cudaSetDevice(c->device);
    long long h = 0;
    for (int l = 1; l <= c->L; ++l) {
        const size_t wbytes = sizeof(float) * (size_t)c->d[l] * c->d[l - 1];  // real rows are first
        float* dw = dev + c->offW[l];
        float* db = dev + c->offb[l];
        if (to_host) {
            MLP_TRY(cudaMemcpyAsync(host + h, dw, wbytes, cudaMemcpyDeviceToHost, c->stream));
            h += (long long)c->d[l] * c->d[l - 1];
            MLP_TRY(cudaMemcpyAsync(host + h, db, sizeof(float) * c->d[l], cudaMemcpyDeviceToHost, c->stream));
        } else {
            MLP_TRY(cudaMemcpyAsync(dw, host + h, wbytes, cudaMemcpyHostToDevice, c->stream));
            h += (long long)c->d[l] * c->d[l - 1];
            MLP_TRY(cudaMemcpyAsync(db, host + h, sizeof(float) * c->d[l], cudaMemcpyHostToDevice, c->stream));
        }
        h += c->d[l];
    }
    MLP_TRY(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

}  // namespace

int lbm_mlp_get_params(lbm_mlp* c, float* params) {
    if (!c || !params) return LBM_EINVAL;
    return copy_params(c, c->p, params, true);
}

int lbm_mlp_set_params(lbm_mlp* c, const float* params) {
    if (!c || !params) return LBM_EINVAL;
    int64_t n = 0;
    lbm_mlp_param_count(c, &n);
    for (int64_t k = 0; k < n; ++k)
        if (!std::isfinite(params[k])) return LBM_EINVAL;
    int st = copy_params(c, c->p, const_cast<float*>(params), false);
    if (st) return st;
    MLP_TRY(cudaMemsetAsync(c->m, 0, sizeof(float) * c->nparam, c->stream));
    MLP_TRY(cudaMemsetAsync(c->v, 0, sizeof(float) * c->nparam, c->stream));
    c->step = 0;
    MLP_TRY(refresh_weights(c));
    MLP_TRY(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_mlp_forward(lbm_mlp* c, const float* x, float* y, int64_t n) {
    if (!c || !x || !y || n < 0) return LBM_EINVAL;
    cudaSetDevice(c->device);
    const int d0 = c->d[0], dL = c->d[c->L];
    for (int64_t s = 0; s < n; s += c->max_batch) {
        const int k = (int)std::min<int64_t>(c->max_batch, n - s);
        MLP_TRY(forward(c, x + s * d0, k));
        k_output<<<blocks_for((long long)k * dL, 256), 256, 0, c->stream>>>(c->yhat, 32, k, dL, c->y_mean, c->y_scale,
                                                                          y + s * dL);
        MLP_TRY(cudaGetLastError());
    }
    return LBM_OK;
}

int lbm_mlp_deformation(lbm_mlp* c, const float* x, int64_t n, float* m6, double* D) {
    if (!c || !x || !m6 || !D || n < 0 || c->d[c->L] != 6) return LBM_EINVAL;
    int st = lbm_mlp_forward(c, x, m6, n);
    if (st) return st;
    k_deform_from_m<<<blocks_for(n, 128), 128, 0, c->stream>>>(m6, n, D);
    MLP_TRY(cudaGetLastError());
    return LBM_OK;
}

int lbm_mlp_gradients(lbm_mlp* c, const float* x, const float* t, int64_t n, double* loss, float* grads) {
    if (!c || !x || !t || n < 32 || n > c->max_batch || n % 32 != 0) return LBM_EINVAL;
    cudaSetDevice(c->device);
    MLP_TRY(forward(c, x, (int)n));
    MLP_TRY(backward(c, t, (int)n));
    MLP_TRY(cudaMemcpyAsync(c->h_loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grads) {
        int st = copy_params(c, c->g, grads, true);
        if (st) return st;
    }
    MLP_TRY(cudaStreamSynchronize(c->stream));
    if (loss) *loss = *c->h_loss;
    return LBM_OK;
}

int lbm_mlp_train_step(lbm_mlp* c, const float* x, const float* t, int64_t n, float lr, double* loss) {
    if (!c || !x || !t || n < 32 || n > c->max_batch || n % 32 != 0 || !(lr > 0.f)) return LBM_EINVAL;
    cudaSetDevice(c->device);
    MLP_TRY(forward(c, x, (int)n));
    MLP_TRY(backward(c, t, (int)n));
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)c->step), c2 = 1.f - std::pow(b2, (float)c->step);
    k_adam<<<blocks_for(c->nparam, 256), 256, 0, c->stream>>>(c->p, c->g, c->m, c->v, c->nparam, lr, b1, b2, 1e-8f,
                                                             c1, c2);
    MLP_TRY(cudaGetLastError());
    MLP_TRY(refresh_weights(c));
    if (loss) {
        MLP_TRY(cudaMemcpyAsync(c->h_loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        MLP_TRY(cudaStreamSynchronize(c->stream));
        *loss = *c->h_loss;
    }
    return LBM_OK;
}

int lbm_mlp_sync(lbm_mlp* c) {
    if (!c) return LBM_EINVAL;
    cudaSetDevice(c->device);
    MLP_TRY(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

}  // extern "C"
