// Learned surrogate of the droplet's conformation tensor (an addition of this
// library beside the paper's method): a multilayer perceptron that maps a
// window of the velocity gradient A(t) to the six entries of the droplet's
// conformation tensor M = I / det(I)^(1/3) (I the second-moment tensor of
// Sec. 2, Eq. 4; M = identity for a sphere, the Maffettone-Minale tensor of
// Eqs. 1, 2).  Forward pass, backward pass and Adam run on the GPU:
//
//   k_gemm_tc   -- C = A B^T on the 5th-generation tensor cores: a
//                  persistent, warp-specialised kernel (TMA loads into a
//                  shared-memory ring, tcgen05.mma into a double-buffered
//                  tensor-memory accumulator, eight epilogue warps) over
//                  128 x BN tiles (BN 128, 64 or 32) and split-K slices; A
//                  [M, K] and B [N, K] with K contiguous; fused epilogues
//                  (bias + ReLU to bfloat16, ReLU-derivative mask to
//                  bfloat16, float32 output)
//   k_gemm_nt   -- the same on warp-level tensor cores (mma.sync m16n8k16,
//                  float32 accumulation) for the shapes k_gemm_tc does not
//                  tile (M not a multiple of 128, N not of 32, K not of 64)
//   k_transpose -- bfloat16 tile transpose (operands of the weight gradients)
//   k_prep, k_loss_grad, k_colsum_*, k_splitsum, k_adam, k_weights, k_output,
//   k_deform_from_m -- input normalisation, mean-square loss and its
//                  gradient, bias gradients, the sum of split-K partial
//                  weight gradients, Adam, bfloat16 weight copies,
//                  output scaling, and D of a predicted M (Eq. 4).
//
// Layers: z_l = h_{l-1} W_l^T + b_l, h_l = max(z_l, 0), last layer linear;
// inputs normalised as (x - x_mean) x_scale, outputs y = y_hat / y_scale +
// y_mean, loss = mean over samples and outputs of (y_hat - t_hat)^2.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
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
    // Split K (kStoreF32 only): slice z = blockIdx.z covers K columns
    // [z k_len, min((z + 1) k_len, K)) and writes its partial product at
    // Cf + z c_split.  k_len = 0: one slice.
    int k_len;
    long long c_split;
};

// The K slice of blockIdx.z (see GemmArgs::k_len).
__device__ __forceinline__ void gemm_slice(GemmArgs& g) {
    if (g.k_len <= 0) return;
    const int k0 = blockIdx.z * g.k_len;
    g.A += k0;
    g.B += k0;
    g.K = min(g.k_len, g.K - k0);
    g.Cf += (long long)blockIdx.z * g.c_split;
}

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
    gemm_slice(g);
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

// ---------------------------------------------------------------------------
// The same C = A B^T on the 5th-generation tensor cores: a persistent kernel,
// one CTA per SM walking 128 x BN output tiles (BN in {32, 64, 128}; the K
// slices of a split-K product are tiles too), with three roles:
//   warp 0    -- one thread loads the A and B tiles of each 64-wide K chunk by
//                TMA (cp.async.bulk.tensor, 128-byte swizzle) into a ring of
//                kTcStages stages, counting the bytes on the stage's "full"
//                mbarrier, once the products of the chunk that used the stage
//                before have released it (its "empty" mbarrier);
//   warp 1    -- allocates 256 TMEM columns (two 128-column float32
//                accumulators); one thread issues tcgen05.mma (kind::f16,
//                M 128, N BN, K 16) for each chunk, releases the stage with
//                tcgen05.commit, and commits a finished tile to its
//                accumulator's "full" mbarrier;
//   warps 2-9 -- the epilogue: two warps per 32 TMEM lanes (rows), each
//                taking every other 32-column block; a warp reads its block
//                with tcgen05.ld, applies the fused epilogue, stores 16-byte
//                vectors and hands the accumulator back (its "empty"
//                mbarrier), while the tensor core fills the other one.
// Every wait is bounded.  A wait that gives up sets bit 1 of *err and stops
// every role; before the CTA exits, the copies and products it issued are
// waited for (bounded) and the tensor memory is released.
constexpr int TC_M = 128, TC_K = 64;
constexpr int kTcThreads = 320;
constexpr int kTcEpiWarps = 8;  // warps 2 .. 9
constexpr int kTcStages = 6;
constexpr unsigned kTcTileA = TC_M * TC_K * 2;               // 16 KB
constexpr unsigned kTcStageBytes = 2 * kTcTileA;             // A tile + B tile (BN <= 128 rows)
constexpr int kTcBars = 2 * kTcStages + 2 + 2 + 1;           // full, empty, acc full, acc empty, drain
constexpr unsigned kTcSmem = 1024 + kTcStages * kTcStageBytes + 8 * kTcBars + 16;
constexpr unsigned long long kTcWaitNs = 2000000000ull;  // 2 s per wait
constexpr unsigned kTcCols = 256;

// Tiles of one product: m_tiles x n_tiles output tiles of 128 x bn, times
// the K slices.
struct TcShape {
    int m_tiles, n_tiles, slices, bn;
};

__device__ __forceinline__ unsigned tc_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a 128-byte swizzled K-major tile: start
// address, stride between 8-row atoms (SBO), swizzle mode 2 (128 bytes).
__device__ __forceinline__ unsigned long long tc_desc_sw128(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= 1ull << 16;                             // leading byte offset: unused with this swizzle
    d |= (unsigned long long)(1024 >> 4) << 32;  // next 8-row atom
    d |= 1ull << 46;                             // descriptor version of sm_100 and later
    d |= 2ull << 61;                             // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: float32 D, bfloat16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ unsigned tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mbar_init(unsigned mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ bool tc_mbar_try_wait(unsigned mbar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ unsigned long long tc_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of the given parity: gives up after
// kTcWaitNs of wall time (try_wait may suspend the thread for a while, so
// the bound is on time, not on polls), or early once *stop is set (if stop
// is not null).
__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity, const volatile int* stop) {
    if (tc_mbar_try_wait(mbar, parity)) return true;
    const unsigned long long t0 = tc_now_ns();
    for (;;) {
        if (tc_mbar_try_wait(mbar, parity)) return true;
        if ((stop && *stop) || tc_now_ns() - t0 > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ void tc_expect_tx(unsigned mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tc_arrive(unsigned mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// TMA load of the box at (c0 = K, c1 = row) of a 2-D tensor map into shared
// memory, counted on mbar.  c0 is a multiple of 64 elements (128 bytes).
__device__ __forceinline__ void tc_tma_load(unsigned dst, const CUtensorMap* map, int c0, int c1, unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Epilogue of 32 consecutive columns n .. n + 31 of row m (accumulators r):
// 16-byte stores of the fused result.
__device__ __forceinline__ void tc_store32(const GemmArgs& g, float* Cf, int m, int n, const unsigned (&r)[32]) {
    if (g.epi == kStoreF32 || g.epi == kBiasF32) {
        float4* dst = reinterpret_cast<float4*>(Cf + (long long)m * g.ldc + n);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float4 v = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                   __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            if (g.epi == kBiasF32) {
                const float4 bq = reinterpret_cast<const float4*>(g.bias + n)[q];
                v.x += bq.x; v.y += bq.y; v.z += bq.z; v.w += bq.w;
            }
            dst[q] = v;
        }
        return;
    }
    uint4* dst = reinterpret_cast<uint4*>(g.Cb + (long long)m * g.ldc + n);
    const uint4* mk = g.epi == kMaskBf16 ? reinterpret_cast<const uint4*>(g.mask + (long long)m * g.ldm + n) : nullptr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[8 * q + e]);
        if (g.epi == kBiasReluBf16) {
            const float4 b0 = reinterpret_cast<const float4*>(g.bias + n)[2 * q];
            const float4 b1 = reinterpret_cast<const float4*>(g.bias + n)[2 * q + 1];
            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = fmaxf(v[e] + bb[e], 0.f);
        } else {  // kMaskBf16: keep where the stored activation is positive
            const uint4 mv = mk[q];
            const unsigned mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (!(__uint_as_float(mw[e] << 16) > 0.f)) v[2 * e] = 0.f;
                if (!(__uint_as_float(mw[e] & 0xFFFF0000u) > 0.f)) v[2 * e + 1] = 0.f;
            }
        }
        unsigned w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);  // .x at the lower address
            w[e] = *reinterpret_cast<const unsigned*>(&h);
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs g,
              TcShape sh, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ int stop_flag;
    const unsigned raw = tc_smem(tc_smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
    const unsigned bar0 = base + kTcStages * kTcStageBytes;
    const unsigned drain_bar = bar0 + 8u * (2 * kTcStages + 4);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(tc_smem_raw + (bar0 + 8u * kTcBars - raw));
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (kTcStages + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * kTcStages + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * kTcStages + 2 + b); };
    volatile int* stop = &stop_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    if (t == 0) {
        stop_flag = 0;
        for (int s = 0; s < kTcStages; ++s) {
            tc_mbar_init(full_bar(s), 1);
            tc_mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc_mbar_init(accf_bar(b), 1);
            tc_mbar_init(acce_bar(b), kTcEpiWarps);  // one arrival per epilogue warp
        }
        tc_mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tmem_slot)),
                     "n"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    const int tiles_mn = sh.m_tiles * sh.n_tiles, tiles = tiles_mn * sh.slices;
    // K range of a tile: chunks [k0 / 64, k0 / 64 + nk)
    auto tile_k = [&](int tile, int& k0, int& nk) {
        const int z = tile / tiles_mn;
        k0 = g.k_len > 0 ? z * g.k_len : 0;
        nk = (g.k_len > 0 ? min(g.k_len, g.K - k0) : g.K) / TC_K;
    };
    auto give_up = [&]() {
        *stop = 1;
        atomicOr(err, 1);
    };
    unsigned issued = 0;  // warp 0, lane 0: chunks loaded

    if (warp == 0) {
        if (lane == 0) {
            const unsigned bytes = kTcTileA + (unsigned)sh.bn * TC_K * 2u;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < tiles && !*stop; tile += gridDim.x) {
                const int r = tile % tiles_mn, m0 = (r / sh.n_tiles) * TC_M, n0 = (r % sh.n_tiles) * sh.bn;
                int k0, nk;
                tile_k(tile, k0, nk);
                for (int kt = 0; kt < nk; ++kt) {
                    const int s = (int)(issued % kTcStages);
                    const unsigned round = issued / kTcStages;
                    if (round > 0 && !tc_wait(empty_bar(s), (round - 1u) & 1u, stop)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    const unsigned a_s = base + (unsigned)s * kTcStageBytes;
                    tc_expect_tx(full_bar(s), bytes);
                    tc_tma_load(a_s, &tmA, k0 + kt * TC_K, m0, full_bar(s));
                    tc_tma_load(a_s + kTcTileA, &tmB, k0 + kt * TC_K, n0, full_bar(s));
                    ++issued;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned idesc = tc_idesc(TC_M, sh.bn);
            unsigned it = 0, tc = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < tiles && !*stop; tile += gridDim.x) {
                int k0, nk;
                tile_k(tile, k0, nk);
                const int buf = (int)(tc & 1u);
                const unsigned use = tc >> 1;
                if (use > 0 && !tc_wait(acce_bar(buf), (use - 1u) & 1u, stop)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned acc = tmem + (unsigned)buf * 128u;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = (int)(it % kTcStages);
                    if (!tc_wait(full_bar(s), (it / kTcStages) & 1u, stop)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned a_s = base + (unsigned)s * kTcStageBytes, b_s = a_s + kTcTileA;
#pragma unroll
                    for (int kk = 0; kk < TC_K / 16; ++kk) {
                        // K step of 16 = 32 bytes along the swizzled 128-byte rows
                        const unsigned long long ad = tc_desc_sw128(a_s + 32u * kk);
                        const unsigned long long bd = tc_desc_sw128(b_s + 32u * kk);
                        const unsigned accumulate = (kt > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(acc),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
                            : "memory");
                    }
                    tc_commit(empty_bar(s));  // the stage is free once these products complete
                }
                if (!ok) break;
                tc_commit(accf_bar(buf));
                ++tc;
            }
            tc_commit(drain_bar);  // completes when every product issued above has
        }
    } else {
        const int q = warp & 3;             // a warp reads TMEM lanes 32 (warp % 4) .. + 31
        const int first = ((warp - 2) >> 2) * 32;  // and column blocks first, first + 64, ...
        unsigned tc = 0;
        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tc) {
            const int buf = (int)(tc & 1u);
            int okw = 1;
            if (lane == 0) okw = tc_wait(accf_bar(buf), (tc >> 1) & 1u, stop) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) {
                if (lane == 0) give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int r = tile % tiles_mn, m0 = (r / sh.n_tiles) * TC_M, n0 = (r % sh.n_tiles) * sh.bn;
            float* Cf = g.Cf ? g.Cf + (long long)(tile / tiles_mn) * g.c_split : nullptr;
            const int m = m0 + q * 32 + lane;
#pragma unroll 1
            for (int cb = first; cb < sh.bn; cb += 64) {
                unsigned v[32];
                const unsigned addr = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(buf * 128 + cb);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                tc_store32(g, Cf, m, n0 + cb, v);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(acce_bar(buf));  // the accumulator may be overwritten
        }
    }

    __syncthreads();
    if (warp == 0 && lane == 0 && *stop) {
        // copies issued but perhaps not consumed: the last one of each stage
        for (int s = 0; s < kTcStages; ++s) {
            if (issued <= (unsigned)s) continue;
            const unsigned last = issued - 1u - ((issued - 1u - (unsigned)s) % kTcStages);
            tc_wait(full_bar(s), (last / kTcStages) & 1u, nullptr);
        }
    }
    if (warp == 1 && lane == 0 && !tc_wait(drain_bar, 0u, nullptr)) atomicOr(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcCols) : "memory");
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

// The same, eight elements per thread (x 16-byte aligned, d0 a multiple of 8):
// two float4 loads, one 16-byte store.
__global__ void k_prep8(const float4* __restrict__ x, long long n8, int d08, const float4* __restrict__ mean,
                        const float4* __restrict__ scale, uint4* __restrict__ xb) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n8) return;
    const int c = (int)(e % d08);
    const float4 a = x[2 * e], b = x[2 * e + 1];
    const float4 ma = mean[2 * c], mb = mean[2 * c + 1], sa = scale[2 * c], sb = scale[2 * c + 1];
    const float v[8] = {(a.x - ma.x) * sa.x, (a.y - ma.y) * sa.y, (a.z - ma.z) * sa.z, (a.w - ma.w) * sa.w,
                        (b.x - mb.x) * sb.x, (b.y - mb.y) * sb.y, (b.z - mb.z) * sb.z, (b.w - mb.w) * sb.w};
    unsigned w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const unsigned*>(&h);
    }
    xb[e] = make_uint4(w[0], w[1], w[2], w[3]);
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
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // n ldg <= 2^22 x 32
    double sq = 0.0;
    if (e < n * ldg) {
        const int r = e / ldg, c = e % ldg;
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

// Sum of the partials divided by count: the mean loss.  A fixed summation
// order (thread t takes partials t, t + 256, ..., then a tree over threads),
// so the result does not depend on scheduling.
constexpr int kLossFinalThreads = 256;
__global__ void __launch_bounds__(kLossFinalThreads) k_loss_final(const double* __restrict__ parts, int nparts,
                                                                  double count, double* __restrict__ out) {
    __shared__ double red[kLossFinalThreads];
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kLossFinalThreads) s += parts[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kLossFinalThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / count;
}

// Bias gradient db[c] = sum_r g[r, c] of a bfloat16 [n, C] matrix, in two
// passes with a fixed order: block (x, s) sums rows [s rows, (s + 1) rows)
// of 32 columns (8 row phases, then the phases in order) into parts[s, c];
// k_colsum_final adds the slices in order.
constexpr int kColSlices = 128;
__global__ void __launch_bounds__(256) k_colsum_part(const bf16* __restrict__ g, int n, int C, int ldg, int rows,
                                                     float* __restrict__ parts) {
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * rows, r1 = min(n, r0 + rows);
    float s = 0.f;
    if (c < C)
        for (int r = r0 + threadIdx.y; r < r1; r += 8) s += __bfloat162float(g[(long long)r * ldg + c]);
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < C) {
        float t = red[0][threadIdx.x];
        for (int k = 1; k < 8; ++k) t += red[k][threadIdx.x];
        parts[(long long)blockIdx.y * C + c] = t;
    }
}

__global__ void k_colsum_final(const float* __restrict__ parts, int S, int C, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += parts[(long long)z * C + c];
    db[c] = s;
}

// out[e] = sum over the S K slices of ws[z count + e], in slice order.
constexpr int kMaxSplit = 32;
__global__ void k_splitsum(const float* __restrict__ ws, int S, long long count, float* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float s = ws[e];
    for (int z = 1; z < S; ++z) s += ws[(long long)z * count + e];
    out[e] = s;
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
    int tensor_path;             // 0: tcgen05 where the shape allows, 1: mma.sync only
    int* d_err;                  // bit 1: a bounded tensor-core wait gave up
    int sms;                     // multiprocessors of the device
    float* ws;                   // split-K partials, kMaxSplit x the largest weight matrix
    float* cs_parts;             // column-sum partials, kColSlices x the widest layer
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

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// cuTensorMapEncodeTiled from the driver, found once through the runtime
// (no link against the driver library); null if the driver lacks it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// TMA map of a bfloat16 [rows, K] matrix with row stride ld (elements):
// boxes of 64 (K) x box_rows, 128-byte swizzle (the layout k_gemm_tc's
// descriptors name).
bool tc_map(CUtensorMap* map, const bf16* ptr, int rows, int K, int ld, int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_K, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The N tile with which k_gemm_tc takes this product, or 0 for k_gemm_nt:
// M a multiple of 128, N of 32 (the tile is the largest of 128, 64, 32
// dividing it), K and the K slice of 64; 16-byte aligned operand rows for TMA
// and 16-byte aligned output, bias and mask rows for the vector epilogue.
int tc_bn(const lbm_mlp* c, const GemmArgs& a) {
    if (c->tensor_path != 0 || !tensor_map_encoder()) return 0;
    if (a.M % TC_M || a.K % TC_K || a.k_len % TC_K) return 0;
    const int bn = a.N % 128 == 0 ? 128 : a.N % 64 == 0 ? 64 : a.N % 32 == 0 ? 32 : 0;
    if (!bn || !aligned16(a.A) || !aligned16(a.B) || a.lda % 8 || a.ldb % 8) return 0;
    bool ok;
    switch (a.epi) {
        case kStoreF32: ok = aligned16(a.Cf) && a.ldc % 4 == 0 && a.c_split % 4 == 0; break;
        case kBiasF32: ok = aligned16(a.Cf) && a.ldc % 4 == 0 && aligned16(a.bias); break;
        case kBiasReluBf16: ok = aligned16(a.Cb) && a.ldc % 8 == 0 && aligned16(a.bias); break;
        default: ok = aligned16(a.Cb) && a.ldc % 8 == 0 && aligned16(a.mask) && a.ldm % 8 == 0;
    }
    return ok ? bn : 0;
}

cudaError_t launch_gemm(lbm_mlp* c, const GemmArgs& a, int slices) {
    const int bn = tc_bn(c, a);
    CUtensorMap ma, mb;
    if (bn && tc_map(&ma, a.A, a.M, a.K, a.lda, TC_M) && tc_map(&mb, a.B, a.N, a.K, a.ldb, bn)) {
        const TcShape sh{a.M / TC_M, a.N / bn, slices, bn};
        const long long tiles = (long long)sh.m_tiles * sh.n_tiles * slices;
        const int grid = (int)std::min<long long>(tiles, c->sms);  // persistent: one CTA per SM at most
        k_gemm_tc<<<grid, kTcThreads, kTcSmem, c->stream>>>(ma, mb, a, sh, c->d_err);
    } else {
        const dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, slices);
        k_gemm_nt<<<grid, kGemmThreads, 0, c->stream>>>(a);
    }
    return cudaGetLastError();
}

GemmArgs gemm_args(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int epi, const float* bias,
                   const bf16* mask, int ldm, float* Cf, bf16* Cb, int ldc) {
    GemmArgs a;
    a.A = A; a.B = B; a.lda = lda; a.ldb = ldb; a.M = M; a.N = N; a.K = K; a.epi = epi;
    a.bias = bias; a.mask = mask; a.ldm = ldm; a.Cf = Cf; a.Cb = Cb; a.ldc = ldc;
    a.k_len = 0; a.c_split = 0;
    return a;
}

cudaError_t gemm(lbm_mlp* c, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int epi,
                 const float* bias, const bf16* mask, int ldm, float* Cf, bf16* Cb, int ldc) {
    return launch_gemm(c, gemm_args(A, lda, B, ldb, M, N, K, epi, bias, mask, ldm, Cf, Cb, ldc), 1);
}

// out [M, N] (row stride N) = A B^T for a long K (the batch of the weight
// gradients): K is cut into slices so that there are about two tiles x
// slices per SM, each slice at least 8 K chunks; the float32 partials go to the
// workspace and k_splitsum adds them in slice order.
cudaError_t gemm_long_k(lbm_mlp* c, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K,
                        float* out) {
    GemmArgs a = gemm_args(A, lda, B, ldb, M, N, K, kStoreF32, nullptr, nullptr, 0, out, nullptr, N);
    const int bn = tc_bn(c, a);
    const int unit = bn ? TC_K : BK;
    const long long tiles =
        bn ? (long long)(M / TC_M) * (N / bn) : (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    long long S = std::max(1LL, 2LL * c->sms / tiles);
    S = std::min<long long>(std::min<long long>(S, kMaxSplit), std::max(1, K / (8 * unit)));
    if (S <= 1) return launch_gemm(c, a, 1);
    const int k_len = (int)(((K + S - 1) / S + unit - 1) / unit * unit);
    const int slices = (K + k_len - 1) / k_len;
    a.Cf = c->ws;
    a.k_len = k_len;
    a.c_split = (long long)M * N;
    cudaError_t e = launch_gemm(c, a, slices);
    if (e != cudaSuccess) return e;
    k_splitsum<<<blocks_for(a.c_split, 256), 256, 0, c->stream>>>(c->ws, slices, a.c_split, out);
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
    if (aligned16(x)) {  // d0 is a multiple of 32
        const long long n8 = (long long)n * d0 / 8;
        k_prep8<<<blocks_for(n8, 256), 256, 0, c->stream>>>(reinterpret_cast<const float4*>(x), n8, d0 / 8,
                                                            reinterpret_cast<const float4*>(c->x_mean),
                                                            reinterpret_cast<const float4*>(c->x_scale),
                                                            reinterpret_cast<uint4*>(c->H[0]));
    } else {
        k_prep<<<blocks_for((long long)n * d0, 256), 256, 0, c->stream>>>(x, n, d0, c->x_mean, c->x_scale, c->H[0]);
    }
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
    k_loss_final<<<1, kLossFinalThreads, 0, c->stream>>>(c->loss_parts, nb, (double)n * dL, c->loss);
    cudaError_t e = cudaGetLastError();
    for (int l = L; l >= 1 && e == cudaSuccess; --l) {
        const int dout = c->dp[l], din = c->d[l - 1];
        // dW_l = G_l^T H_{l-1}: operands with the batch index contiguous
        e = transpose(c, c->G[l], n, dout, dout, c->T1, n);
        if (e == cudaSuccess) e = transpose(c, c->H[l - 1], n, din, din, c->T2, n);
        if (e == cudaSuccess) e = gemm_long_k(c, c->T1, n, c->T2, n, dout, din, n, c->g + c->offW[l]);
        if (e == cudaSuccess) {
            const int S = (int)std::min<long long>(kColSlices, blocks_for(n, 256));
            const int rows = (n + S - 1) / S;
            k_colsum_part<<<dim3((dout + 31) / 32, S), dim3(32, 8), 0, c->stream>>>(c->G[l], n, dout, dout, rows,
                                                                                   c->cs_parts);
            k_colsum_final<<<blocks_for(dout, 128), 128, 0, c->stream>>>(c->cs_parts, S, dout, c->g + c->offb[l]);
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
    // dynamic shared memory of the tensor-core GEMM above the 48 KB default
    if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return LBM_ECUDA;
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
    alloc((void**)&c->d_err, sizeof(int));
    long long largest = 0;
    for (int l = 1; l <= nlayers; ++l) largest = std::max(largest, (long long)c->dp[l] * c->d[l - 1]);
    alloc((void**)&c->ws, sizeof(float) * kMaxSplit * largest);
    alloc((void**)&c->cs_parts, sizeof(float) * kColSlices * widest);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
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
    cudaFree(c->loss_parts); cudaFree(c->loss); cudaFree(c->d_err); cudaFree(c->ws); cudaFree(c->cs_parts);
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
    if (!c || n < 0 || (n > 0 && (!x || !y))) return LBM_EINVAL;
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
    if (!c || n < 0 || (n > 0 && (!x || !m6 || !D)) || c->d[c->L] != 6) return LBM_EINVAL;
    int st = lbm_mlp_forward(c, x, m6, n);
    if (st || n == 0) return st;  // no launch for an empty batch
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
    int err = 0;
    MLP_TRY(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MLP_TRY(cudaStreamSynchronize(c->stream));
    return err ? LBM_ETIMEOUT : LBM_OK;
}

int lbm_mlp_set_tensor_path(lbm_mlp* c, int32_t path) {
    if (!c || path < 0 || path > 1) return LBM_EINVAL;
    c->tensor_path = path;
    return LBM_OK;
}

}  // extern "C"
