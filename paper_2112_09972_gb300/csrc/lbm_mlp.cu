// Learned surrogate of the droplet's conformation tensor (an addition of this
// library beside the paper's method): a multilayer perceptron that maps a
// window of the velocity gradient A(t) to the six entries of the droplet's
// conformation tensor M = I / det(I)^(1/3) (I the second-moment tensor of
// Sec. 2, Eq. 4; M = identity for a sphere, the Maffettone-Minale tensor of
// Eqs. 1, 2).  Forward pass, backward pass and Adam run on the GPU:
//
//   k_gemm_tc   -- C = A B^T on the 5th-generation tensor cores (tcgen05.mma,
//                  accumulator in tensor memory) for 128 x 128 tiles, A [M, K]
//                  and B [N, K] with K contiguous, fused epilogues (bias +
//                  ReLU to bfloat16, ReLU-derivative mask to bfloat16,
//                  float32 output)
//   k_gemm_nt   -- the same on warp-level tensor cores (mma.sync m16n8k16,
//                  float32 accumulation) for the shapes k_gemm_tc does not
//                  tile (ragged M or N, the 32-wide output layer)
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

#include <cuda_bf16.h>
#include <cuda_runtime.h>
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
// The same C = A B^T on the 5th-generation tensor cores (tcgen05): a 128 x 128
// float32 tile accumulates in tensor memory (TMEM, 128 columns); operands are
// staged K-major in shared memory in the 128-byte swizzled layout by cp.async;
// one thread issues tcgen05.mma (kind::f16, bfloat16 inputs, M 128, N 128,
// K 16) and commits each K chunk to that stage's mbarrier; the four warps then
// read their 32 TMEM lanes (rows) with tcgen05.ld and apply the epilogue.
// Requires M and N multiples of 128 and K a multiple of 64.
constexpr int TC_M = 128, TC_N = 128, TC_K = 64;
constexpr int kTcThreads = 128;
constexpr unsigned kTcWaitPolls = 1u << 22;

__device__ __forceinline__ unsigned tc_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading-dimension (K
// direction) and stride-dimension (M/N direction) byte offsets, no swizzle.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version of sm_100 and later
    return d;          // base offset 0, swizzle mode 0 (none)
}

// Instruction descriptor of kind::f16: float32 D, bfloat16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr unsigned tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
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

// Shared memory of k_gemm_tc: kTcStages stages of the A and B tiles of one K
// chunk, each tile 128 rows of 128 bytes (64 bfloat16) in the 128-byte
// swizzled K-major layout (8-row atoms of 1024 bytes; the 16-byte piece j of
// row r sits at piece j ^ (r % 8) of its row), then one mbarrier per stage
// and the TMEM base address.  Chunks are loaded kTcAhead chunks ahead, into
// the stage whose products (two chunks back) have completed.  Three stages
// (97 KB) let two CTAs share an SM, so that one's epilogue overlaps the
// other's loads and products.
constexpr int kTcStages = 3, kTcAhead = kTcStages - 2;
constexpr unsigned kTcTileBytes = TC_M * TC_K * 2;  // 16 KB per operand tile
constexpr unsigned kTcSmem = 1024 + kTcStages * 2 * kTcTileBytes + 8 * kTcStages + 16;

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Shared-memory matrix descriptor of a 128-byte swizzled K-major tile: start
// address, stride between 8-row atoms (SBO), swizzle mode 2 (128 bytes).
__device__ __forceinline__ unsigned long long tc_desc_sw128(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= 1ull << 16;                          // leading byte offset: unused with this swizzle
    d |= (unsigned long long)(1024 >> 4) << 32;  // next 8-row atom
    d |= 1ull << 46;                          // descriptor version of sm_100 and later
    d |= 2ull << 61;                          // 128-byte swizzle
    return d;
}

__global__ void __launch_bounds__(kTcThreads, 2) k_gemm_tc(GemmArgs g, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    gemm_slice(g);
    const unsigned raw = tc_smem(tc_smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
    const unsigned mbar0 = base + kTcStages * 2 * kTcTileBytes;  // mbarrier of stage s at mbar0 + 8 s
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(tc_smem_raw + (mbar0 + 8 * kTcStages - raw));
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;

    if (warp == 0) {  // 128 TMEM columns: lanes = rows, columns = N
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(tc_smem(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int st = 0; st < kTcStages; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8u * st) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    constexpr unsigned IDESC = tc_idesc(TC_M, TC_N);
    const int nk = g.K / TC_K;
    auto tile = [&](int st) { return base + (unsigned)(2 * st) * kTcTileBytes; };
    auto load = [&](int kt, int st) {  // one commit group per call (empty past the last chunk)
        if (kt < nk) {
            const unsigned a_s = tile(st), b_s = a_s + kTcTileBytes;
            const int k0 = kt * TC_K;
            for (int c = t; c < TC_M * (TC_K / 8); c += kTcThreads) {
                const int r = c >> 3, j = c & 7;
                const unsigned off = (unsigned)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
                cp_async16(a_s + off, g.A + (long long)(m0 + r) * g.lda + k0 + 8 * j);
                cp_async16(b_s + off, g.B + (long long)(n0 + r) * g.ldb + k0 + 8 * j);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    bool ok = true;
    unsigned phase = 0, pending = 0;  // per stage: parity of its next completion, a commit not yet waited
    auto wait_stage = [&](int st) {
        unsigned polls = 0;
        while (!tc_mbar_try_wait(mbar0 + 8u * st, (phase >> st) & 1u)) {
            if (++polls == kTcWaitPolls) {
                ok = false;
                return;
            }
        }
        phase ^= 1u << st;
        pending &= ~(1u << st);
    };

    for (int q = 0; q < kTcAhead; ++q) load(q, q);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt % kTcStages;
        // chunk kt + kTcAhead goes to the stage chunk kt - 2 used
        const int nx = kt + kTcAhead, sx = nx % kTcStages;
        if (nx < nk && ((pending >> sx) & 1u)) wait_stage(sx);
        load(nx, sx);
        asm volatile("cp.async.wait_group %0;" ::"n"(kTcAhead) : "memory");  // chunk kt has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");        // generic writes -> tensor core reads
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            break;
        }
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a_s = tile(st), b_s = a_s + kTcTileBytes;
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk) {
                // K step of 16 = 32 bytes along the swizzled 128-byte rows
                const unsigned long long ad = tc_desc_sw128(a_s + 32u * kk);
                const unsigned long long bd = tc_desc_sw128(b_s + 32u * kk);
                const unsigned acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             mbar0 + 8u * st)
                         : "memory");
        }
        pending |= 1u << st;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the loop
    // the products not waited for yet (at most one per stage)
    for (int st = 0; st < kTcStages; ++st)
        if ((pending >> st) & 1u) wait_stage(st);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) {
        // a wait gave up: report it, and wait once more (bounded) for the
        // products in flight before the tensor memory is released
        if (t == 0) atomicOr(err, 1);
        for (int st = 0; st < kTcStages; ++st) {
            if (!((pending >> st) & 1u)) continue;
            unsigned polls = 0;
            while (!tc_mbar_try_wait(mbar0 + 8u * st, (phase >> st) & 1u) && ++polls < kTcWaitPolls) {
            }
        }
    }

    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (rows), 32 columns at a time
    if (ok) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < TC_N; cb += 32) {
            unsigned r[32];
            const unsigned addr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)cb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // this thread's row, 32 consecutive columns: 16-byte stores
            const int n = n0 + cb;
            if (g.epi == kStoreF32 || g.epi == kBiasF32) {
                float4* dst = reinterpret_cast<float4*>(g.Cf + (long long)m * g.ldc + n);
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
            } else {
                uint4* dst = reinterpret_cast<uint4*>(g.Cb + (long long)m * g.ldc + n);
                const uint4* mk =
                    g.epi == kMaskBf16 ? reinterpret_cast<const uint4*>(g.mask + (long long)m * g.ldm + n) : nullptr;
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
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
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

// Whether k_gemm_tc takes this product: the 128 x 128 x 64 tiling, 16-byte
// aligned operand rows for cp.async, and 16-byte aligned output, bias and
// mask rows for the vector epilogue.
bool tc_ok(const lbm_mlp* c, const GemmArgs& a) {
    if (c->tensor_path != 0 || a.M % TC_M || a.N % TC_N || a.K % TC_K || a.k_len % TC_K) return false;
    if (!aligned16(a.A) || !aligned16(a.B) || a.lda % 8 || a.ldb % 8) return false;
    switch (a.epi) {
        case kStoreF32: return aligned16(a.Cf) && a.ldc % 4 == 0 && a.c_split % 4 == 0;
        case kBiasF32: return aligned16(a.Cf) && a.ldc % 4 == 0 && aligned16(a.bias);
        case kBiasReluBf16: return aligned16(a.Cb) && a.ldc % 8 == 0 && aligned16(a.bias);
        default: return aligned16(a.Cb) && a.ldc % 8 == 0 && aligned16(a.mask) && a.ldm % 8 == 0;
    }
}

cudaError_t launch_gemm(lbm_mlp* c, const GemmArgs& a, int slices) {
    if (tc_ok(c, a)) {
        const dim3 grid(a.N / TC_N, a.M / TC_M, slices);
        k_gemm_tc<<<grid, kTcThreads, kTcSmem, c->stream>>>(a, c->d_err);
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
// gradients): K is cut into slices so that the tiles x slices fill about two
// CTAs per SM, each slice at least 8 K chunks; the float32 partials go to the
// workspace and k_splitsum adds them in slice order.
cudaError_t gemm_long_k(lbm_mlp* c, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K,
                        float* out) {
    GemmArgs a = gemm_args(A, lda, B, ldb, M, N, K, kStoreF32, nullptr, nullptr, 0, out, nullptr, N);
    const bool tc = tc_ok(c, a);
    const int unit = tc ? TC_K : BK;
    const long long tiles =
        tc ? (long long)(M / TC_M) * (N / TC_N) : (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
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
