// Row-tiled, cluster-pipelined variant of the fused pull-stream + Shan-Chen
// force + collision step (Sec. 2, Eqs. 6-10 of Milan et al., arXiv:2112.09972)
// for boxes whose x extent is one CTA row (Lx = TX in {32, 64, 128, 256}),
// with float32 populations or 16-bit deviation storage (lbm_dev.cuh) and
// float32 arithmetic.
//
// Work decomposition.  A CTA of TX threads owns one row y of the box and
// marches a chunk of z planes; CY consecutive rows form a thread-block
// cluster.  Per plane and thread (one node x):
//   * the 38 populations pulled into the node (x - c_i) are read and summed
//     into the node's post-streaming densities, which go into a ring of
//     density planes in shared memory (CY + 2 slots); one plane later the same 38
//     values are read again for the collision (that second read is served by
//     L1/L2).  Holding no populations on chip keeps each CTA at a few KB of
//     shared memory and few registers, so many CTAs per SM hide the latency;
//   * each CTA pushes its row of densities into the rings of the CTAs that
//     own rows y -/+ 1 with st.async, which counts the bytes on the
//     receiving CTA's mbarrier for that plane; the force (Eq. 7) then reads
//     all 18 neighbour densities from local shared memory after a bounded
//     mbarrier wait.  Only the two rows just outside the cluster are pulled
//     a second time (ratio 2/CY); that work is split evenly over the CTAs of
//     the cluster, which push those densities into the edge CTAs' rings.
// There is no cluster-wide barrier and no memory fence per plane: a CTA waits
// only for the two rows it reads.  DRAM sees about one read and one write of
// every population; L2 serves the second read and the outer-halo reads.
//
// Sums over opposite velocity pairs are differenced first (c_{2k} = -c_{2k-1}),
// and the equilibria of a pair share their even part.
//
// Variants (lbm_opts.row_variant): the direct loads above (the automatic
// choice); whole pulled rows staged in shared memory by bulk copies
// (k_stream_collide_rows<..., STAGED = true>); and loader and collider
// threads per row (k_stream_collide_ws).  All three share collide_node and
// store bit-identical states.  The direct variant also has an MRT instance
// for float32 storage (collide_node<..., MRT = true>).

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "lbm_centre.cuh"
#include "lbm_dev.cuh"
#include "lbm_internal.h"
#include "lbm_lattice.cuh"

namespace cg = cooperative_groups;

namespace lbmgb {
namespace {

struct FastModel {
    float inv_tau[2], tau[2], G, rho_b[2];
    float mrt[5];  // MRT free rates (s_e, s_eps, s_q, s_pi, s_m) when the kernel relaxes moments
};

// Shared-memory, cluster-address and mbarrier helpers (inline PTX).
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cluster_addr(unsigned local, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Store two floats into (possibly another CTA's) shared memory and count
// 8 bytes on that CTA's mbarrier when they land.
__device__ __forceinline__ void st_async_f2(unsigned raddr, float a, float b, unsigned rmbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(a), "f"(b), "r"(rmbar)
                 : "memory");
}

// Wall-time bound of one mbarrier wait (%globaltimer, ns).  A wait that gives
// up sets error bit 4, reported as LBM_ETIMEOUT, and the kernel carries on
// without blocking.  The bound is on time, not on polls: try_wait may
// suspend the thread for a while.
constexpr unsigned long long kWaitNs = 2000000000ull;
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try_wait_cta(unsigned mbar, unsigned parity);
// Bounded wait for the phase of the given parity (cluster scope when remote
// st.async bytes count on the barrier); false when it gave up.
__device__ __forceinline__ bool wait_bounded(unsigned mbar, unsigned parity, bool cluster_scope,
                                             unsigned long long limit_ns) {
    auto poll = [&]() { return cluster_scope ? mbar_try_wait(mbar, parity) : mbar_try_wait_cta(mbar, parity); };
    if (poll()) return true;
    const unsigned long long t0 = now_ns();
    while (!poll())
        if (now_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void mbar_arrive(unsigned mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

template <int TX, int CY>
struct FastLayout {
    static constexpr int RW = TX + 2;            // ring row width (x halo columns -1, TX)
    static constexpr int HN = 2 * TX / CY;       // outer-halo nodes pulled per CTA
    // Density ring slots.  Plane p lives in slot p mod S.  The rows beyond
    // the cluster are written by every CTA of the cluster, and a CTA can run
    // at most CY - 1 planes ahead of the edge CTA it writes to, so S = CY + 2
    // slots keep a slot's next plane from landing before its last reader.
    static constexpr int S = CY + 2;
    static constexpr int RING = S * 3 * RW * 2;  // [slot][row -1..1][col][component]
    static constexpr unsigned TX_BYTES = 2u * TX * 2u * 4u;  // rows -1 and +1, both components
    static constexpr size_t bytes = sizeof(float) * RING + sizeof(unsigned long long) * S;
};

// Pulled population (s, i) of the node whose (s=0, i=0) element index is b.
// The first read of a plane keeps its lines in L2 (evict_last policy) for the
// second read one plane later, which marks them last-use.
__device__ __forceinline__ const float* pulled_ptr(const float* src, const Layout& L, long long b, int s, int i) {
    return src + b + (long long)(s * 19 + i) * L.array -
           ((long long)cz_(i) * L.plane + (long long)cy_(i) * L.pitch + cx_(i));
}
__device__ __forceinline__ float ld_keep(const float* p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float pulled(const float* __restrict__ src, const Layout& L, long long b, int s, int i,
                                        unsigned long long pol) {
    return ld_keep(pulled_ptr(src, L, b, s, i), pol);
}
__device__ __forceinline__ float pulled_last(const float* __restrict__ src, const Layout& L, long long b, int s, int i) {
    return __ldlu(pulled_ptr(src, L, b, s, i));
}

// 16-bit deviation storage: the word of the deviation pair {A, B} of
// direction i pulled into the node whose first word (i = 1) has index b, and
// the node's own float4 block {rho*_A, rho*_B, f*_0A, f*_0B}.
__device__ __forceinline__ const unsigned* dev_ptr(const unsigned* src, const Layout& L, long long b, int i) {
    return src + b + (long long)(i - 1) * L.array -
           ((long long)cz_(i) * (L.plane >> 1) + (long long)cy_(i) * L.pitch + cx_(i));
}
__device__ __forceinline__ unsigned ld_keep_u32(const unsigned* p, unsigned long long pol) {
    unsigned v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_keep_f4(const float4* p, unsigned long long pol) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

// ---- TMA-staged variant: bulk copies of whole pulled rows into shared memory ----

// Bulk copy of `bytes` (a multiple of 16) from a 16-byte aligned global
// address to this CTA's shared memory, counted on the CTA's mbarrier.
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
// Order this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait_cta(unsigned mbar, unsigned parity) {
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

// Shared-memory image of one plane of one row for the staged variant: every
// array the row's pulled populations come from, as a row segment that starts
// at x = -4 (16-byte aligned) and covers x - c_ix for every x of the row.
// Each source row is y - c_iy of plane p - c_iz, so over the grid every
// population row is copied exactly once.
template <int TX, typename ST>
struct StagePlane;

template <int TX>
struct StagePlane<TX, float> {
    static constexpr int SEG = TX + 8;  // floats per segment, x = -4 .. TX + 3
    static constexpr unsigned BYTES = 38u * SEG * 4u;
    static __device__ __forceinline__ void issue(const float* src, const Layout& L, int y, int p, unsigned dst,
                                                 unsigned mbar) {
#pragma unroll
        for (int a = 0; a < 38; ++a) {
            const int s = a / 19, i = a % 19;
            bulk_g2s(dst + 4u * SEG * a, src + L.at(s, i, -4, y - cy_(i), p - cz_(i)), 4u * SEG, mbar);
        }
    }
    static __device__ __forceinline__ void densities(const float* st, int x, float& ra, float& rb) {
        ra = st[x + 4];
        rb = st[19 * SEG + x + 4];
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            ra += st[i * SEG + x - cx_(i) + 4] + st[(i + 1) * SEG + x - cx_(i + 1) + 4];
            rb += st[(19 + i) * SEG + x - cx_(i) + 4] + st[(20 + i) * SEG + x - cx_(i + 1) + 4];
        }
    }
    static __device__ __forceinline__ void populations(const float* st, int x, float (&f)[2][19]) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 19; ++i) f[s][i] = st[(s * 19 + i) * SEG + x - cx_(i) + 4];
    }
};

template <int TX, typename T>
struct StagePlane<TX, Dev<T>> {
    static constexpr int SEG = TX + 8;  // words per deviation segment, x = -4 .. TX + 3
    static constexpr unsigned NODE_BYTES = 16u * TX;
    static constexpr unsigned BYTES = NODE_BYTES + 18u * SEG * 4u;
    static __device__ __forceinline__ void issue(const Dev<T>* src, const Layout& L, int y, int p, unsigned dst,
                                                 unsigned mbar) {
        bulk_g2s(dst, reinterpret_cast<const float4*>(src) + L.dev_node(0, y, p), NODE_BYTES, mbar);
        const unsigned* w = reinterpret_cast<const unsigned*>(src);
#pragma unroll
        for (int i = 1; i < 19; ++i)
            bulk_g2s(dst + NODE_BYTES + 4u * SEG * (i - 1), w + L.dev_word(i, -4, y - cy_(i), p - cz_(i)), 4u * SEG,
                     mbar);
    }
    static __device__ __forceinline__ const unsigned* words(const float* st) {
        return reinterpret_cast<const unsigned*>(reinterpret_cast<const char*>(st) + NODE_BYTES);
    }
    static __device__ __forceinline__ void densities(const float* st, int x, float& ra, float& rb) {
        const float4 o = reinterpret_cast<const float4*>(st)[x];
        const unsigned* w = words(st);
        float da = 0.f, db = 0.f;
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float2 u = dev_unpack2<T>(w[(i - 1) * SEG + x - cx_(i) + 4]);
            const float2 v = dev_unpack2<T>(w[i * SEG + x - cx_(i + 1) + 4]);
            da += u.x + v.x;
            db += u.y + v.y;
        }
        ra = o.z + (1.f - wgt<float>(0)) * o.x + da;
        rb = o.w + (1.f - wgt<float>(0)) * o.y + db;
    }
    static __device__ __forceinline__ void populations(const float* st, int x, float (&f)[2][19]) {
        const float4 o = reinterpret_cast<const float4*>(st)[x];
        const unsigned* w = words(st);
        f[0][0] = o.z;
        f[1][0] = o.w;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const float2 v = dev_unpack2<T>(w[(i - 1) * SEG + x - cx_(i) + 4]);
            f[0][i] = wgt<float>(i) * o.x + v.x;
            f[1][i] = wgt<float>(i) * o.y + v.y;
        }
    }
};

// Storage-specific reads and writes of the row kernel.  A node is named by
// its plane-0 indices (NodeIx); plane p adds p planes.
struct NodeIx {
    long long a;  // float32: element of (s=0, i=0); deviations: float4 block index
    long long b;  // deviations: 2-byte index of deviation (s=0, i=1)
};

template <typename S>
struct RowIO;

template <>
struct RowIO<float> {
    static __device__ __forceinline__ NodeIx node(const Layout& L, int x, int y) { return {L.at(0, 0, x, y, 0), 0}; }
    // post-streaming densities of the node at plane p (first read, kept in L2)
    static __device__ __forceinline__ void densities(const float* __restrict__ src, const Layout& L, NodeIx n, int p,
                                                     unsigned long long keep, float& ra, float& rb) {
        const long long b = n.a + (long long)p * L.plane;
        ra = pulled(src, L, b, 0, 0, keep);
        rb = pulled(src, L, b, 1, 0, keep);
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            ra += pulled(src, L, b, 0, i, keep) + pulled(src, L, b, 0, i + 1, keep);
            rb += pulled(src, L, b, 1, i, keep) + pulled(src, L, b, 1, i + 1, keep);
        }
    }
    // the node's 38 pulled populations at plane p (second read, last use)
    static __device__ __forceinline__ void populations(const float* __restrict__ src, const Layout& L, NodeIx n, int p,
                                                       float (&f)[2][19]) {
        const long long b = n.a + (long long)p * L.plane;
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 19; ++i) f[s][i] = pulled_last(src, L, b, s, i);
    }
    // one read of the 38 pulled populations and the densities summed from
    // them in the order of densities() (the warp-specialised kernel)
    static __device__ __forceinline__ void load_all(const float* __restrict__ src, const Layout& L, NodeIx n, int p,
                                                    float (&f)[2][19], float& ra, float& rb) {
        populations(src, L, n, p, f);
        ra = f[0][0];
        rb = f[1][0];
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            ra += f[0][i] + f[0][i + 1];
            rb += f[1][i] + f[1][i + 1];
        }
    }
};

template <typename T>
struct RowIO<Dev<T>> {
    static __device__ __forceinline__ NodeIx node(const Layout& L, int x, int y) {
        return {L.dev_node(x, y, 0), L.dev_word(1, x, y, 0)};
    }
    static __device__ __forceinline__ void densities(const Dev<T>* __restrict__ src, const Layout& L, NodeIx n, int p,
                                                     unsigned long long keep, float& ra, float& rb) {
        const float4 o = ld_keep_f4(reinterpret_cast<const float4*>(src) + n.a + (long long)p * (L.plane >> 3), keep);
        const unsigned* d = reinterpret_cast<const unsigned*>(src);
        const long long b = n.b + (long long)p * (L.plane >> 1);
        // sum_i (w_i rho* + d_i) + f*_0 = f*_0 + (1 - w_0) rho* + sum_i d_i
        float da = 0.f, db = 0.f;
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float2 u = dev_unpack2<T>(ld_keep_u32(dev_ptr(d, L, b, i), keep));
            const float2 v = dev_unpack2<T>(ld_keep_u32(dev_ptr(d, L, b, i + 1), keep));
            da += u.x + v.x;
            db += u.y + v.y;
        }
        ra = o.z + (1.f - wgt<float>(0)) * o.x + da;
        rb = o.w + (1.f - wgt<float>(0)) * o.y + db;
    }
    static __device__ __forceinline__ void populations(const Dev<T>* __restrict__ src, const Layout& L, NodeIx n, int p,
                                                       float (&f)[2][19]) {
        const float4 o = __ldlu(reinterpret_cast<const float4*>(src) + n.a + (long long)p * (L.plane >> 3));
        const unsigned* d = reinterpret_cast<const unsigned*>(src);
        const long long b = n.b + (long long)p * (L.plane >> 1);
        f[0][0] = o.z;
        f[1][0] = o.w;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const float2 v = dev_unpack2<T>(__ldlu(dev_ptr(d, L, b, i)));
            f[0][i] = wgt<float>(i) * o.x + v.x;
            f[1][i] = wgt<float>(i) * o.y + v.y;
        }
    }
    // one read of the block and the 18 pulled words: the populations of
    // populations() and the densities of densities(), with their arithmetic
    static __device__ __forceinline__ void load_all(const Dev<T>* __restrict__ src, const Layout& L, NodeIx n, int p,
                                                    float (&f)[2][19], float& ra, float& rb) {
        const float4 o = __ldlu(reinterpret_cast<const float4*>(src) + n.a + (long long)p * (L.plane >> 3));
        const unsigned* d = reinterpret_cast<const unsigned*>(src);
        const long long b = n.b + (long long)p * (L.plane >> 1);
        f[0][0] = o.z;
        f[1][0] = o.w;
        float da = 0.f, db = 0.f;
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float2 u = dev_unpack2<T>(__ldlu(dev_ptr(d, L, b, i)));
            const float2 v = dev_unpack2<T>(__ldlu(dev_ptr(d, L, b, i + 1)));
            da += u.x + v.x;
            db += u.y + v.y;
            f[0][i] = wgt<float>(i) * o.x + u.x;
            f[1][i] = wgt<float>(i) * o.y + u.y;
            f[0][i + 1] = wgt<float>(i + 1) * o.x + v.x;
            f[1][i + 1] = wgt<float>(i + 1) * o.y + v.y;
        }
        ra = o.z + (1.f - wgt<float>(0)) * o.x + da;
        rb = o.w + (1.f - wgt<float>(0)) * o.y + db;
    }
};

// Shared memory of the staged variant beyond the density ring: NST stage
// mbarriers, then (128-byte aligned) NST plane images.
template <int TX, int CY, typename ST>
struct StagedLayout {
    static constexpr int NST = 3;  // planes z+1 (resident), z+2 and z+3 (in flight)
    static constexpr size_t mbar_off = FastLayout<TX, CY>::bytes;
    static constexpr size_t stage_off = ((mbar_off + 8 * NST + 127) / 128) * 128;
    static constexpr size_t bytes = stage_off + (size_t)NST * StagePlane<TX, ST>::BYTES;
};

// Collision of node (x, y, z) from its 38 pulled populations f and the
// density ring (slots s0, s1, s2 hold planes z - 1, z, z + 1; row 0 is this
// CTA's row, rows -1 / +1 its neighbours, columns -1 and TX the x halo):
// momentum (Eq. 6), Shan-Chen force (Eq. 7), common velocity with the force
// shift, BGK relaxation to the equilibrium of Eq. 8 (Eqs. 9, 10) -- or, with
// MRT (float32 storage), the moment relaxation of the generic kernel -- and
// the store of the post-collision state (float32 populations with the rest
// population closing the mass balance, or 16-bit deviations).  Also
// accumulates the centre-of-mass partials of the droplet phase and flags
// non-finite densities.  Shared by the row kernels so that every variant
// computes bit-identical states.
template <int TX, typename ST, bool MRT = false>
__device__ __forceinline__ void collide_node(const float* ring, int s0, int s1, int s2, int x, int y, int z,
                                             const float (&f)[2][19], const FastModel& m, const Layout& L,
                                             ST* __restrict__ dst, int* __restrict__ d_err, float (&cm)[4], float px,
                                             float py) {
    constexpr int RW = TX + 2;
    auto ridx = [&](int slot, int row, int col) { return ((slot * 3 + row + 1) * RW + col + 1) * 2; };
    // neighbour density of component s at offset (dx, dy, dz)
    auto nb = [&](int s, int dx, int dy, int dz) -> float {
        const int slot = dz == 0 ? s1 : (dz > 0 ? s2 : s0);
        return ring[ridx(slot, dy, x + dx) + s];
    };
    const float rho[2] = {ring[ridx(s1, 0, x)], ring[ridx(s1, 0, x) + 1]};
    // momentum (Eq. 6), opposite pairs differenced first
    float j[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float d = f[s][i] - f[s][i + 1];
            if (cx_(i)) jx += (float)cx_(i) * d;
            if (cy_(i)) jy += (float)cy_(i) * d;
            if (cz_(i)) jz += (float)cz_(i) * d;
        }
        j[s][0] = jx; j[s][1] = jy; j[s][2] = jz;
    }
    // Shan-Chen force (Eq. 7) sums, neighbour pairs differenced first
    float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float d = wgt<float>(i) * (nb(s, cx_(i), cy_(i), cz_(i)) - nb(s, -cx_(i), -cy_(i), -cz_(i)));
            if (cx_(i)) acc[s][0] += (float)cx_(i) * d;
            if (cy_(i)) acc[s][1] += (float)cy_(i) * d;
            if (cz_(i)) acc[s][2] += (float)cz_(i) * d;
        }
    }
    const float den = rho[0] * m.inv_tau[0] + rho[1] * m.inv_tau[1];
    float up[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) up[a] = (j[0][a] * m.inv_tau[0] + j[1][a] * m.inv_tau[1]) / den;
    if (!(isfinite(rho[0]) && isfinite(rho[1]))) atomicOr(d_err, 1);
    {
        const float phi = (rho[0] - rho[1]) / (rho[0] + rho[1]);
        const float w = phi > 0.f ? phi : 0.f;
        cm[0] += w;
        cm[1] += w * px;
        cm[2] += w * py;
        cm[3] += w * ((float)z - 0.5f * (float)(L.Lz - 1));
    }
    if constexpr (is_dev_t<ST>::value) {
        // 16-bit deviations from w_i times the density of the node each
        // population streams to (this CTA's density planes), the pair of
        // components of one direction in one word
        using T = decltype(dev_tag(ST{}));
        float ux[2], uy[2], uz[2], u2x[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float sh = -m.G * m.tau[s];  // tau_s F^s / rho_s per unit of the other sum
            ux[s] = up[0] + sh * acc[1 - s][0];
            uy[s] = up[1] + sh * acc[1 - s][1];
            uz[s] = up[2] + sh * acc[1 - s][2];
            u2x[s] = 1.5f * (ux[s] * ux[s] + uy[s] * uy[s] + uz[s] * uz[s]);
        }
        unsigned* d = reinterpret_cast<unsigned*>(dst);
        const long long db = L.dev_word(1, x, y, z);
        float others[2] = {0.f, 0.f};
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            float da[2], dbv[2], refa[2], refb[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float cu = (float)cx_(i) * ux[s] + (float)cy_(i) * uy[s] + (float)cz_(i) * uz[s];
                const float rw = rho[s] * wgt<float>(i);
                const float even = rw * (1.f + 4.5f * cu * cu - u2x[s]);
                const float odd = rw * (3.f * cu);
                const float fa = f[s][i], fb = f[s][i + 1];
                const float oa = fa - (fa - (even + odd)) * m.inv_tau[s];
                const float ob = fb - (fb - (even - odd)) * m.inv_tau[s];
                refa[s] = wgt<float>(i) * nb(s, cx_(i), cy_(i), cz_(i));
                refb[s] = wgt<float>(i) * nb(s, -cx_(i), -cy_(i), -cz_(i));
                da[s] = oa - refa[s];
                dbv[s] = ob - refb[s];
            }
            const unsigned wa = dev_pack2<T>(da[0], da[1]), wb = dev_pack2<T>(dbv[0], dbv[1]);
            __stcs(d + db + (long long)(i - 1) * L.array, wa);
            __stcs(d + db + (long long)i * L.array, wb);
            // the values the readers will rebuild, for the mass balance
            const float2 qa = dev_unpack2<T>(wa), qb = dev_unpack2<T>(wb);
            others[0] += (refa[0] + qa.x) + (refb[0] + qb.x);
            others[1] += (refa[1] + qa.y) + (refb[1] + qb.y);
        }
        __stcs(reinterpret_cast<float4*>(dst) + L.dev_node(x, y, z),
               make_float4(rho[0], rho[1], rho[0] - others[0], rho[1] - others[1]));
    } else {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float sh = -m.G * m.tau[s];  // tau_s F^s / rho_s per unit of the other sum
            const float ux = up[0] + sh * acc[1 - s][0];
            const float uy = up[1] + sh * acc[1 - s][1];
            const float uz = up[2] + sh * acc[1 - s][2];
            const float u2x = 1.5f * (ux * ux + uy * uy + uz * uz);
            const float it = m.inv_tau[s];
            const float r = rho[s];
            // moving populations; the rest population then closes the mass
            // balance exactly (sum of outputs = rho), which keeps fp32
            // rounding from drifting the interface
            const long long b = L.at(s, 0, x, y, z);
            float others = 0.f;
            if constexpr (MRT) {
                // MRT: relax the moments of the deviation from equilibrium
                // (d'Humieres basis; momentum and stress at 1/tau)
                float dv[19], out[19];
#pragma unroll
                for (int i = 0; i < 19; ++i) dv[i] = f[s][i] - feq<float>(i, r, ux, uy, uz, u2x);
                mrt_relax<float>(f[s], dv, it, m.mrt, out);
#pragma unroll
                for (int i = 1; i < 19; i += 2) {
                    __stcs(dst + b + (long long)i * L.array, out[i]);
                    __stcs(dst + b + (long long)(i + 1) * L.array, out[i + 1]);
                    others += out[i] + out[i + 1];
                }
            } else {
#pragma unroll
                for (int i = 1; i < 19; i += 2) {
                    const float cu = (float)cx_(i) * ux + (float)cy_(i) * uy + (float)cz_(i) * uz;
                    const float rw = r * wgt<float>(i);
                    const float even = rw * (1.f + 4.5f * cu * cu - u2x);
                    const float odd = rw * (3.f * cu);
                    const float fa = f[s][i], fb = f[s][i + 1];
                    const float oa = fa - (fa - (even + odd)) * it;
                    const float ob = fb - (fb - (even - odd)) * it;
                    __stcs(dst + b + (long long)i * L.array, oa);
                    __stcs(dst + b + (long long)(i + 1) * L.array, ob);
                    others += oa + ob;
                }
            }
            __stcs(dst + b, r - others);
        }
    }
}

template <int TX, int CY, int MINB, typename ST, bool STAGED, bool MRT = false>
__global__ void __launch_bounds__(TX, MINB)
    k_stream_collide_rows(const ST* __restrict__ src, ST* __restrict__ dst, Layout L, FastModel m, int zchunk,
                          CentreParts cp, int* __restrict__ d_err) {
    using IO = RowIO<ST>;
    using FL = FastLayout<TX, CY>;
    using SP = StagePlane<TX, ST>;
    using SL = StagedLayout<TX, CY, ST>;
    constexpr int RW = FL::RW, HN = FL::HN, S = FL::S, NST = SL::NST;
    extern __shared__ __align__(128) float ring[];  // [S][3][RW][2], then S mbarriers (staged: see StagedLayout)
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(ring + FL::RING);
    __shared__ double red[4 * ((TX + 31) / 32)];

    cg::cluster_group cluster = cg::this_cluster();
    const int x = threadIdx.x;
    const int y = blockIdx.y;
    const int rank = (int)cluster.block_rank();  // == y % CY for cluster dims (1, CY, 1)
    const int Y0 = y - rank;
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, L.Lz);

    // Outer-halo node handled by this thread (threads x < HN): the first half
    // of them cover row Y0 - 1 (kept in rank 0's ring row -1), the second half
    // row Y0 + CY (kept in rank CY-1's ring row +1), TX/CY columns per CTA.
    const bool hthr = x < HN;
    const int hside = x < HN / 2 ? 0 : 1;
    const int hcol = rank * (HN / 2) + (x % (HN / 2));
    const int hy = hside ? Y0 + CY : Y0 - 1;
    const bool hin = hy >= 0 && hy < L.Ly;

    // ring index of (slot, row in -1..1, col in -1..TX), component 0
    auto ridx = [&](int slot, int row, int col) { return ((slot * 3 + row + 1) * RW + col + 1) * 2; };
    const unsigned ring_s = smem_u32(ring);
    const unsigned mbar_s = smem_u32(mbar);
    // Where this CTA's own row goes in the neighbours' rings, and where its
    // outer-halo node goes in the edge CTA's ring (cluster addresses).
    const unsigned below_ring = rank > 0 ? cluster_addr(ring_s, rank - 1) : 0u;  // their row +1
    const unsigned below_mbar = rank > 0 ? cluster_addr(mbar_s, rank - 1) : 0u;
    const unsigned above_ring = rank < CY - 1 ? cluster_addr(ring_s, rank + 1) : 0u;  // their row -1
    const unsigned above_mbar = rank < CY - 1 ? cluster_addr(mbar_s, rank + 1) : 0u;
    const unsigned halo_ring = cluster_addr(ring_s, hside ? CY - 1 : 0);
    const unsigned halo_mbar = cluster_addr(mbar_s, hside ? CY - 1 : 0);

    // staged variant: plane images and their mbarriers (one arrival, by
    // thread 0, plus the bytes of the copies)
    const unsigned smbar_s = smem_u32(ring) + (unsigned)SL::mbar_off;
    const unsigned stage_s = smem_u32(ring) + (unsigned)SL::stage_off;
    const float* stage = reinterpret_cast<const float*>(reinterpret_cast<const char*>(ring) + SL::stage_off);

    // ghost density in every slot (x halo columns keep it for good), barriers
    for (int e = x; e < FL::RING; e += TX) ring[e] = m.rho_b[e & 1];
    if (x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(mbar_s + 8u * k, 1u);
        if constexpr (STAGED)
            for (int k = 0; k < NST; ++k) mbar_init(smbar_s + 8u * k, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();  // barriers initialised before any remote store arrives

    const NodeIx node0 = IO::node(L, x, y);
    const NodeIx hnode0 = IO::node(L, hcol, hin ? hy : 0);
    unsigned long long keep;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));

    auto slot_of = [&](int p) { return (p - (zc0 - 1)) % S; };

    // Staged variant: plane p of this row lives in stage (p - zc0 + 1) mod NST.
    // Thread 0 fills a stage (expect_tx, then the copies); every thread waits
    // on the stage's mbarrier (bounded) before its first read of the plane.
    // Only the planes this chunk reads and that lie in the box are copied.
    auto stage_of = [&](int p) { return (p - zc0 + 1) % NST; };
    auto plane_wanted = [&](int p) { return p >= 0 && p < L.Lz && p >= zc0 - 1 && p <= zc1; };
    unsigned sphase = 0u;   // bit k: parity of stage k's next completion (every thread)
    unsigned pending = 0u;  // thread 0: stages with copies it has not seen complete
    auto fill = [&](int p) {
        if (!plane_wanted(p)) return;
        const int k = stage_of(p);
        mbar_expect_tx(smbar_s + 8u * k, SP::BYTES);
        SP::issue(src, L, y, p, stage_s + (unsigned)(k * SP::BYTES), smbar_s + 8u * k);
        pending |= 1u << k;
    };
    auto stage_wait = [&](int p) {
        const int k = stage_of(p);
        const unsigned par = (sphase >> k) & 1u;
        if (wait_bounded(smbar_s + 8u * k, par, false, kWaitNs)) pending &= ~(1u << k);
        else atomicOr(d_err, 4);
        sphase ^= 1u << k;
    };
    auto stage_ptr = [&](int p) { return stage + (size_t)stage_of(p) * (SP::BYTES / 4); };
    if constexpr (STAGED) {
        if (x == 0)
            for (int q = -1; q <= 1; ++q) fill(zc0 + q);
    }

    // Post-streaming densities of plane p: the own node into row 0 of this
    // CTA's ring and into the neighbours' rows -1 / +1; the outer-halo node
    // (threads x < HN) into the edge CTA's row -1 / +1.  Ghost densities
    // outside the box.  Every CTA then expects TX_BYTES on its slot barrier.
    auto densities = [&](int p) {
        const int slot = slot_of(p);
        const bool in = p >= 0 && p < L.Lz;
        float ra = m.rho_b[0], rb = m.rho_b[1];
        if (in) {
            if constexpr (STAGED) {
                stage_wait(p);
                SP::densities(stage_ptr(p), x, ra, rb);
            } else {
                IO::densities(src, L, node0, p, keep, ra, rb);
            }
        }
        *reinterpret_cast<float2*>(ring + ridx(slot, 0, x)) = make_float2(ra, rb);
        const unsigned mb = 8u * slot;
        if (rank > 0) st_async_f2(below_ring + 4u * ridx(slot, 1, x), ra, rb, below_mbar + mb);
        if (rank < CY - 1) st_async_f2(above_ring + 4u * ridx(slot, -1, x), ra, rb, above_mbar + mb);
        if (hthr) {
            float ha = m.rho_b[0], hb = m.rho_b[1];
            if (in && hin) IO::densities(src, L, hnode0, p, keep, ha, hb);
            st_async_f2(halo_ring + 4u * ridx(slot, hside ? 1 : -1, hcol), ha, hb, halo_mbar + mb);
        }
        if (x == 0) mbar_expect_tx(mbar_s + mb, FL::TX_BYTES);
    };
    // Wait (bounded) until the neighbour rows of plane p have landed.
    unsigned phase = 0u;  // bit k: parity of slot k's next phase
    auto wait_rows = [&](int p) {
        const int slot = slot_of(p);
        const unsigned par = (phase >> slot) & 1u;
        if (!wait_bounded(mbar_s + 8u * slot, par, true, kWaitNs)) atomicOr(d_err, 4);
        phase ^= 1u << slot;
    };

    float cm[4] = {0.f, 0.f, 0.f, 0.f};
    const float px = (float)x - 0.5f * (float)(L.Lx - 1), py = (float)y - 0.5f * (float)(L.Ly - 1);

    densities(zc0 - 1);
    densities(zc0);
    wait_rows(zc0 - 1);
    wait_rows(zc0);
    if constexpr (STAGED) {
        __syncthreads();  // plane zc0 - 1 read by all: its stage takes plane zc0 + 2
        if (x == 0) {
            fence_proxy_async();
            fill(zc0 + 2);
        }
    }
    for (int z = zc0; z < zc1; ++z) {
        densities(z + 1);
        // this node's populations for the collision, read while the
        // neighbour rows of plane z + 1 are in flight
        float f[2][19];
        if constexpr (STAGED) SP::populations(stage_ptr(z), x, f);
        else IO::populations(src, L, node0, z, f);
        __syncthreads();  // own row of plane z + 1 complete
        if constexpr (STAGED) {
            // plane z has been read by every thread: its stage takes plane z + 3
            if (x == 0) {
                fence_proxy_async();
                fill(z + 3);
            }
        }
        wait_rows(z + 1);

        collide_node<TX, ST, MRT>(ring, slot_of(z - 1), slot_of(z), slot_of(z + 1), x, y, z, f, m, L, dst, d_err, cm,
                                  px, py);
        // Before a later plane reuses this plane's own-row slot, all threads
        // must be done reading it: the __syncthreads of the next iterations
        // (S > 3 planes apart) order that.
    }
    // staged variant: copies whose completion thread 0 did not observe (a
    // wait that gave up) are waited for again, bounded, before the CTA exits
    if constexpr (STAGED) {
        if (x == 0) {
            for (int k = 0; k < NST; ++k) {
                if (!((pending >> k) & 1u)) continue;
                wait_bounded(smbar_s + 8u * k, ((sphase >> k) & 1u) ^ 1u, false, kWaitNs);
            }
        }
    }
    // no CTA leaves while another may still address its shared memory
    cluster.sync();

    // centre-of-mass partials of the written state (fixed-order reduction)
    double cmd[4] = {(double)cm[0], (double)cm[1], (double)cm[2], (double)cm[3]};
    centre_epilogue(cmd, cp, red);
}

// ---- Warp-specialised variant: loader and collider threads per row ----
//
// A CTA of 2 TX threads owns one row: threads 0 .. TX-1 (loaders) and
// TX .. 2 TX-1 (colliders) each take node x = t mod TX.  Per plane p a loader
// reads the node's 38 pulled populations once, sums its densities into the
// ring (own row, the neighbour CTAs' rows by st.async, the outer-halo node as
// in the direct variant) and stages the populations in shared memory (NP
// planes in flight); the colliders collide plane z from shared memory once
// the densities of plane z + 1 have landed.  Loads of later planes are in
// flight while earlier planes are collided, on other warps, and no
// population is read twice.
//
// Barriers (all waits bounded): ring slot k completes when this CTA's TX
// loaders have written their own row of the slot's plane and the 2 TX x 8
// bytes of the rows -1 / +1 have landed; full[b] when the loaders have staged
// a plane in buffer b; empty[b] when the colliders are done with it.
//
// Ring slots: a loader pushes plane p's densities only after it has staged
// plane p - 1, which waited for its colliders to be done with plane
// p - 1 - NP = p - 3; those colliders finished plane p - 3 only after the CTAs
// next to them had pushed plane p - 2.  So a loader is at most two planes
// ahead of the loaders of the CTAs next to it in the cluster and at most
// 2 (CY - 1) planes ahead of any CTA of the cluster (the outer-halo rows go
// from every CTA to the edge CTAs), whose colliders may still be reading
// three planes behind that CTA's own loader: S = 2 CY + 2 slots.
template <int TX, int CY>
struct WsLayout {
    static constexpr int RW = TX + 2;
    static constexpr int HN = 2 * TX / CY;
    static constexpr int S = 2 * CY + 2;
    static constexpr int NP = 2;
    static constexpr int RING = S * 3 * RW * 2;  // [slot][row -1..1][col][component] floats
    static constexpr int POPS = NP * 38 * TX;    // [buffer][s * 19 + i][x] floats
    static constexpr unsigned TX_BYTES = 2u * TX * 2u * 4u;
    static constexpr int NBAR = S + 2 * NP;
    static constexpr size_t bytes = sizeof(float) * (RING + POPS) + sizeof(unsigned long long) * NBAR;
};

__device__ __forceinline__ bool ws_wait(unsigned mbar, unsigned parity, bool cluster_scope) {
    return wait_bounded(mbar, parity, cluster_scope, kWaitNs);
}

template <int TX, int CY, int MINB, typename ST>
__global__ void __launch_bounds__(2 * TX, MINB)
    k_stream_collide_ws(const ST* __restrict__ src, ST* __restrict__ dst, Layout L, FastModel m, int zchunk,
                        CentreParts cp, int* __restrict__ d_err) {
    using IO = RowIO<ST>;
    using WL = WsLayout<TX, CY>;
    constexpr int RW = WL::RW, HN = WL::HN, S = WL::S, NP = WL::NP;
    extern __shared__ __align__(128) float ring[];  // [S][3][RW][2], then [NP][38][TX], then NBAR mbarriers
    float* pops = ring + WL::RING;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(pops + WL::POPS);
    __shared__ double red[4 * ((2 * TX + 31) / 32)];

    cg::cluster_group cluster = cg::this_cluster();
    const int t = threadIdx.x;
    const bool loader = t < TX;
    const int x = loader ? t : t - TX;
    const int y = blockIdx.y;
    const int rank = (int)cluster.block_rank();  // == y % CY for cluster dims (1, CY, 1)
    const int Y0 = y - rank;
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, L.Lz);

    // outer-halo node of loader threads x < HN (as in the direct variant)
    const bool hthr = loader && x < HN;
    const int hside = x < HN / 2 ? 0 : 1;
    const int hcol = rank * (HN / 2) + (x % (HN / 2));
    const int hy = hside ? Y0 + CY : Y0 - 1;
    const bool hin = hy >= 0 && hy < L.Ly;

    auto ridx = [&](int slot, int row, int col) { return ((slot * 3 + row + 1) * RW + col + 1) * 2; };
    const unsigned ring_s = smem_u32(ring);
    const unsigned rbar_s = smem_u32(bars);        // S ring-slot barriers
    const unsigned full_s = rbar_s + 8u * S;       // NP: a plane staged
    const unsigned empty_s = full_s + 8u * NP;     // NP: a staged plane read
    const unsigned below_ring = rank > 0 ? cluster_addr(ring_s, rank - 1) : 0u;  // their row +1
    const unsigned below_mbar = rank > 0 ? cluster_addr(rbar_s, rank - 1) : 0u;
    const unsigned above_ring = rank < CY - 1 ? cluster_addr(ring_s, rank + 1) : 0u;  // their row -1
    const unsigned above_mbar = rank < CY - 1 ? cluster_addr(rbar_s, rank + 1) : 0u;
    const unsigned halo_ring = cluster_addr(ring_s, hside ? CY - 1 : 0);
    const unsigned halo_mbar = cluster_addr(rbar_s, hside ? CY - 1 : 0);

    for (int e = t; e < WL::RING; e += 2 * TX) ring[e] = m.rho_b[e & 1];  // ghost density, x halo columns for good
    if (t == 0) {
        for (int k = 0; k < S; ++k) mbar_init(rbar_s + 8u * k, (unsigned)TX);
        for (int b = 0; b < NP; ++b) {
            mbar_init(full_s + 8u * b, (unsigned)TX);
            mbar_init(empty_s + 8u * b, (unsigned)TX);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();  // barriers initialised before any remote store arrives

    auto slot_of = [&](int p) { return (p - (zc0 - 1)) % S; };
    float cm[4] = {0.f, 0.f, 0.f, 0.f};

    if (loader) {
        const NodeIx node0 = IO::node(L, x, y);
        const NodeIx hnode0 = IO::node(L, hcol, hin ? hy : 0);
        unsigned long long keep;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        unsigned ephase = 0u;  // bit b: parity of empty[b]'s next phase
        for (int p = zc0 - 1; p <= zc1; ++p) {
            const bool in = p >= 0 && p < L.Lz;
            const bool staged = p >= zc0 && p < zc1;  // a plane this CTA collides
            float f[2][19];
            float ra = m.rho_b[0], rb = m.rho_b[1];
            if (in) IO::load_all(src, L, node0, p, f, ra, rb);
            float ha = m.rho_b[0], hb = m.rho_b[1];
            if (hthr && in && hin) IO::densities(src, L, hnode0, p, keep, ha, hb);  // read again by its own CTA
            // densities first: the colliders of plane p - 1 wait for them
            const int slot = slot_of(p);
            const unsigned mb = 8u * slot;
            *reinterpret_cast<float2*>(ring + ridx(slot, 0, x)) = make_float2(ra, rb);
            if (rank > 0) st_async_f2(below_ring + 4u * ridx(slot, 1, x), ra, rb, below_mbar + mb);
            if (rank < CY - 1) st_async_f2(above_ring + 4u * ridx(slot, -1, x), ra, rb, above_mbar + mb);
            if (hthr) st_async_f2(halo_ring + 4u * ridx(slot, hside ? 1 : -1, hcol), ha, hb, halo_mbar + mb);
            if (x == 0) mbar_expect_tx(rbar_s + mb, WL::TX_BYTES);  // this thread's arrival, and the bytes
            else mbar_arrive(rbar_s + mb);
            // then the populations, into a buffer the colliders are done with
            // (plane p - NP); they wait in registers meanwhile
            if (staged) {
                const int b = (p - zc0) % NP;
                if (p - zc0 >= NP) {
                    if (!ws_wait(empty_s + 8u * b, (ephase >> b) & 1u, false)) atomicOr(d_err, 4);
                    ephase ^= 1u << b;
                }
                float* P = pops + (size_t)b * 38 * TX;
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int i = 0; i < 19; ++i) P[(s * 19 + i) * TX + x] = f[s][i];
                mbar_arrive(full_s + 8u * b);
            }
        }
    } else {
        const float px = (float)x - 0.5f * (float)(L.Lx - 1), py = (float)y - 0.5f * (float)(L.Ly - 1);
        unsigned rphase = 0u, fphase = 0u;  // bit k: parity of ring slot k's / full[k]'s next phase
        auto wait_ring = [&](int p) {
            const int slot = slot_of(p);
            if (!ws_wait(rbar_s + 8u * slot, (rphase >> slot) & 1u, true)) atomicOr(d_err, 4);
            rphase ^= 1u << slot;
        };
        wait_ring(zc0 - 1);
        wait_ring(zc0);
        for (int z = zc0; z < zc1; ++z) {
            wait_ring(z + 1);
            const int b = (z - zc0) % NP;
            if (!ws_wait(full_s + 8u * b, (fphase >> b) & 1u, false)) atomicOr(d_err, 4);
            fphase ^= 1u << b;
            float f[2][19];
            const float* P = pops + (size_t)b * 38 * TX;
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < 19; ++i) f[s][i] = P[(s * 19 + i) * TX + x];
            collide_node<TX, ST>(ring, slot_of(z - 1), slot_of(z), slot_of(z + 1), x, y, z, f, m, L, dst, d_err, cm,
                                 px, py);
            // the buffer may take plane z + NP (released after the collision,
            // so that the populations can stay in shared memory until used)
            mbar_arrive(empty_s + 8u * b);
        }
    }
    // no CTA leaves while another may still address its shared memory
    cluster.sync();

    // centre-of-mass partials of the written state (fixed-order reduction)
    double cmd[4] = {(double)cm[0], (double)cm[1], (double)cm[2], (double)cm[3]};
    centre_epilogue(cmd, cp, red);
}

constexpr int kRowMinBlocks = 6;

// Resident CTAs per SM asked of the compiler (it sets the register budget).
// Direct-load variant: 6 x 128 threads' worth (80 registers), except at
// Lx = 128, where 4 CTAs (128 registers) step 1.7 % (fp32) and 2.8 % (fp16
// deviations) faster at 128^3 -- the 512-CTA grid fills only 3.4 per SM, so
// the bound costs no occupancy; at Lx = 256, 3 CTAs (80 registers) beat 2
// (128 registers) by 2 % (fp32) and 13 % (fp16 deviations), measured on
// GB300.  The staged variant is bounded by its shared memory (about 2 x
// 128-thread CTAs per SM).
template <int TX, bool STAGED>
constexpr int row_min_blocks() {
    return STAGED ? (256 / TX > 0 ? 256 / TX : 1) : (TX == 128 ? 4 : kRowMinBlocks * 128 / TX);
}

template <int TX, int CY, typename S, bool STAGED>
constexpr size_t row_smem() {
    return STAGED ? StagedLayout<TX, CY, S>::bytes : FastLayout<TX, CY>::bytes;
}

template <int TX, int CY, typename S, bool STAGED, bool MRT>
cudaError_t launch_rows(const void* src, void* dst, const Layout& L, const Model& m, int zchunk, int nchunks,
                        CentreParts cp, int* d_err, cudaStream_t s) {
    auto k = k_stream_collide_rows<TX, CY, row_min_blocks<TX, STAGED>(), S, STAGED, MRT>;
    const size_t smem = row_smem<TX, CY, S, STAGED>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FastModel fm;
    for (int q = 0; q < 2; ++q) {
        fm.inv_tau[q] = (float)(1.0 / m.tau[q]);
        fm.tau[q] = (float)m.tau[q];
        fm.rho_b[q] = (float)m.rho_b[q];
    }
    fm.G = (float)m.G;
    for (int k = 0; k < 5; ++k) fm.mrt[k] = (float)m.mrt_rates[k];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, L.Ly, nchunks);
    cfg.blockDim = dim3(TX, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CY;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, (const S*)src, (S*)dst, L, fm, zchunk, cp, d_err);
}

template <int TX, int CY, typename S, bool STAGED, bool MRT>
int max_clusters() {
    auto k = k_stream_collide_rows<TX, CY, row_min_blocks<TX, STAGED>(), S, STAGED, MRT>;
    const size_t smem = row_smem<TX, CY, S, STAGED>();
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, CY, 1);
    cfg.blockDim = dim3(TX, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CY;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

constexpr int kRowCluster = 8;

template <int TX, typename S, bool STAGED, bool MRT = false>
cudaError_t rows_for(bool query, const void* src, void* dst, const Layout& L, const Model& m, int zchunk,
                     CentreParts cp, int* d_err, cudaStream_t s, int* resident) {
    if (query) {
        *resident = max_clusters<TX, kRowCluster, S, STAGED, MRT>() * kRowCluster;
        return cudaSuccess;
    }
    const int nchunks = (L.Lz + zchunk - 1) / zchunk;
    return launch_rows<TX, kRowCluster, S, STAGED, MRT>(src, dst, L, m, zchunk, nchunks, cp, d_err, s);
}

// Resident CTAs per SM asked of the compiler for the warp-specialised
// variant (2 TX threads, about 93 KB of shared memory at TX = 128: two CTAs
// of 256 threads per SM).
template <int TX>
constexpr int ws_min_blocks() {
    return TX >= 256 ? 1 : 256 / TX;
}

template <int TX, int CY, typename S>
cudaError_t ws_for(bool query, const void* src, void* dst, const Layout& L, const Model& m, int zchunk,
                   CentreParts cp, int* d_err, cudaStream_t s, int* resident) {
    auto k = k_stream_collide_ws<TX, CY, ws_min_blocks<TX>(), S>;
    const size_t smem = WsLayout<TX, CY>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        if (query) {
            cudaGetLastError();
            *resident = 0;
            return cudaSuccess;
        }
        return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(2 * TX, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CY;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (query) {
        cfg.gridDim = dim3(1, CY, 1);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        *resident = n * CY;
        return cudaSuccess;
    }
    FastModel fm;
    for (int q = 0; q < 2; ++q) {
        fm.inv_tau[q] = (float)(1.0 / m.tau[q]);
        fm.tau[q] = (float)m.tau[q];
        fm.rho_b[q] = (float)m.rho_b[q];
    }
    fm.G = (float)m.G;
    cfg.gridDim = dim3(1, L.Ly, (L.Lz + zchunk - 1) / zchunk);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, k, (const S*)src, (S*)dst, L, fm, zchunk, cp, d_err);
}

template <int TX, typename S>
cudaError_t rows_variant(int variant, bool query, const void* src, void* dst, const Layout& L, const Model& m,
                         int zchunk, CentreParts cp, int* d_err, cudaStream_t s, int* resident) {
    if (m.mrt) {  // MRT: float32 storage, direct loads only
        if constexpr (std::is_same<S, float>::value)
            return rows_for<TX, S, false, true>(query, src, dst, L, m, zchunk, cp, d_err, s, resident);
        return cudaErrorInvalidValue;
    }
    if (variant == kRowWs) return ws_for<TX, kRowCluster, S>(query, src, dst, L, m, zchunk, cp, d_err, s, resident);
    if (variant == kRowStaged) return rows_for<TX, S, true>(query, src, dst, L, m, zchunk, cp, d_err, s, resident);
    return rows_for<TX, S, false>(query, src, dst, L, m, zchunk, cp, d_err, s, resident);
}

// Dispatch on the row width, the storage type and the variant.
cudaError_t rows_dispatch(int prec, int variant, bool query, const void* src, void* dst, const Layout& L,
                          const Model& m, int zchunk, CentreParts cp, int* d_err, cudaStream_t s, int* resident) {
#define LBM_ROWS_TX(TXV)                                                                                        \
    if (L.Lx == TXV) {                                                                                          \
        if (prec == kFP32)                                                                                      \
            return rows_variant<TXV, float>(variant, query, src, dst, L, m, zchunk, cp, d_err, s, resident);     \
        if (prec == kFP16Dev)                                                                                   \
            return rows_variant<TXV, Dev<__half>>(variant, query, src, dst, L, m, zchunk, cp, d_err, s, resident); \
        if (prec == kBF16Dev)                                                                                   \
            return rows_variant<TXV, Dev<__nv_bfloat16>>(variant, query, src, dst, L, m, zchunk, cp, d_err, s,   \
                                                         resident);                                             \
    }
    LBM_ROWS_TX(32)
    LBM_ROWS_TX(64)
    LBM_ROWS_TX(128)
    LBM_ROWS_TX(256)
#undef LBM_ROWS_TX
    return cudaErrorInvalidValue;
}

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing
// arrives on (arrive = 0), or that thread 0 completes first (arrive = 1),
// with the helper every kernel of this file uses.
__device__ int g_wait_selftest;
__global__ void k_wait_selftest(unsigned long long limit_ns, int arrive) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) mbar_arrive(b);
    __syncthreads();
    const bool ok = wait_bounded(b, 0u, false, limit_ns);
    if (threadIdx.x == 0) g_wait_selftest = ok ? 1 : 0;
}

}  // namespace

bool rows_kernel_applies(const Layout& L, int prec, int periodic) {
    if ((prec != kFP32 && !is_dev(prec)) || periodic) return false;
    if (L.Lx != 32 && L.Lx != 64 && L.Lx != 128 && L.Lx != 256) return false;
    return L.Ly % kRowCluster == 0 && L.Lz >= 2;
}

int rows_kernel_resident_ctas(const Layout& L, int prec, int variant, int mrt) {
    int n = 0;
    Model m = {};
    m.mrt = mrt;
    CentreParts cp = {};
    if (rows_dispatch(prec, variant, true, nullptr, nullptr, L, m, 1, cp, nullptr, 0, &n) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_wait_selftest(unsigned long long limit_ns, int arrive, cudaStream_t s, int* gave_up) {
    const int unset = -1;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_wait_selftest, &unset, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, arrive);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int r = unset;
    if ((e = cudaMemcpyFromSymbolAsync(&r, g_wait_selftest, sizeof(int), 0, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (r < 0) return cudaErrorUnknown;
    *gave_up = r == 0 ? 1 : 0;
    return cudaSuccess;
}

cudaError_t launch_stream_collide_rows(int prec, int variant, const void* src, void* dst, const Layout& L,
                                       const Model& m, const Grad& A, int zchunk, CentreParts cp, int* d_err,
                                       cudaStream_t s) {
    (void)A;  // this kernel reads the ghost shell written by the ghost kernel
    return rows_dispatch(prec, variant, false, src, dst, L, m, zchunk, cp, d_err, s, nullptr);
}

}  // namespace lbmgb
