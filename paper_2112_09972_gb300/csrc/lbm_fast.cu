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
//     density planes in shared memory (4 slots); one plane later the same 38
//     values are read again for the collision (that second read is served by
//     L2).  Holding no populations on chip keeps each CTA at a few KB of
//     shared memory, so many CTAs per SM hide the latency;
//   * each CTA pushes its row of densities into the rings of the CTAs that
//     own rows y -/+ 1 with st.async, which counts the bytes on the
//     receiving CTA's mbarrier for that plane; the force (Eq. 7) then reads
//     all 18 neighbour densities from local shared memory after a bounded
//     mbarrier wait.  The two rows just outside the cluster are pulled a
//     second time by the two CTAs nearest each edge (half a row each), which
//     push them into the edge CTA's ring.  Every CTA's ring is written only by
//     itself and by the CTAs next to it, so no CTA runs more than one plane
//     ahead of its neighbours and four ring slots suffice (proof at
//     FastLayout).
// There is no cluster-wide barrier and no memory fence per plane: a CTA waits
// only for the two rows it reads.  DRAM sees about one read and one write of
// every population; L2 serves the second read and the outer-halo reads.
//
// Addressing.  In the row-interleaved layout (lbm_internal.h) every
// population a node pulls, and every population it writes, lies at a
// compile-time byte offset (fixed by Lx) from one of three pointers to the
// node's own element in planes z - 1, z, z + 1; the loads and stores carry
// those offsets as immediates, so the per-node address arithmetic is three
// pointer increments per plane.
//
// March direction.  Chunks with odd index march down in z, the others up, so
// the two chunks that meet at a chunk boundary read the planes on either side
// of it (each chunk's halo plane is the other's last plane) at the same time,
// at the end or at the start of both marches, and L2 serves the second of
// the two reads.  Every variant marches in the same order, so all three
// store bit-identical states.
//
// Sums over opposite velocity pairs are differenced first (c_{2k} = -c_{2k-1}),
// and the equilibria of a pair share their even part.
//
// Variants (lbm_opts.row_variant): the direct loads above; whole pulled rows
// staged in shared memory by bulk copies (k_stream_collide_rows<..., STAGED =
// true>, the automatic choice); and loader and collider
// threads per row (k_stream_collide_ws).  All three share collide_node.  The
// direct variant also has an MRT instance for float32 storage
// (collide_node<..., MRT = true>).

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "lbm_centre.cuh"
#include "lbm_dev.cuh"
#include "lbm_internal.h"
#include "lbm_lattice.cuh"
#include "lbm_pdl.cuh"

namespace cg = cooperative_groups;

// Build-time launch parameters of the direct row kernel: resident CTAs per SM
// asked of the compiler (its register budget) at each row width, and whether
// odd chunks march down in z.
#ifndef LBM_ROWS_MINB_32
#define LBM_ROWS_MINB_32 24
#endif
#ifndef LBM_ROWS_MINB_64
#define LBM_ROWS_MINB_64 12
#endif
#ifndef LBM_ROWS_MINB_128
#define LBM_ROWS_MINB_128 5
#endif
#ifndef LBM_ROWS_MINB_256
#define LBM_ROWS_MINB_256 3
#endif
#ifndef LBM_ROWS_ALTERNATE
#define LBM_ROWS_ALTERNATE 1
#endif
// L2 priority of the outer-halo loads: 0 evict_last, 1 evict_first, 2 evict_normal.
#ifndef LBM_ROWS_HALO_POLICY
#define LBM_ROWS_HALO_POLICY 2
#endif

namespace lbmgb {
namespace {

struct FastModel {
    float inv_tau[2], tau[2], G, rho_b[2];
    float omit[2];  // 1 - 1/tau
    float sh[2];    // -G tau: the velocity shift tau_s F^s / rho_s per unit of the other component's force sum
    float mrt[5];   // MRT free rates (s_e, s_eps, s_q, s_pi, s_m) when the kernel relaxes moments
};

FastModel fast_model(const Model& m) {
    FastModel fm;
    for (int q = 0; q < 2; ++q) {
        fm.inv_tau[q] = (float)(1.0 / m.tau[q]);
        fm.tau[q] = (float)m.tau[q];
        fm.rho_b[q] = (float)m.rho_b[q];
        fm.omit[q] = (float)(1.0 - 1.0 / m.tau[q]);
        fm.sh[q] = (float)(-m.G * m.tau[q]);
    }
    fm.G = (float)m.G;
    for (int k = 0; k < 5; ++k) fm.mrt[k] = (float)m.mrt_rates[k];
    return fm;
}

// Compile-time loop: f(std::integral_constant<int, 0>) ... f(..., N - 1).
template <typename F, int... I>
__device__ __forceinline__ void sfor_(F& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    sfor_(f, std::make_integer_sequence<int, N>{});
}

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
// Asynchronous copies of 4 bytes (at a pointer plus an immediate byte
// offset) and of 16 bytes from global to this thread's shared memory, and the
// wait for all of this thread's such copies.
template <int OFF>
__device__ __forceinline__ void cp_async4(unsigned dst, const void* src, unsigned long long pol) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1+%3], 4, %2;" ::"r"(dst), "l"(src), "l"(pol),
                 "n"(OFF)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, unsigned long long pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Global loads and stores at a pointer plus an immediate byte offset.  The
// first read of a plane keeps its lines in L2 (evict_last policy) for the
// second read one plane later, which marks them last-use; the written state
// is streamed out.  The populations read are never written by the kernel, so
// the loads may be scheduled freely.
template <int OFF>
__device__ __forceinline__ float ld_keep(const void* p, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1+%3], %2;" : "=f"(v) : "l"(p), "l"(pol), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ float ld_last(const void* p) {
    float v;
    asm("ld.global.lu.f32 %0, [%1+%2];" : "=f"(v) : "l"(p), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ unsigned ld_keep_u32(const void* p, unsigned long long pol) {
    unsigned v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1+%3], %2;" : "=r"(v) : "l"(p), "l"(pol), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ unsigned ld_last_u32(const void* p) {
    unsigned v;
    asm("ld.global.lu.b32 %0, [%1+%2];" : "=r"(v) : "l"(p), "n"(OFF));
    return v;
}
__device__ __forceinline__ float4 ld_keep_f4(const void* p, unsigned long long pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_last_f4(const void* p) {
    float4 v;
    asm("ld.global.lu.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
template <int OFF>
__device__ __forceinline__ void st_cs(void* p, float v) {
    asm volatile("st.global.cs.f32 [%0+%2], %1;" ::"l"(p), "f"(v), "n"(OFF));
}
template <int OFF>
__device__ __forceinline__ void st_cs_u32(void* p, unsigned v) {
    asm volatile("st.global.cs.b32 [%0+%2], %1;" ::"l"(p), "r"(v), "n"(OFF));
}
__device__ __forceinline__ void st_cs_f4(void* p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
}

// Compile-time geometry of the row-interleaved layout for row width TX (the
// values make_layout computes): entries before x = 0, entries per population
// row and layout units per row block (elements of 4 bytes for float32, units
// of 2 bytes for deviations).
template <int TX, typename ST>
struct RowGeo;
template <int TX>
struct RowGeo<TX, float> {
    static constexpr int X0 = 8, PITCH = TX + 16, ROW = 38 * PITCH;
};
template <int TX, typename T>
struct RowGeo<TX, Dev<T>> {
    static constexpr int X0 = 16, PITCH = TX + 32, ROW = 44 * PITCH;
};

// Storage-specific reads and writes of the row kernels.  A node's accesses
// go through its pointer `base` (the node in plane -1) and, per plane p, the
// three pointers P3 of planes p - 1, p, p + 1.
template <int TX, typename ST>
struct RowIO;

template <int TX>
struct RowIO<TX, float> {
    using G = RowGeo<TX, float>;
    struct P3 {
        const char* m;
        const char* o;
        const char* p;
    };
    using Out = float*;  // element (s = 0, i = 0) of the node in the written plane
    // element (s = 0, i = 0) of node (x, y) in plane -1
    static __device__ __forceinline__ const char* base(const float* src, int x, int y) {
        return reinterpret_cast<const char*>(src + (long long)(y + 1) * G::ROW + G::X0 + x);
    }
    // the same node, component s (the halo threads sum one component each)
    static __device__ __forceinline__ const char* base_c(const float* src, int x, int y, int s) {
        return base(src, x, y) + 4 * s * 19 * G::PITCH;
    }
    static __device__ __forceinline__ P3 planes(const char* b, const Layout& L, int p) {
        const long long pl = 4 * L.plane;
        const char* o = b + (long long)(p + 1) * pl;
        return {o - pl, o, o + pl};
    }
    static __device__ __forceinline__ Out out(float* dst, const Layout& L, int x, int y, int z) {
        return dst + (long long)(z + 1) * L.plane + (long long)(y + 1) * G::ROW + G::X0 + x;
    }
    // byte offset of population (s, i) pulled into the node (it comes from
    // x - c_i, which lies in plane p - c_iz: the pointer src_plane picks)
    template <int S, int I>
    static constexpr int poff() {
        return 4 * ((S * 19 + I) * G::PITCH - cy_(I) * G::ROW - cx_(I));
    }
    template <int I>
    static __device__ __forceinline__ const char* src_plane(const P3& q) {
        return cz_(I) > 0 ? q.m : (cz_(I) < 0 ? q.p : q.o);
    }
    // component S's post-streaming density (first read, kept in L2)
    template <int S>
    static __device__ __forceinline__ float density(const P3& q, unsigned long long pol) {
        float r = ld_keep<poff<S, 0>()>(q.o, pol);
        sfor<9>([&](auto K) {
            constexpr int i = 2 * decltype(K)::value + 1;
            r += ld_keep<poff<S, i>()>(src_plane<i>(q), pol) + ld_keep<poff<S, i + 1>()>(src_plane<i + 1>(q), pol);
        });
        return r;
    }
    static __device__ __forceinline__ void densities(const P3& q, unsigned long long pol, float& ra, float& rb) {
        ra = density<0>(q, pol);
        rb = density<1>(q, pol);
    }
    // the node's 38 pulled populations (second read, last use); rs: unused
    // in float32 (the deviation forms return the node's rho* there)
    static __device__ __forceinline__ void populations(const P3& q, float (&f)[2][19], float (&rs)[2]) {
        rs[0] = rs[1] = 0.f;
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            f[0][i] = ld_last<poff<0, i>()>(src_plane<i>(q));
            f[1][i] = ld_last<poff<1, i>()>(src_plane<i>(q));
        });
    }
    // one read of the 38 pulled populations and the densities summed from
    // them in the order of density() (the warp-specialised kernel)
    static __device__ __forceinline__ void load_all(const P3& q, float (&f)[2][19], float (&rs)[2], float& ra,
                                                    float& rb) {
        populations(q, f, rs);
        ra = f[0][0];
        rb = f[1][0];
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            ra += f[0][i] + f[0][i + 1];
            rb += f[1][i] + f[1][i + 1];
        }
    }
    template <int S, int I>
    static __device__ __forceinline__ void store(Out o, float v) {
        st_cs<4 * (S * 19 + I) * G::PITCH>(o, v);
    }
};

// 16-bit deviation storage: per node the float4 block {rho*_A, rho*_B, f*_0A,
// f*_0B} and the 18 words of deviation pairs {A, B}.  The plane pointers
// point at the node's word slot (x0 + x) of its row block; the node's own
// block lies a per-thread constant further (12 (x0 + x) bytes), and the word
// of direction i at the immediate 4 (3 + i) pitch.
template <int TX, typename T>
struct RowIO<TX, Dev<T>> {
    using G = RowGeo<TX, Dev<T>>;
    struct P3 {
        const char* m;
        const char* o;
        const char* p;
        int blk;  // byte offset of the node's float4 block from o
    };
    struct Out {
        unsigned* w;  // word slot of the node in the written plane
        float4* b;    // the node's float4 block
    };
    static __device__ __forceinline__ const char* base(const Dev<T>* src, int x, int y) {
        return reinterpret_cast<const char*>(src) + 2LL * (long long)(y + 1) * G::ROW + 4 * (G::X0 + x);
    }
    static __device__ __forceinline__ P3 planes(const char* b, const Layout& L, int p, int x) {
        const long long pl = 2 * L.plane;
        const char* o = b + (long long)(p + 1) * pl;
        return {o - pl, o, o + pl, 12 * (G::X0 + x)};
    }
    static __device__ __forceinline__ Out out(Dev<T>* dst, const Layout& L, int x, int y, int z) {
        char* o = reinterpret_cast<char*>(dst) + 2LL * ((long long)(z + 1) * L.plane + (long long)(y + 1) * G::ROW) +
                  4 * (G::X0 + x);
        return {reinterpret_cast<unsigned*>(o), reinterpret_cast<float4*>(o + 12 * (G::X0 + x))};
    }
    template <int I>
    static constexpr int woff() {  // byte offset of the word of direction I pulled into the node
        return 4 * (3 + I) * G::PITCH - 2 * cy_(I) * G::ROW - 4 * cx_(I);
    }
    template <int I>
    static __device__ __forceinline__ const char* src_plane(const P3& q) {
        return cz_(I) > 0 ? q.m : (cz_(I) < 0 ? q.p : q.o);
    }
    // sum_i (w_i rho* + d_i) + f*_0 = f*_0 + (1 - w_0) rho* + sum_i d_i, from
    // the node's block o and its pulled words word(integral_constant<int, i>)
    template <typename W>
    static __device__ __forceinline__ void sum_words(const float4& o, W&& word, float& ra, float& rb) {
        float da = 0.f, db = 0.f;
        sfor<9>([&](auto K) {
            constexpr int i = 2 * decltype(K)::value + 1;
            const float2 u = dev_unpack2<T>(word(std::integral_constant<int, i>{}));
            const float2 v = dev_unpack2<T>(word(std::integral_constant<int, i + 1>{}));
            da += u.x + v.x;
            db += u.y + v.y;
        });
        ra = o.z + (1.f - wgt<float>(0)) * o.x + da;
        rb = o.w + (1.f - wgt<float>(0)) * o.y + db;
    }
    static __device__ __forceinline__ void densities(const P3& q, unsigned long long pol, float& ra, float& rb) {
        const float4 o = ld_keep_f4(q.o + q.blk, pol);
        sum_words(
            o,
            [&](auto I) {
                constexpr int i = decltype(I)::value;
                return ld_keep_u32<woff<i>()>(src_plane<i>(q), pol);
            },
            ra, rb);
    }
    // The collision's input in deviation form: f[s][0] the rest population,
    // f[s][i >= 1] the pulled deviation d_i (the population is
    // w_i rho*_s + d_i; collide_node folds w_i rho*_s into its constants),
    // rs the node's rho* of both components.
    static __device__ __forceinline__ void populations(const P3& q, float (&f)[2][19], float (&rs)[2]) {
        const float4 o = ld_last_f4(q.o + q.blk);
        f[0][0] = o.z;
        f[1][0] = o.w;
        rs[0] = o.x;
        rs[1] = o.y;
        sfor<18>([&](auto K) {
            constexpr int i = decltype(K)::value + 1;
            const float2 v = dev_unpack2<T>(ld_last_u32<woff<i>()>(src_plane<i>(q)));
            f[0][i] = v.x;
            f[1][i] = v.y;
        });
    }
    // one read of the block and the 18 pulled words: the input of
    // populations() and the densities of densities(), with their arithmetic
    static __device__ __forceinline__ void load_all(const P3& q, float (&f)[2][19], float (&rs)[2], float& ra,
                                                    float& rb) {
        const float4 o = ld_last_f4(q.o + q.blk);
        f[0][0] = o.z;
        f[1][0] = o.w;
        rs[0] = o.x;
        rs[1] = o.y;
        float da = 0.f, db = 0.f;
        sfor<9>([&](auto K) {
            constexpr int i = 2 * decltype(K)::value + 1;
            const float2 u = dev_unpack2<T>(ld_last_u32<woff<i>()>(src_plane<i>(q)));
            const float2 v = dev_unpack2<T>(ld_last_u32<woff<i + 1>()>(src_plane<i + 1>(q)));
            da += u.x + v.x;
            db += u.y + v.y;
            f[0][i] = u.x;
            f[1][i] = u.y;
            f[0][i + 1] = v.x;
            f[1][i + 1] = v.y;
        });
        ra = o.z + (1.f - wgt<float>(0)) * o.x + da;
        rb = o.w + (1.f - wgt<float>(0)) * o.y + db;
    }
    template <int I>
    static __device__ __forceinline__ void store_word(Out o, unsigned v) {
        st_cs_u32<4 * (3 + I) * G::PITCH>(o.w, v);
    }
};

// Outer-halo pulls of the staged variant, prefetched into shared memory one
// march step ahead by asynchronous copies (each halo thread copies the
// values it sums into its own slots, so no barrier is involved; it waits for
// its own copies before it sums them, in the order of RowIO::density /
// RowIO::densities).  Float32: thread x copies the 19 pulled populations of
// its component, slot [i][x].  Deviations: threads x < TX / 2 copy the
// node's float4 block (slot [x]) and its 18 pulled words (slots [i - 1][x]).
template <int TX, typename ST>
struct HaloPrefetch;
template <int TX>
struct HaloPrefetch<TX, float> {
    using IO = RowIO<TX, float>;
    static constexpr unsigned BYTES = 19u * 4u * TX;
    static __device__ __forceinline__ void issue(const typename IO::P3& q, unsigned long long pol, unsigned buf,
                                                 int x) {
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            cp_async4<IO::template poff<0, i>()>(buf + 4u * (unsigned)(i * TX + x), IO::template src_plane<i>(q), pol);
        });
    }
    static __device__ __forceinline__ float sum(const float* buf, int x) {
        const float* b = buf + x;
        float r = b[0];
#pragma unroll
        for (int i = 1; i < 19; i += 2) r += b[i * TX] + b[(i + 1) * TX];
        return r;
    }
};
template <int TX, typename T>
struct HaloPrefetch<TX, Dev<T>> {
    using IO = RowIO<TX, Dev<T>>;
    static constexpr int NT = TX / 2;  // halo threads
    static constexpr unsigned BYTES = 16u * NT + 18u * 4u * NT;
    static __device__ __forceinline__ void issue(const typename IO::P3& q, unsigned long long pol, unsigned buf,
                                                 int x) {
        cp_async16(buf + 16u * (unsigned)x, q.o + q.blk, pol);
        sfor<18>([&](auto K) {
            constexpr int i = decltype(K)::value + 1;
            cp_async4<IO::template woff<i>()>(buf + 16u * NT + 4u * (unsigned)((i - 1) * NT + x),
                                              IO::template src_plane<i>(q), pol);
        });
    }
    static __device__ __forceinline__ void sum(const float* buf, int x, float& ra, float& rb) {
        const float4 o = reinterpret_cast<const float4*>(buf)[x];
        const unsigned* w = reinterpret_cast<const unsigned*>(buf + 4 * NT) + x;
        IO::sum_words(
            o, [&](auto I) { return w[(decltype(I)::value - 1) * NT]; }, ra, rb);
    }
};

// ---- TMA-staged variant: bulk copies of whole pulled rows into shared memory ----

// Direction i's velocity at run time (the bulk copies are spread over the
// lanes of a warp, one population row per lane).
__device__ __forceinline__ void dir_rt(int i, int& cx, int& cy, int& cz) {
    // 2 bits per direction and axis: 0 -> -1, 1 -> 0, 2 -> +1
    constexpr unsigned long long TX_ = [] {
        unsigned long long t = 0;
        for (int k = 0; k < 19; ++k) t |= (unsigned long long)(cx_(k) + 1) << (2 * k);
        return t;
    }();
    constexpr unsigned long long TY_ = [] {
        unsigned long long t = 0;
        for (int k = 0; k < 19; ++k) t |= (unsigned long long)(cy_(k) + 1) << (2 * k);
        return t;
    }();
    constexpr unsigned long long TZ_ = [] {
        unsigned long long t = 0;
        for (int k = 0; k < 19; ++k) t |= (unsigned long long)(cz_(k) + 1) << (2 * k);
        return t;
    }();
    cx = (int)((TX_ >> (2 * i)) & 3ull) - 1;
    cy = (int)((TY_ >> (2 * i)) & 3ull) - 1;
    cz = (int)((TZ_ >> (2 * i)) & 3ull) - 1;
}

// Shared-memory image of one plane of one row for the staged variant: every
// population row the row's pulled populations come from, as a segment of
// SEG entries in which x sits at index x + 4.  Only the x range a direction
// reads is copied: x = 0 .. TX - 1 for c_ix = 0, from x = -4 (the 16-byte
// aligned start that covers the ghost at x = -1) for c_ix = +1, up to
// x = TX + 3 (covering x = TX) for c_ix = -1.  Each source row is y - c_iy of
// plane p - c_iz, so over the grid every population row is copied once.  The
// copies are issued by the lanes of warp 0, one population row per lane,
// after lane 0 has armed the plane's mbarrier with their total size.
//
// Raw is what a thread carries in registers from the plane's density pass to
// its collision one march step later (the stage is refilled in between).
template <int TX, typename ST>
struct StagePlane;

template <int TX>
struct StagePlane<TX, float> {
    static constexpr int SEG = TX + 8;
    static constexpr unsigned SMEM = 38u * SEG * 4u;                               // bytes of the image
    static constexpr unsigned BYTES = 2u * (9u * 4u * TX + 10u * 4u * (TX + 4));  // bytes copied per plane
    struct Raw {
        float f[2][19];
    };
    static __device__ __forceinline__ void issue(const float* src, const Layout& L, int y, int p, unsigned dst,
                                                 unsigned mbar, int lane) {
        for (int a = lane; a < 38; a += 32) {
            const int s = a / 19, i = a - 19 * s;
            int cx, cy, cz;
            dir_rt(i, cx, cy, cz);
            const int lo = cx > 0 ? -4 : 0;
            const unsigned len = cx != 0 ? 4u * (TX + 4) : 4u * TX;
            bulk_g2s(dst + 4u * (unsigned)(SEG * a + lo + 4), src + L.at(s, i, lo, y - cy, p - cz), len, mbar);
        }
    }
    // the node's 38 pulled populations and its densities, summed in the
    // order of RowIO::density
    static __device__ __forceinline__ void load(const float* st, int x, Raw& r, float& ra, float& rb) {
        const float* b = st + x + 4;
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            r.f[0][i] = b[i * SEG - cx_(i)];
            r.f[1][i] = b[(19 + i) * SEG - cx_(i)];
        });
        ra = r.f[0][0];
        rb = r.f[1][0];
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            ra += r.f[0][i] + r.f[0][i + 1];
            rb += r.f[1][i] + r.f[1][i + 1];
        }
    }
    static __device__ __forceinline__ void unpack(const Raw& r, float (&f)[2][19], float (&rs)[2]) {
        rs[0] = rs[1] = 0.f;
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 19; ++i) f[s][i] = r.f[s][i];
    }
};

template <int TX, typename T>
struct StagePlane<TX, Dev<T>> {
    static constexpr int SEG = TX + 8;  // words per deviation segment
    static constexpr unsigned NODE_BYTES = 16u * TX;
    static constexpr unsigned SMEM = NODE_BYTES + 18u * SEG * 4u;
    static constexpr unsigned BYTES = NODE_BYTES + 8u * 4u * TX + 10u * 4u * (TX + 4);
    struct Raw {
        float4 o;
        unsigned w[19];  // w[i]: the word of direction i >= 1
    };
    static __device__ __forceinline__ void issue(const Dev<T>* src, const Layout& L, int y, int p, unsigned dst,
                                                 unsigned mbar, int lane) {
        if (lane == 0) {
            bulk_g2s(dst, reinterpret_cast<const float4*>(src) + L.dev_node(0, y, p), NODE_BYTES, mbar);
        } else if (lane < 19) {
            const int i = lane;
            int cx, cy, cz;
            dir_rt(i, cx, cy, cz);
            const int lo = cx > 0 ? -4 : 0;
            const unsigned len = cx != 0 ? 4u * (TX + 4) : 4u * TX;
            const unsigned* w = reinterpret_cast<const unsigned*>(src);
            bulk_g2s(dst + NODE_BYTES + 4u * (unsigned)(SEG * (i - 1) + lo + 4), w + L.dev_word(i, lo, y - cy, p - cz),
                     len, mbar);
        }
    }
    static __device__ __forceinline__ void load(const float* st, int x, Raw& r, float& ra, float& rb) {
        r.o = reinterpret_cast<const float4*>(st)[x];
        const unsigned* b = reinterpret_cast<const unsigned*>(reinterpret_cast<const char*>(st) + NODE_BYTES) + x + 4;
        float da = 0.f, db = 0.f;
        sfor<9>([&](auto K) {
            constexpr int i = 2 * decltype(K)::value + 1;
            r.w[i] = b[(i - 1) * SEG - cx_(i)];
            r.w[i + 1] = b[i * SEG - cx_(i + 1)];
            const float2 u = dev_unpack2<T>(r.w[i]);
            const float2 v = dev_unpack2<T>(r.w[i + 1]);
            da += u.x + v.x;
            db += u.y + v.y;
        });
        ra = r.o.z + (1.f - wgt<float>(0)) * r.o.x + da;
        rb = r.o.w + (1.f - wgt<float>(0)) * r.o.y + db;
    }
    // the collision's input in deviation form (RowIO<TX, Dev<T>>::populations)
    static __device__ __forceinline__ void unpack(const Raw& r, float (&f)[2][19], float (&rs)[2]) {
        f[0][0] = r.o.z;
        f[1][0] = r.o.w;
        rs[0] = r.o.x;
        rs[1] = r.o.y;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const float2 v = dev_unpack2<T>(r.w[i]);
            f[0][i] = v.x;
            f[1][i] = v.y;
        }
    }
};

// Density ring of the direct and staged row kernels: S slots, each three
// rows (-1, 0, +1: the neighbour row below, this CTA's row, the neighbour row
// above) of RW = TX + 2 columns (x = -1 .. TX) of float2 {rho_A, rho_B},
// then S mbarriers.  Plane number k of the march (k = 0 .. n + 1) lives in
// slot k mod S.
//
// Why S = 4 slots suffice.  The writers of a CTA b's ring are b itself and
// the CTAs next to b in the cluster (its neighbour rows; the outer-halo rows
// of an edge CTA come from the edge CTA and its neighbour).  Each writer a of
// b is in turn written by b.  A CTA pushes plane k (march order) only after
// it waited for plane k - 1 of its ring, i.e. after b pushed plane k - 1,
// which b did only after it had collided plane k - 3.  Slot k mod S last held
// plane k - S, whose last reader is the collision of plane k - S + 1 (it reads
// planes k - S .. k - S + 2).  So b is done with the slot when a pushes into
// it if k - S + 1 <= k - 3, i.e. S >= 4.  b's own threads write row 0 of the
// slot only after the __syncthreads of the previous march step, which every
// thread reaches after colliding plane k - 3: the same bound.  The barrier of
// a slot therefore completes once per use, and the wait for plane k uses
// parity (k / S) mod 2.
template <int TX, int CY>
struct FastLayout {
    static constexpr int RW = TX + 2;
    static constexpr int S = 4;
    static constexpr int SLOT = 3 * RW;                  // float2 per slot
    static constexpr unsigned TX_BYTES = 2u * TX * 8u;  // rows -1 and +1 of a slot land by st.async
    static constexpr size_t ring_bytes = sizeof(float2) * S * SLOT;
    static constexpr size_t bytes = ring_bytes + sizeof(unsigned long long) * S;
};

// Shared memory of the staged variant beyond the density ring: NST stage
// mbarriers, then (128-byte aligned) NST plane images, then the outer-halo
// prefetch slots (HaloPrefetch).  March plane k lives in stage k mod NST:
// while plane k is collided (from registers), the copies of planes k + 2 ..
// k + 1 + NST are in flight, and so are the halo copies of plane k + 2.
// (A third stage was measured: no faster for 16-bit storage, where 128-wide
// rows keep 4 resident CTAs per SM with it, and slower for float32, where it
// costs resident CTAs.)
template <int TX, int CY, typename ST>
struct StagedLayout {
    static constexpr int NST = 2;
    static constexpr size_t mbar_off = FastLayout<TX, CY>::bytes;
    static constexpr size_t stage_off = ((mbar_off + 8 * NST + 127) / 128) * 128;
    // the outer-halo prefetch slots (rows up to 128 wide, and 16-bit storage
    // at any width: for float32 rows of 256 they would halve the resident
    // CTAs per SM)
    static constexpr bool HALO = TX <= 128 || is_dev_t<ST>::value;
    static constexpr size_t halo_off = stage_off + (size_t)NST * StagePlane<TX, ST>::SMEM;
    static constexpr size_t bytes = halo_off + (HALO ? (size_t)HaloPrefetch<TX, ST>::BYTES : 0);
};

// Collision of one node from its 38 pulled populations f and the density
// ring (rzm, rz0, rzp: this node's column in the slots of planes z - 1, z,
// z + 1; row r of a slot is r * RW further): momentum (Eq. 6), Shan-Chen
// force (Eq. 7), common velocity with the force shift, BGK relaxation to the
// equilibrium of Eq. 8 (Eqs. 9, 10) -- or, with MRT (float32 storage), the
// moment relaxation of the generic kernel -- and the store of the
// post-collision state (float32 populations with the rest population closing
// the mass balance, or 16-bit deviations).  Also accumulates the
// centre-of-mass partials of the droplet phase and flags non-finite
// densities.  Shared by the row kernels so that every variant computes
// bit-identical states.
template <int TX, typename ST, bool MRT = false>
__device__ __forceinline__ void collide_node(const float2* rzm, const float2* rz0, const float2* rzp,
                                             const float (&f)[2][19], const float (&rs)[2], const FastModel& m,
                                             typename RowIO<TX, ST>::Out out, float (&cm)[4], int& bad, float px,
                                             float py, float pz) {
    using IO = RowIO<TX, ST>;
    constexpr int RW = TX + 2;
    // neighbour densities {A, B} at offset (dx, dy, dz)
    auto nb = [&](int dx, int dy, int dz) -> float2 {
        const float2* r = dz == 0 ? rz0 : (dz > 0 ? rzp : rzm);
        return r[(dy + 1) * RW + dx];
    };
    const float2 rho2 = rz0[RW];
    const float rho[2] = {rho2.x, rho2.y};
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
    // Shan-Chen force (Eq. 7) sums sum_i w_i rho_s(x + c_i) c_i, neighbour
    // pairs differenced first; the weight folds into the multiplier
    float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const float2 np = nb(cx_(i), cy_(i), cz_(i)), nm = nb(-cx_(i), -cy_(i), -cz_(i));
        const float dA = np.x - nm.x, dB = np.y - nm.y;
        if (cx_(i)) { acc[0][0] += (wgt<float>(i) * cx_(i)) * dA; acc[1][0] += (wgt<float>(i) * cx_(i)) * dB; }
        if (cy_(i)) { acc[0][1] += (wgt<float>(i) * cy_(i)) * dA; acc[1][1] += (wgt<float>(i) * cy_(i)) * dB; }
        if (cz_(i)) { acc[0][2] += (wgt<float>(i) * cz_(i)) * dA; acc[1][2] += (wgt<float>(i) * cz_(i)) * dB; }
    }
    const float den = rho[0] * m.inv_tau[0] + rho[1] * m.inv_tau[1];
    const float rden = __frcp_rn(den);
    float up[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) up[a] = (j[0][a] * m.inv_tau[0] + j[1][a] * m.inv_tau[1]) * rden;
    if (!(isfinite(rho[0]) && isfinite(rho[1]))) bad |= 1;
    {
        const float phi = __fdividef(rho[0] - rho[1], rho[0] + rho[1]);
        const float w = fmaxf(phi, 0.f);
        cm[0] += w;
        cm[1] = fmaf(w, px, cm[1]);
        cm[2] = fmaf(w, py, cm[2]);
        cm[3] = fmaf(w, pz, cm[3]);
    }
    if constexpr (is_dev_t<ST>::value) {
        // 16-bit deviations from w_i times the density of the node each
        // population streams to (this CTA's density planes), the pair of
        // components of one direction in one word
        // f holds the pulled deviations (f_i = w_i rho*_s + d_i, rs = rho*):
        // (1 - 1/tau) f_i = (1 - 1/tau) d_i + (1 - 1/tau) w_i rho*_s, whose
        // second term joins the equilibrium's constant (W1 / W2 below), and
        // the momentum's opposite-pair differences are those of the d_i
        using T = decltype(dev_tag(ST{}));
        float ux[2], uy[2], uz[2], base[2], e1[2], e2[2], W1[2], W2[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            ux[s] = fmaf(m.sh[s], acc[1 - s][0], up[0]);
            uy[s] = fmaf(m.sh[s], acc[1 - s][1], up[1]);
            uz[s] = fmaf(m.sh[s], acc[1 - s][2], up[2]);
            base[s] = 1.f - 1.5f * (ux[s] * ux[s] + uy[s] * uy[s] + uz[s] * uz[s]);
            const float ir = m.inv_tau[s] * rho[s];
            e1[s] = ir * wgt<float>(1);  // axis directions
            e2[s] = ir * wgt<float>(7);  // edge directions
            const float orr = m.omit[s] * rs[s];
            W1[s] = orr * wgt<float>(1);
            W2[s] = orr * wgt<float>(7);
        }
        float others[2] = {0.f, 0.f};
        sfor<9>([&](auto K) {
            constexpr int i = 2 * decltype(K)::value + 1;
            // densities of the destinations x + c_i and x - c_i (read again
            // from shared memory rather than held since the force)
            const float2 np = nb(cx_(i), cy_(i), cz_(i)), nm = nb(-cx_(i), -cy_(i), -cz_(i));
            float da[2], dbv[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float cu = (float)cx_(i) * ux[s] + (float)cy_(i) * uy[s] + (float)cz_(i) * uz[s];
                const float e = i < 7 ? e1[s] : e2[s];
                const float ev = fmaf(e, fmaf(4.5f * cu, cu, base[s]), i < 7 ? W1[s] : W2[s]);
                const float od = (3.f * e) * cu;
                const float oa = fmaf(m.omit[s], f[s][i], ev + od);
                const float ob = fmaf(m.omit[s], f[s][i + 1], ev - od);
                // deviations from w_i times the destinations' densities
                da[s] = fmaf(-wgt<float>(i), s ? np.y : np.x, oa);
                dbv[s] = fmaf(-wgt<float>(i), s ? nm.y : nm.x, ob);
            }
            const unsigned wa = dev_pack2<T>(da[0], da[1]), wb = dev_pack2<T>(dbv[0], dbv[1]);
            IO::template store_word<i>(out, wa);
            IO::template store_word<i + 1>(out, wb);
            // the values the readers will rebuild, for the mass balance
            const float2 qa = dev_unpack2<T>(wa), qb = dev_unpack2<T>(wb);
            others[0] += fmaf(wgt<float>(i), np.x, qa.x) + fmaf(wgt<float>(i), nm.x, qb.x);
            others[1] += fmaf(wgt<float>(i), np.y, qa.y) + fmaf(wgt<float>(i), nm.y, qb.y);
        });
        st_cs_f4(out.b, make_float4(rho[0], rho[1], rho[0] - others[0], rho[1] - others[1]));
    } else {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float ux = fmaf(m.sh[s], acc[1 - s][0], up[0]);
            const float uy = fmaf(m.sh[s], acc[1 - s][1], up[1]);
            const float uz = fmaf(m.sh[s], acc[1 - s][2], up[2]);
            const float r = rho[s];
            // moving populations; the rest population then closes the mass
            // balance exactly (sum of outputs = rho), which keeps fp32
            // rounding from drifting the interface
            float others = 0.f;
            if constexpr (MRT) {
                // MRT: relax the moments of the deviation from equilibrium
                // (d'Humieres basis; momentum and stress at 1/tau)
                const float u2x = 1.5f * (ux * ux + uy * uy + uz * uz);
                float dv[19], o[19];
#pragma unroll
                for (int i = 0; i < 19; ++i) dv[i] = f[s][i] - feq<float>(i, r, ux, uy, uz, u2x);
                mrt_relax<float>(f[s], dv, m.inv_tau[s], m.mrt, o);
                sfor<9>([&](auto K) {
                    constexpr int i = 2 * decltype(K)::value + 1;
                    if (s == 0) {
                        IO::template store<0, i>(out, o[i]);
                        IO::template store<0, i + 1>(out, o[i + 1]);
                    } else {
                        IO::template store<1, i>(out, o[i]);
                        IO::template store<1, i + 1>(out, o[i + 1]);
                    }
                    others += o[i] + o[i + 1];
                });
            } else {
                const float base = 1.f - 1.5f * (ux * ux + uy * uy + uz * uz);
                const float ir = m.inv_tau[s] * r;
                const float e1 = ir * wgt<float>(1), e2 = ir * wgt<float>(7);
                const float om = m.omit[s];
                sfor<9>([&](auto K) {
                    constexpr int i = 2 * decltype(K)::value + 1;
                    const float cu = (float)cx_(i) * ux + (float)cy_(i) * uy + (float)cz_(i) * uz;
                    const float e = i < 7 ? e1 : e2;
                    const float ev = e * fmaf(4.5f * cu, cu, base);
                    const float od = (3.f * e) * cu;
                    const float oa = fmaf(om, f[s][i], ev + od);
                    const float ob = fmaf(om, f[s][i + 1], ev - od);
                    if (s == 0) {
                        IO::template store<0, i>(out, oa);
                        IO::template store<0, i + 1>(out, ob);
                    } else {
                        IO::template store<1, i>(out, oa);
                        IO::template store<1, i + 1>(out, ob);
                    }
                    others += oa + ob;
                });
            }
            if (s == 0) IO::template store<0, 0>(out, r - others);
            else IO::template store<1, 0>(out, r - others);
        }
    }
}

// Outer-halo share of a CTA of the direct and staged kernels: the rows just
// outside the cluster (y0 - 1 below, y0 + CY above) are pulled by the two
// CTAs nearest each edge, half a row each, and pushed into the edge CTA's
// ring (row -1 of rank 0, row +1 of rank CY - 1).  Float32: thread x sums
// component x & 1 of halo node x / 2 of the CTA's half; deviations (both
// components in one word): threads x < TX / 2 sum a whole node each.
template <int TX, int CY, typename ST>
struct HaloShare {
    bool cta;   // this CTA pulls outer-halo nodes
    bool thr;   // this thread pushes one (float32: the even thread of a pair)
    bool in;    // the halo row lies in the box
    int col;    // the halo node's column
    int comp;   // float32: the component this thread sums
    int row;    // ring row of the edge CTA it lands in (-1 or +1)
    int rank;   // the edge CTA
    int y;      // the halo row
    __device__ __forceinline__ HaloShare(int x, int r, int Y0, int Ly) {
        static_assert(CY >= 4, "the two halo pairs of CTAs must not overlap");
        const bool lo = r < 2, hi = r >= CY - 2;
        cta = lo || hi;
        const int half = lo ? r : r - (CY - 2);
        y = lo ? Y0 - 1 : Y0 + CY;
        in = y >= 0 && y < Ly;
        row = lo ? -1 : 1;
        rank = lo ? 0 : CY - 1;
        if constexpr (is_dev_t<ST>::value) {
            thr = cta && x < TX / 2;
            col = half * (TX / 2) + x;
            comp = 0;
        } else {
            thr = cta && (x & 1) == 0;
            col = half * (TX / 2) + (x >> 1);
            comp = x & 1;
        }
    }
};

// The march of a CTA of the direct and staged kernels: the z chunk
// blockIdx.z of the CTA's row, odd chunks marching down when `alt`.  (The
// kernel walks a list of such segments, continuing its march counter across
// them; one segment per CTA is what the launches use.)
struct Segment {
    int g;      // row group (rows g CY .. g CY + CY - 1)
    int z0, z1; // planes [z0, z1)
    bool down;
};
template <int CY>
struct MarchPlan {
    int nseg, Lz, zchunk;
    bool down;
    __device__ __forceinline__ MarchPlan(const Layout& L, int zchunk_, int alt) {
        Lz = L.Lz;
        zchunk = zchunk_;
        nseg = 1;
        down = alt && (blockIdx.z & 1);
    }
    __device__ __forceinline__ Segment seg(int) const {
        Segment sg;
        sg.down = down;
        sg.g = (int)blockIdx.y / CY;
        sg.z0 = (int)blockIdx.z * zchunk;
        sg.z1 = min(sg.z0 + zchunk, Lz);
        return sg;
    }
};

// The last CTA of a batched launch advances the device step counter (thread 0).
__device__ __forceinline__ void rows_batch_count(const RowsBatch& rb) {
    if (threadIdx.x != 0) return;
    __threadfence();
    if (atomicAdd(rb.ctas_done, 1u) == gridDim.x * gridDim.y * gridDim.z - 1u) {
        *rb.d_step += 1;
        *rb.ctas_done = 0u;
    }
}

// BATCH: the batched ensemble (RowsBatch): the box, its row and z chunk come
// from the row-group table instead of the launch's single box, nodes at
// x >= Lx of a padded row are idle (their ring entries hold the ghost
// density), and the centre of mass is reduced per box.
template <int TX, int CY, int MINB, typename ST, bool STAGED, bool MRT = false, bool BATCH = false>
__global__ void __launch_bounds__(TX, MINB)
    k_stream_collide_rows(const ST* __restrict__ src_p, ST* __restrict__ dst_p, Layout Lp, FastModel m, int zchunk,
                          int alt, CentreParts cp, int* __restrict__ d_err, RowsBatch bt) {
    using IO = RowIO<TX, ST>;
    using FL = FastLayout<TX, CY>;
    using SP = StagePlane<TX, ST>;
    using SL = StagedLayout<TX, CY, ST>;
    using HS = HaloShare<TX, CY, ST>;
    constexpr int RW = FL::RW, S = FL::S, NST = SL::NST;
    constexpr bool DEV = is_dev_t<ST>::value;
    extern __shared__ __align__(128) float2 ring[];  // [S][3][RW], then S mbarriers (staged: see StagedLayout)
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(ring + S * FL::SLOT);
    __shared__ float red[4 * ((TX + 31) / 32)];

    __shared__ Layout sL;  // BATCH: the box's layout

    // BATCH: this cluster's row group {box, first row, the box's z chunks}; a
    // cluster beyond its box's chunks leaves at once (all its CTAs together,
    // before any barrier)
    int4 gi = make_int4(0, 0, 0, 0);
    if constexpr (BATCH) {
        gi = bt.group[blockIdx.y / CY];
        if ((int)blockIdx.z >= gi.z) {
            rows_batch_count(bt);
            return;
        }
        if (threadIdx.x == 0) sL = bt.box[gi.x].L;
        __syncthreads();
    }
    const Layout& L = BATCH ? sL : Lp;
    const ST* __restrict__ src = BATCH ? reinterpret_cast<const ST*>(bt.box[gi.x].f[bt.parity]) : src_p;
    ST* __restrict__ dst = BATCH ? reinterpret_cast<ST*>(bt.box[gi.x].f[1 - bt.parity]) : dst_p;

    cg::cluster_group cluster = cg::this_cluster();
    const int x = threadIdx.x;
    const int rank = (int)cluster.block_rank();  // == blockIdx.y % CY for cluster dims (1, CY, 1)
    const MarchPlan<CY> plan(L, zchunk, alt);
    const bool xact = !BATCH || x < L.Lx;  // BATCH: a node of the box (not row padding)

    const unsigned ring_s = smem_u32(ring);
    const unsigned mbar_s = smem_u32(mbar);
    // Where this CTA's own row goes in the neighbours' rings (cluster addresses).
    const unsigned below_ring = rank > 0 ? cluster_addr(ring_s, rank - 1) : 0u;  // their row +1
    const unsigned below_mbar = rank > 0 ? cluster_addr(mbar_s, rank - 1) : 0u;
    const unsigned above_ring = rank < CY - 1 ? cluster_addr(ring_s, rank + 1) : 0u;  // their row -1
    const unsigned above_mbar = rank < CY - 1 ? cluster_addr(mbar_s, rank + 1) : 0u;

    // staged variant: plane images and their mbarriers (one arrival, by
    // lane 0 of warp 0, plus the bytes of the copies)
    const unsigned smbar_s = smem_u32(ring) + (unsigned)SL::mbar_off;
    const unsigned stage_s = smem_u32(ring) + (unsigned)SL::stage_off;
    const float* stage = reinterpret_cast<const float*>(reinterpret_cast<const char*>(ring) + SL::stage_off);
    // staged variant: the outer-halo prefetch slots
    using HP = HaloPrefetch<TX, ST>;
    constexpr bool PREF = STAGED && SL::HALO;
    const unsigned halo_s = smem_u32(ring) + (unsigned)SL::halo_off;
    const float* halo_buf = reinterpret_cast<const float*>(reinterpret_cast<const char*>(ring) + SL::halo_off);

    // ghost density in every slot (x halo columns keep it for good), barriers
    for (int e = x; e < S * FL::SLOT; e += TX) ring[e] = make_float2(m.rho_b[0], m.rho_b[1]);
    if (x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(mbar_s + 8u * k, 1u);
        if constexpr (STAGED)
            for (int k = 0; k < NST; ++k) mbar_init(smbar_s + 8u * k, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();  // barriers initialised before any remote store arrives
    pdl_wait();      // (a no-op unless launched with the programmatic attribute)

    // L2 policies: the direct variant's first read of a plane keeps its lines
    // (evict_last) for the second read one plane later; the outer-halo rows
    // are read once here (their owner reads them too), so they do not claim
    // that priority.
    unsigned long long keep, once;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
#if LBM_ROWS_HALO_POLICY == 1
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(once));
#elif LBM_ROWS_HALO_POLICY == 2
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(once));
#else
    once = keep;
#endif
    auto planes = [&](const char* b, int p, int col) {
        if constexpr (DEV) return IO::planes(b, L, p, col);
        else return IO::planes(b, L, p);
    };

    float cm[4] = {0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    const float px = (float)x - 0.5f * (float)(L.Lx - 1);
    unsigned sphase = 0u;   // bit s: parity of stage s's next completion (every thread)
    unsigned pending = 0u;  // lane 0 of warp 0: stages with copies it has not seen complete

    // March plane K (counted over all segments of the CTA) uses ring slot
    // K mod S, whose barrier's wait parity is (K / S) mod 2, and stage K mod NST.
    int K0 = 0;
    for (int j = 0; j < plan.nseg; ++j) {
        const Segment sg = plan.seg(j);
        const int Y0 = BATCH ? gi.y : sg.g * CY;
        const int y = Y0 + rank;
        const int zc0 = sg.z0, zc1 = sg.z1;
        const int n = zc1 - zc0;
        const bool down = sg.down;
        // k-th plane of the segment's march (k = 0 and n + 1 are the halo planes)
        auto plane_of = [&](int k) { return down ? zc1 - k : zc0 - 1 + k; };
        const HS hs(x, rank, Y0, L.Ly);
        const bool hin = hs.in && (!BATCH || hs.col < L.Lx);  // the halo node lies in the box
        const unsigned halo_ring = cluster_addr(ring_s, hs.rank);
        const unsigned halo_mbar = cluster_addr(mbar_s, hs.rank);
        const char* nbase = IO::base(src, x, y);
        const char* hbase;
        if constexpr (DEV) hbase = IO::base(src, hs.col, hs.in ? hs.y : 0);
        else hbase = IO::base_c(src, hs.col, hs.in ? hs.y : 0, hs.comp);
        const float py = (float)y - 0.5f * (float)(L.Ly - 1);

        // Staged variant: warp 0 fills a stage (lane 0 arms its mbarrier with
        // the bytes to come, then every lane issues its population rows); every
        // thread waits on the stage's mbarrier (bounded) before it reads the
        // plane.  Only the planes this segment reads and that lie in the box
        // are copied.
        auto plane_wanted = [&](int k) {
            const int p = plane_of(k);
            return k <= n + 1 && p >= 0 && p < L.Lz;
        };
        auto fill = [&](int k) {  // warp 0
            if (!plane_wanted(k)) return;
            const int st = (K0 + k) % NST;
            if (x == 0) {
                mbar_expect_tx(smbar_s + 8u * st, SP::BYTES);
                pending |= 1u << st;
            }
            __syncwarp();
            SP::issue(src, L, y, plane_of(k), stage_s + (unsigned)(st * SP::SMEM), smbar_s + 8u * st, x);
        };
        auto stage_wait = [&](int k) {
            const int st = (K0 + k) % NST;
            const unsigned par = (sphase >> st) & 1u;
            if (wait_bounded(smbar_s + 8u * st, par, false, kWaitNs)) pending &= ~(1u << st);
            else atomicOr(d_err, 4);
            sphase ^= 1u << st;
        };
        auto stage_ptr = [&](int k) { return stage + (size_t)((K0 + k) % NST) * (SP::SMEM / 4); };

        // Post-streaming densities of march plane k: the own node into row 0
        // of this CTA's ring and into the neighbours' rows -1 / +1; the
        // outer-halo share into the edge CTA's ring.  Ghost densities outside
        // the box.  Every CTA then expects TX_BYTES on its slot barrier.  The
        // staged variant also keeps the node's pulled populations in `carry`.
        // Staged variant: the outer-halo copies of march plane k into this
        // thread's prefetch slots (issued one march step before its
        // densities() call reads them, so a whole collision hides them).
        auto prefetch_halo = [&](int k) {
            const int p = plane_of(k);
            if (!(hs.cta && hin && k <= n + 1 && p >= 0 && p < L.Lz)) return;
            if constexpr (DEV) {
                if (hs.thr) HP::issue(planes(hbase, p, hs.col), once, halo_s, x);
            } else {
                HP::issue(planes(hbase, p, 0), once, halo_s, x);
            }
        };
        auto densities = [&](int k, typename SP::Raw* carry) {
            const int p = plane_of(k);
            const int sl = (K0 + k) & (S - 1);
            const bool in = p >= 0 && p < L.Lz;
            float ra = m.rho_b[0], rb = m.rho_b[1];
            // the outer-halo loads first, so that their latency overlaps the rest
            float hv = 0.f, ha = m.rho_b[0], hb = m.rho_b[1];
            if (hs.cta && in && hin) {
                if constexpr (PREF) {
                    cp_async_wait_all();  // this thread's copies of plane k (prefetch_halo)
                    if constexpr (DEV) {
                        if (hs.thr) HP::sum(halo_buf, x, ha, hb);
                    } else {
                        hv = HP::sum(halo_buf, x);
                    }
                } else if constexpr (DEV) {
                    if (hs.thr) IO::densities(planes(hbase, p, hs.col), once, ha, hb);
                } else {
                    hv = IO::template density<0>(planes(hbase, p, 0), once);
                }
            }
            if (in) {
                if constexpr (STAGED) {
                    stage_wait(k);
                    SP::load(stage_ptr(k), x, *carry, ra, rb);
                } else {
                    IO::densities(planes(nbase, p, x), keep, ra, rb);
                }
            }
            if constexpr (BATCH)
                if (!xact) {  // row padding: the ghost density, like the ring's x halo columns
                    ra = m.rho_b[0];
                    rb = m.rho_b[1];
                }
            ring[sl * FL::SLOT + RW + x + 1] = make_float2(ra, rb);
            const unsigned col = 8u * (unsigned)(sl * FL::SLOT + x + 1);  // row -1 of the slot, this column
            const unsigned mb = 8u * sl;
            if (rank > 0) st_async_f2(below_ring + col + 16u * RW, ra, rb, below_mbar + mb);
            if (rank < CY - 1) st_async_f2(above_ring + col, ra, rb, above_mbar + mb);
            if (hs.cta) {
                const unsigned hoff = 8u * (unsigned)(sl * FL::SLOT + (hs.row + 1) * RW + hs.col + 1);
                if constexpr (DEV) {
                    if (hs.thr) st_async_f2(halo_ring + hoff, ha, hb, halo_mbar + mb);
                } else {
                    // (a select, not an index: a run-time index into the
                    // kernel's parameters would copy them to local memory)
                    const float v = in && hin ? hv : (hs.comp ? m.rho_b[1] : m.rho_b[0]);
                    const float other = __shfl_xor_sync(0xffffffffu, v, 1);
                    if (hs.thr) st_async_f2(halo_ring + hoff, v, other, halo_mbar + mb);
                }
            }
            if (x == 0) mbar_expect_tx(mbar_s + mb, FL::TX_BYTES);
            // the slots are free again (their values went into the pushes above)
            if constexpr (PREF) prefetch_halo(k + 1);
        };
        // Wait (bounded) until the neighbour rows of march plane k have landed.
        auto wait_rows = [&](int k) {
            const unsigned par = (unsigned)((K0 + k) / S) & 1u;
            if (!wait_bounded(mbar_s + 8u * ((K0 + k) & (S - 1)), par, true, kWaitNs)) atomicOr(d_err, 4);
        };
        auto collide = [&](int k, const float (&f)[2][19], const float (&rs)[2]) {
            const int z = plane_of(k);
            const float2* rprev = ring + ((K0 + k - 1) & (S - 1)) * FL::SLOT + x + 1;
            const float2* rcur = ring + ((K0 + k) & (S - 1)) * FL::SLOT + x + 1;
            const float2* rnext = ring + ((K0 + k + 1) & (S - 1)) * FL::SLOT + x + 1;
            collide_node<TX, ST, MRT>(down ? rnext : rprev, rcur, down ? rprev : rnext, f, rs, m,
                                      IO::out(dst, L, x, y, z), cm, bad, px, py, (float)z - 0.5f * (float)(L.Lz - 1));
        };

        // The segment starts as every later march step does: a CTA pushes
        // plane k only after its wait for plane k - 1 (the ring argument of
        // FastLayout), and the first collision follows the __syncthreads of
        // the step that pushes plane 2.
        if constexpr (STAGED) {
            // Planes k + 1 .. k + 1 + NST are in the stages or in flight while
            // plane k is collided from the registers its density pass filled.
            typename SP::Raw cur, nxt;
            if (x < 32) {
                fence_proxy_async();  // a previous segment read the stages
#pragma unroll
                for (int k = 0; k < NST; ++k) fill(k);
            }
            if constexpr (PREF) prefetch_halo(0);
            densities(0, &nxt);
            __syncthreads();  // march plane 0 read by all: its stage takes plane NST
            if (x < 32) {
                fence_proxy_async();
                fill(NST);
            }
            wait_rows(0);
            densities(1, &cur);
            __syncthreads();
            if (x < 32) {
                fence_proxy_async();
                fill(NST + 1);
            }
            wait_rows(1);
            // one march step: the density pass of plane k + 1 into `next`,
            // the collision of plane k from `now`
            auto step = [&](int k, const typename SP::Raw& now, typename SP::Raw& next) {
                densities(k + 1, &next);
                __syncthreads();  // own row of plane k + 1 complete; its stage read by all
                if (x < 32) {
                    fence_proxy_async();
                    fill(k + 1 + NST);
                }
                wait_rows(k + 1);
                if (xact) {
                    float f[2][19], rs[2];
                    SP::unpack(now, f, rs);
                    collide(k, f, rs);
                }
            };
            if constexpr (DEV) {
                for (int k = 1; k <= n; ++k) {
                    step(k, cur, nxt);
                    cur = nxt;
                }
            } else {
                // two steps per trip, so that the carried registers swap
                // roles instead of being copied
                for (int k = 1; k <= n; k += 2) {
                    step(k, cur, nxt);
                    if (k + 1 <= n) step(k + 1, nxt, cur);
                }
            }
        } else {
            densities(0, nullptr);
            wait_rows(0);
            densities(1, nullptr);
            wait_rows(1);
            for (int k = 1; k <= n; ++k) {
                densities(k + 1, nullptr);
                // this node's populations for the collision, read while the
                // neighbour rows of plane k + 1 are in flight
                float f[2][19], rs[2];
                IO::populations(planes(nbase, plane_of(k), x), f, rs);
                __syncthreads();  // own row of plane k + 1 complete
                wait_rows(k + 1);
                if (xact) collide(k, f, rs);
                // Before a later plane reuses this plane's own-row slot, all
                // threads must be done reading it: the __syncthreads of the
                // next iterations (S - 1 march planes apart) order that.
            }
        }
        __syncthreads();  // the last plane's ring row and stage read by all before the next segment
        K0 += n + 2;
    }
    pdl_trigger();  // this CTA's march is done: the next step's ghost kernel may launch
    if (bad) atomicOr(d_err, bad);
    // staged variant: copies whose completion lane 0 of warp 0 did not observe
    // (a wait that gave up) are waited for again, bounded, before the CTA exits
    if constexpr (STAGED) {
        if (x == 0) {
            for (int st = 0; st < NST; ++st) {
                if (!((pending >> st) & 1u)) continue;
                wait_bounded(smbar_s + 8u * st, ((sphase >> st) & 1u) ^ 1u, false, kWaitNs);
            }
        }
    }
    // no CTA leaves while another may still address its shared memory
    cluster.sync();

    // centre-of-mass partials of the written state (fixed-order reduction)
    if constexpr (BATCH) {
        // the box's centre of mass, in the order of its CTAs (row, z chunk)
        const RowsBatchBox& B = bt.box[gi.x];
        centre_reduce(cm, bt.parts + 4LL * B.part0, (long long)(gi.y + rank) * gi.z + blockIdx.z, (unsigned)B.ctas,
                      bt.box_done + gi.x, bt.box_sums + 8LL * gi.x, bt.box_frame + 4LL * gi.x, red);
        rows_batch_count(bt);
    } else {
        centre_epilogue(cm, cp, red);
    }
}

// ---- Warp-specialised variant: loader and collider threads per row ----
//
// A CTA of 2 TX threads owns one row: threads 0 .. TX-1 (loaders) and
// TX .. 2 TX-1 (colliders) each take node x = t mod TX.  Per march plane k a
// loader reads the node's 38 pulled populations once, sums its densities into
// the ring (own row, the neighbour CTAs' rows by st.async, and its share of
// the rows outside the cluster, which every CTA of the cluster helps pull)
// and stages the populations in shared memory (NP planes in flight); the
// colliders collide plane k from shared memory once the densities of plane
// k + 1 have landed.  Loads of later planes are in flight while earlier
// planes are collided, on other warps, and no population is read twice.
//
// Barriers (all waits bounded): ring slot s completes when this CTA's TX
// loaders have written their own row of the slot's plane and the 2 TX x 8
// bytes of the rows -1 / +1 have landed; full[b] when the loaders have staged
// a plane in buffer b; empty[b] when the colliders are done with it.
//
// Ring slots: a loader pushes plane k's densities only after it has staged
// plane k - 1, which waited for its colliders to be done with plane
// k - 1 - NP = k - 3; those colliders finished plane k - 3 only after the CTAs
// next to them had pushed plane k - 2.  So a loader is at most two planes
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
    static constexpr int SLOT = 3 * RW;           // float2 per slot
    static constexpr int POPS = NP * 40 * TX;     // [buffer][s * 19 + i][x] floats, then rho* [2][x]
    static constexpr unsigned TX_BYTES = 2u * TX * 8u;
    static constexpr int NBAR = S + 2 * NP;
    static constexpr size_t bytes = sizeof(float2) * S * SLOT + sizeof(float) * POPS + sizeof(unsigned long long) * NBAR;
};

__device__ __forceinline__ bool ws_wait(unsigned mbar, unsigned parity, bool cluster_scope) {
    return wait_bounded(mbar, parity, cluster_scope, kWaitNs);
}

template <int TX, int CY, int MINB, typename ST>
__global__ void __launch_bounds__(2 * TX, MINB)
    k_stream_collide_ws(const ST* __restrict__ src, ST* __restrict__ dst, Layout L, FastModel m, int zchunk, int alt,
                        CentreParts cp, int* __restrict__ d_err) {
    using IO = RowIO<TX, ST>;
    using WL = WsLayout<TX, CY>;
    constexpr int RW = WL::RW, HN = WL::HN, S = WL::S, NP = WL::NP;
    constexpr bool DEV = is_dev_t<ST>::value;
    extern __shared__ __align__(128) float2 ring[];  // [S][3][RW], then [NP][38][TX] floats, then NBAR mbarriers
    float* pops = reinterpret_cast<float*>(ring + S * WL::SLOT);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(pops + WL::POPS);
    __shared__ float red[4 * ((2 * TX + 31) / 32)];

    cg::cluster_group cluster = cg::this_cluster();
    const int t = threadIdx.x;
    const bool loader = t < TX;
    const int x = loader ? t : t - TX;
    const int y = blockIdx.y;
    const int rank = (int)cluster.block_rank();  // == y % CY for cluster dims (1, CY, 1)
    const int Y0 = y - rank;
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, L.Lz);
    const int n = zc1 - zc0;
    const bool down = alt && (blockIdx.z & 1);
    auto plane_of = [&](int k) { return down ? zc1 - k : zc0 - 1 + k; };

    // outer-halo node of loader threads x < HN: the first half of them cover
    // row Y0 - 1 (kept in rank 0's ring row -1), the second half row Y0 + CY
    // (kept in rank CY - 1's ring row +1), TX / CY columns per CTA
    const bool hthr = loader && x < HN;
    const int hside = x < HN / 2 ? 0 : 1;
    const int hcol = rank * (HN / 2) + (x % (HN / 2));
    const int hy = hside ? Y0 + CY : Y0 - 1;
    const bool hin = hy >= 0 && hy < L.Ly;

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

    for (int e = t; e < S * WL::SLOT; e += 2 * TX) ring[e] = make_float2(m.rho_b[0], m.rho_b[1]);
    if (t == 0) {
        for (int k = 0; k < S; ++k) mbar_init(rbar_s + 8u * k, (unsigned)TX);
        for (int b = 0; b < NP; ++b) {
            mbar_init(full_s + 8u * b, (unsigned)TX);
            mbar_init(empty_s + 8u * b, (unsigned)TX);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();  // barriers initialised before any remote store arrives
    pdl_wait();      // (a no-op unless launched with the programmatic attribute)

    auto planes = [&](const char* b, int p, int col) {
        if constexpr (DEV) return IO::planes(b, L, p, col);
        else return IO::planes(b, L, p);
    };
    float cm[4] = {0.f, 0.f, 0.f, 0.f};
    int bad = 0;

    if (loader) {
        const char* nbase = IO::base(src, x, y);
        const char* hbase = IO::base(src, hcol, hin ? hy : 0);
        unsigned long long keep;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        unsigned ephase = 0u;  // bit b: parity of empty[b]'s next phase
        for (int k = 0; k <= n + 1; ++k) {
            const int p = plane_of(k);
            const bool in = p >= 0 && p < L.Lz;
            const bool staged = k >= 1 && k <= n;  // a plane this CTA collides
            float f[2][19], rs[2];
            float ra = m.rho_b[0], rb = m.rho_b[1];
            if (in) IO::load_all(planes(nbase, p, x), f, rs, ra, rb);
            float ha = m.rho_b[0], hb = m.rho_b[1];
            if (hthr && in && hin) IO::densities(planes(hbase, p, hcol), keep, ha, hb);  // read again by its own CTA
            // densities first: the colliders of plane k - 1 wait for them
            const int slot = k % S;
            const unsigned mb = 8u * slot;
            const unsigned col = 8u * (unsigned)(slot * WL::SLOT + x + 1);
            ring[slot * WL::SLOT + RW + x + 1] = make_float2(ra, rb);
            if (rank > 0) st_async_f2(below_ring + col + 16u * RW, ra, rb, below_mbar + mb);
            if (rank < CY - 1) st_async_f2(above_ring + col, ra, rb, above_mbar + mb);
            if (hthr)
                st_async_f2(halo_ring + 8u * (unsigned)(slot * WL::SLOT + (hside ? 2 : 0) * RW + hcol + 1), ha, hb,
                            halo_mbar + mb);
            if (x == 0) mbar_expect_tx(rbar_s + mb, WL::TX_BYTES);  // this thread's arrival, and the bytes
            else mbar_arrive(rbar_s + mb);
            // then the populations, into a buffer the colliders are done with
            // (plane k - NP); they wait in registers meanwhile
            if (staged) {
                const int b = (k - 1) % NP;
                if (k - 1 >= NP) {
                    if (!ws_wait(empty_s + 8u * b, (ephase >> b) & 1u, false)) atomicOr(d_err, 4);
                    ephase ^= 1u << b;
                }
                float* P = pops + (size_t)b * 40 * TX;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
#pragma unroll
                    for (int i = 0; i < 19; ++i) P[(s * 19 + i) * TX + x] = f[s][i];
                    P[(38 + s) * TX + x] = rs[s];
                }
                mbar_arrive(full_s + 8u * b);
            }
        }
    } else {
        const float px = (float)x - 0.5f * (float)(L.Lx - 1), py = (float)y - 0.5f * (float)(L.Ly - 1);
        unsigned rphase = 0u, fphase = 0u;  // bit s: parity of ring slot s's / full[s]'s next phase
        auto wait_ring = [&](int k) {
            const int slot = k % S;
            if (!ws_wait(rbar_s + 8u * slot, (rphase >> slot) & 1u, true)) atomicOr(d_err, 4);
            rphase ^= 1u << slot;
        };
        wait_ring(0);
        wait_ring(1);
        for (int k = 1; k <= n; ++k) {
            wait_ring(k + 1);
            const int b = (k - 1) % NP;
            if (!ws_wait(full_s + 8u * b, (fphase >> b) & 1u, false)) atomicOr(d_err, 4);
            fphase ^= 1u << b;
            float f[2][19], rs[2];
            const float* P = pops + (size_t)b * 40 * TX;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
#pragma unroll
                for (int i = 0; i < 19; ++i) f[s][i] = P[(s * 19 + i) * TX + x];
                rs[s] = P[(38 + s) * TX + x];
            }
            const int z = plane_of(k);
            const float2* rprev = ring + ((k - 1) % S) * WL::SLOT + x + 1;
            const float2* rcur = ring + (k % S) * WL::SLOT + x + 1;
            const float2* rnext = ring + ((k + 1) % S) * WL::SLOT + x + 1;
            collide_node<TX, ST>(down ? rnext : rprev, rcur, down ? rprev : rnext, f, rs, m, IO::out(dst, L, x, y, z),
                                 cm, bad, px, py, (float)z - 0.5f * (float)(L.Lz - 1));
            // the buffer may take plane k + NP (released after the collision,
            // so that the populations can stay in shared memory until used)
            mbar_arrive(empty_s + 8u * b);
        }
    }
    pdl_trigger();  // this CTA's march is done: the next step's ghost kernel may launch
    if (bad) atomicOr(d_err, bad);
    // no CTA leaves while another may still address its shared memory
    cluster.sync();

    // centre-of-mass partials of the written state (fixed-order reduction)
    centre_epilogue(cm, cp, red);
}

// Resident CTAs per SM asked of the compiler (it sets the register budget)
// for the direct-load variant, per row width; the staged variant holds two
// plane images and the halo slots (float32: about 64 KB of shared memory at
// TX = 128, 105 KB at 256; 16-bit storage: 42 KB and 82 KB), so 3 CTAs of
// 128 threads or 2 of 256 fit per SM.
template <int TX, bool STAGED>
constexpr int row_min_blocks() {
    if (STAGED) return TX >= 256 ? 2 : 512 / TX;
    return TX == 32 ? LBM_ROWS_MINB_32
                    : (TX == 64 ? LBM_ROWS_MINB_64 : (TX == 128 ? LBM_ROWS_MINB_128 : LBM_ROWS_MINB_256));
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
    const FastModel fm = fast_model(m);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, L.Ly, nchunks);
    cfg.blockDim = dim3(TX, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    // (no programmatic-serialization attribute: measured at 128^3, CTAs that
    // start while the ghost kernel runs are placed unevenly over the SMs and
    // the step took 212 us instead of 133 us)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CY;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, (const S*)src, (S*)dst, L, fm, zchunk, (int)LBM_ROWS_ALTERNATE, cp, d_err,
                              RowsBatch{});
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

constexpr int kRowCluster = kRowClusterRows;

// The batched ensemble's launch (RowsBatch): float32, staged, rows of width
// kRowsBatchWidth.
using RowsBatchKernel = StagedLayout<kRowsBatchWidth, kRowCluster, float>;
constexpr size_t rows_batch_bytes() { return RowsBatchKernel::bytes; }

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
// variant (2 TX threads, about 95 KB of shared memory at TX = 128: two CTAs
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
    const FastModel fm = fast_model(m);
    cfg.gridDim = dim3(1, L.Ly, (L.Lz + zchunk - 1) / zchunk);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, k, (const S*)src, (S*)dst, L, fm, zchunk, (int)LBM_ROWS_ALTERNATE, cp, d_err);
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

// The kernels address the layout with the compile-time geometry of RowGeo;
// the layout of the context must be the one make_layout gives for Lx.
template <int TX, typename S>
bool geometry_matches(const Layout& L) {
    using G = RowGeo<TX, S>;
    return L.x0 == G::X0 && L.pitch == G::PITCH && L.row == (long long)G::ROW;
}

// Dispatch on the row width, the storage type and the variant.
cudaError_t rows_dispatch(int prec, int variant, bool query, const void* src, void* dst, const Layout& L,
                          const Model& m, int zchunk, CentreParts cp, int* d_err, cudaStream_t s, int* resident) {
#define LBM_ROWS_TX(TXV)                                                                                         \
    if (L.Lx == TXV) {                                                                                           \
        if (prec == kFP32 && geometry_matches<TXV, float>(L))                                                    \
            return rows_variant<TXV, float>(variant, query, src, dst, L, m, zchunk, cp, d_err, s, resident);      \
        if (prec == kFP16Dev && geometry_matches<TXV, Dev<__half>>(L))                                           \
            return rows_variant<TXV, Dev<__half>>(variant, query, src, dst, L, m, zchunk, cp, d_err, s, resident); \
        if (prec == kBF16Dev && geometry_matches<TXV, Dev<__nv_bfloat16>>(L))                                    \
            return rows_variant<TXV, Dev<__nv_bfloat16>>(variant, query, src, dst, L, m, zchunk, cp, d_err, s,    \
                                                         resident);                                              \
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

Layout make_layout_rows(int Lx, int Ly, int Lz) {
    using G = RowGeo<kRowsBatchWidth, float>;
    Layout L = make_layout(Lx, Ly, Lz, kFP32);  // x0 is G::X0 for float32
    L.pitch = G::PITCH;
    L.row = (long long)G::ROW;
    L.plane = (long long)L.ny * L.row;
    L.total = (long long)L.nz * L.plane;
    return L;
}

bool rows_batch_applies(int Lx, int Ly, int Lz) {
    return Lx >= 2 && Lx <= kRowsBatchWidth && Ly >= kRowCluster && Ly % kRowCluster == 0 && Lz >= 2;
}

size_t rows_batch_smem() { return rows_batch_bytes(); }

cudaError_t launch_rows_batch(const RowsBatch& rb, int groups, int max_chunks, int zchunk, const Model& m,
                              int* d_err, cudaStream_t s) {
    constexpr int TX = kRowsBatchWidth, CY = kRowCluster;
    if (groups < 1 || (long long)groups * CY > 65535 || max_chunks < 1 || max_chunks > 65535 || zchunk < 1)
        return cudaErrorInvalidValue;
    auto k = k_stream_collide_rows<TX, CY, row_min_blocks<TX, true>(), float, true, false, true>;
    const size_t smem = rows_batch_bytes();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const FastModel fm = fast_model(m);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, groups * CY, max_chunks);
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
    const Layout L0 = {};
    return cudaLaunchKernelEx(&cfg, k, (const float*)nullptr, (float*)nullptr, L0, fm, zchunk,
                              (int)LBM_ROWS_ALTERNATE, CentreParts{}, d_err, rb);
}

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
