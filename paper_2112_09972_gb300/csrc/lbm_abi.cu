// Host side of the C ABI declared in include/lbm.h: parameter validation,
// device memory, the gradient knot table, launch orchestration, profiling
// events and checkpoints.  Every entry point catches its own failures and
// returns an lbm_status; nothing throws across the interface.

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbmgb;

struct lbm_ctx {
    int box[3];
    double R, xi, rho_hi, rho_lo;
    Model model;
    int prec;       // lbm_precision: 0 fp64, 1 fp32, 2 / 3 16-bit deviations (fp16 / bf16)
    int elem;       // bytes per layout element (8, 4, or the 2-byte unit of deviation storage)
    Layout L;
    Shape shape;
    int device, num_sms;
    cudaStream_t stream;
    bool own_stream;
    void* f[2];
    int cur;                // buffer holding the current post-collision populations
    bool initialised;       // populations hold a state (lazy init on first use)
    int64_t step;           // steps taken; step n uses A(t_n = n)
    int* d_err;             // latched device error bits: 1 non-finite, 2 Mach, 4 wait timeout
    int* h_err;             // pinned mirror
    int latched;            // latched status returned by later calls
    // gradient knots (host); A(t_n) is evaluated here and passed by value
    std::vector<double> kt, kA;
    // per-CTA droplet moments of the current state (frame origin of the next step)
    CentreParts centre;
    // reduction scratch
    double* d_partials;
    int red_blocks;
    double* d_result;  // 32 doubles
    double* h_result;  // pinned
    // profiling: events around the launches of every prof-th step (0: off)
    int prof;
    std::vector<cudaEvent_t> ev[2];
    int64_t prof_n[2];
};

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (e == cudaErrorMemoryAllocation) return LBM_ENOMEM;
    return LBM_ECUDA;
}

#define LBM_TRY(expr)                               \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

// Flat-interface minority density: ln(h/l) = G (h - l) with l < 1/G.
double coexistence_lo(double G, double h) {
    if (G * h <= 1.0) return -1.0;
    double a = 1e-300, b = 1.0 / G;  // f(a) > 0 > f(b)
    auto fn = [&](double l) { return std::log(h / l) - G * (h - l); };
    for (int it = 0; it < 400; ++it) {
        const double m = (a > 0 && b / a > 4.0) ? std::sqrt(a * b) : 0.5 * (a + b);
        if (fn(m) > 0.0) a = m; else b = m;
        if (b - a <= 1e-16 * b) break;
    }
    return 0.5 * (a + b);
}

// A(t) from the knot table: linear between knots, constant outside.
Grad gradient_at(const lbm_ctx* c, double t) {
    Grad g;
    const size_t n = c->kt.size();
    if (n == 0) {
        for (int j = 0; j < 9; ++j) g.a[j] = 0.0;
        return g;
    }
    if (t <= c->kt[0]) {
        for (int j = 0; j < 9; ++j) g.a[j] = c->kA[j];
        return g;
    }
    if (t >= c->kt[n - 1]) {
        for (int j = 0; j < 9; ++j) g.a[j] = c->kA[9 * (n - 1) + j];
        return g;
    }
    // first knot with t_k > t
    const size_t hi = (size_t)(std::upper_bound(c->kt.begin(), c->kt.end(), t) - c->kt.begin());
    const size_t lo = hi - 1;
    const double w = (t - c->kt[lo]) / (c->kt[hi] - c->kt[lo]);
    for (int j = 0; j < 9; ++j) {
        const double a = c->kA[9 * lo + j], b = c->kA[9 * hi + j];
        g.a[j] = a + w * (b - a);
    }
    return g;
}

int check_latched(lbm_ctx* c) {
    if (c->latched) return c->latched;
    // A Mach violation at the boundary is the usual cause of a later
    // non-finite density, so it is reported first.
    int bits = *c->h_err;
    if (bits & 4) c->latched = LBM_ETIMEOUT;
    else if (bits & 2) c->latched = LBM_EMACH;
    else if (bits & 1) c->latched = LBM_ENONFINITE;
    return c->latched;
}

// Synchronise and fold the device error word into the latched status.
int sync_and_check(lbm_ctx* c) {
    LBM_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LBM_TRY(cudaStreamSynchronize(c->stream));
    return check_latched(c);
}

int lazy_init(lbm_ctx* c) {
    if (c->initialised) return LBM_OK;
    LBM_TRY(launch_init(c->prec, c->f[c->cur], c->L, c->R, c->xi, c->rho_hi, c->rho_lo, gradient_at(c, 0.0), c->stream));
    LBM_TRY(launch_centre(c->prec, c->f[c->cur], c->L, c->centre, c->stream));
    c->initialised = true;
    return LBM_OK;
}

int set_device(lbm_ctx* c) { return cuda_status(cudaSetDevice(c->device)); }

bool finite_all(const double* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

bool gradient_ok(const double* A) {
    if (!finite_all(A, 9)) return false;
    double mx = 1.0;
    for (int j = 0; j < 9; ++j) mx = std::max(mx, std::fabs(A[j]));
    return std::fabs(A[0] + A[4] + A[8]) <= 1e-12 * mx;
}

// 64-bit FNV-1a over a byte range.
uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ULL) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    return h;
}

// Doubles of the population block of a checkpoint: the float64 populations,
// or the raw device buffer for deviation storage (whose float64 round trip
// would not be bit-exact).
size_t ckpt_pop_words(const lbm_ctx* c) {
    if (is_dev(c->prec)) return ((size_t)c->L.total * c->elem + 7) / 8;
    return 38ull * c->box[0] * c->box[1] * c->box[2];
}

struct CkptHeader {
    char magic[8];
    int32_t version, box[3], prec, bc;
    double R, xi, rho_hi, rho_lo, tau[2], G, rho_b[2];
    int64_t step, nknots, npop, ncentre;
};

}  // namespace

extern "C" {

void lbm_opts_default(lbm_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = LBM_FP32;
    o->bc = LBM_BC_GHOST_LINEAR;
    o->rho_hi = 0.0;
    o->rho_lo = 0.0;
    o->xi = 0.0;
    o->mach_limit = 0.0;
    o->cuda_stream = nullptr;
    o->device = -1;
    o->tile_y = 0;
    o->z_chunk = 0;
}

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "out of memory";
        case LBM_ECUDA: return "CUDA runtime error";
        case LBM_ENONFINITE: return "non-finite density on the device";
        case LBM_EMACH: return "ghost velocity above the Mach guard";
        case LBM_ETIMEOUT: return "bounded device wait timed out";
        case LBM_EIO: return "checkpoint file missing, short or corrupt";
        default: return "unknown status";
    }
}

int lbm_selftest_wait(int64_t limit_ns, int32_t arrive, int32_t device) {
    if (limit_ns < 1000 || limit_ns > 10000000000LL || (arrive != 0 && arrive != 1)) return LBM_EINVAL;
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return LBM_ECUDA;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LBM_ECUDA;
    int gave_up = 0;
    const cudaError_t e = launch_wait_selftest((unsigned long long)limit_ns, arrive, s, &gave_up);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return LBM_ECUDA;
    return gave_up ? LBM_ETIMEOUT : LBM_OK;
}

int lbm_create(lbm_ctx** out, const int32_t box[3], double R, const double visc[2], double G, const lbm_opts* opts) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!box || !visc) return LBM_EINVAL;
    lbm_opts o;
    lbm_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != LBM_FP64 && o.precision != LBM_FP32 && o.precision != LBM_FP16_DEV &&
        o.precision != LBM_BF16_DEV)
        return LBM_EINVAL;
    if (o.bc != LBM_BC_GHOST_LINEAR && o.bc != LBM_BC_PERIODIC_TEST) return LBM_EINVAL;
    if (o.frame != LBM_FRAME_DROPLET && o.frame != LBM_FRAME_BOX) return LBM_EINVAL;
    if (o.row_variant < 0 || o.row_variant > 3) return LBM_EINVAL;
    if (o.collision != LBM_COLLISION_BGK && o.collision != LBM_COLLISION_MRT) return LBM_EINVAL;
    double mrt_rates[5] = {1.19, 1.4, 1.2, 1.4, 1.98};  // d'Humieres et al. (2002)
    for (int k = 0; k < 5; ++k) {
        if (o.mrt_rates[k] > 0.0) mrt_rates[k] = o.mrt_rates[k];
        if (!(mrt_rates[k] > 0.0 && mrt_rates[k] < 2.0)) return LBM_EINVAL;
    }
    for (int a = 0; a < 3; ++a)
        if (box[a] < 4 || box[a] > 4096) return LBM_EINVAL;
    const int mn = std::min(box[0], std::min(box[1], box[2]));
    if (!(R >= 0.0) || !std::isfinite(R)) return LBM_EINVAL;
    if (o.bc == LBM_BC_GHOST_LINEAR && 2.0 * R > mn - 2) return LBM_EINVAL;
    if (!(visc[0] > 0.0) || !(visc[1] > 0.0) || !std::isfinite(visc[0]) || !std::isfinite(visc[1])) return LBM_EINVAL;
    if (!(G >= 0.0) || !std::isfinite(G)) return LBM_EINVAL;
    const double hi = o.rho_hi > 0.0 ? o.rho_hi : 1.0;
    double lo = o.rho_lo;
    if (!(lo > 0.0)) {
        lo = coexistence_lo(G, hi);
        if (!(lo > 0.0)) lo = hi;  // no phase separation: a uniform mixture
    }
    if (!(lo <= hi) || !std::isfinite(lo) || !std::isfinite(hi)) return LBM_EINVAL;
    const double xi = o.xi > 0.0 ? o.xi : 1.0;
    const double mach = o.mach_limit > 0.0 ? o.mach_limit : 0.9;

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete c; return LBM_ECUDA; }
    c->device = dev;
    if (cudaSetDevice(dev) != cudaSuccess) { delete c; return LBM_ECUDA; }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int a = 0; a < 3; ++a) c->box[a] = box[a];
    c->R = R; c->xi = xi; c->rho_hi = hi; c->rho_lo = lo;
    c->model.tau[0] = 3.0 * visc[0] + 0.5;  // Eq. 10
    c->model.tau[1] = 3.0 * visc[1] + 0.5;
    c->model.G = G;
    c->model.rho_b[0] = lo;  // the droplet component is the minority at the boundary
    c->model.rho_b[1] = hi;
    c->model.periodic = o.bc == LBM_BC_PERIODIC_TEST;
    c->model.mach2 = mach * mach / 3.0;
    c->model.droplet_frame = o.frame == LBM_FRAME_DROPLET;
    c->model.mrt = o.collision == LBM_COLLISION_MRT;
    for (int k = 0; k < 5; ++k) c->model.mrt_rates[k] = mrt_rates[k];
    c->prec = o.precision;
    c->elem = elem_bytes_of(c->prec);
    c->L = make_layout(box[0], box[1], box[2], c->prec);
    c->shape = choose_shape(c->L, c->prec, o.bc == LBM_BC_PERIODIC_TEST, c->model.mrt, o.tile_y, o.z_chunk,
                            o.row_variant, c->num_sms);
    c->cur = 0;
    c->stream = (cudaStream_t)o.cuda_stream;
    c->own_stream = false;
    int st = LBM_OK;
    if (!c->stream) {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return LBM_ECUDA; }
        c->own_stream = true;
    }
    c->red_blocks = std::max(moments_blocks(c->L, c->num_sms), 1);
    const size_t bytes = (size_t)c->L.total * c->elem;
    cudaError_t e = cudaMalloc(&c->f[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->f[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_partials, sizeof(double) * 10 * c->red_blocks);
    c->centre.n = (int)(c->shape.grid.x * c->shape.grid.y * c->shape.grid.z);
    // partials, the 8 sums, the counter (16 bytes), the float32 frame origin (16 bytes)
    const size_t centre_bytes = sizeof(double) * (4 * (size_t)c->centre.n + 8) + 32;
    if (e == cudaSuccess) e = cudaMalloc(&c->centre.p, centre_bytes);
    if (e == cudaSuccess) {
        c->centre.sum = c->centre.p + 4 * c->centre.n;
        c->centre.counter = (unsigned*)(c->centre.sum + 8);
        c->centre.frame = (float*)(c->centre.sum + 10);
        e = cudaMemsetAsync(c->centre.p, 0, centre_bytes, c->stream);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_result, sizeof(double) * 32);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_result, sizeof(double) * 32);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(int));
    // Zero both buffers once: ghost entries that no direction reads stay defined.
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[0], 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[1], 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        st = cuda_status(e);
        lbm_destroy(c);
        return st;
    }
    *c->h_err = 0;
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->d_err);
    cudaFree(c->d_partials);
    cudaFree(c->centre.p);
    cudaFree(c->d_result);
    if (c->h_result) cudaFreeHost(c->h_result);
    if (c->h_err) cudaFreeHost(c->h_err);
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t ev : c->ev[k]) cudaEventDestroy(ev);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbm_set_gradient_table(lbm_ctx* c, const int64_t* t, const double* A, int64_t n) {
    if (!c || n < 0 || (n > 0 && (!t || !A))) return LBM_EINVAL;
    double last = c->kt.empty() ? -INFINITY : c->kt.back();
    for (int64_t k = 0; k < n; ++k) {
        if (!gradient_ok(A + 9 * k)) return LBM_EINVAL;
        if (!((double)t[k] > last)) return LBM_EINVAL;
        last = (double)t[k];
    }
    for (int64_t k = 0; k < n; ++k) {
        c->kt.push_back((double)t[k]);
        c->kA.insert(c->kA.end(), A + 9 * k, A + 9 * k + 9);
    }
    return LBM_OK;
}

int lbm_set_gradient(lbm_ctx* c, const double A[9], int64_t t) { return lbm_set_gradient_table(c, &t, A, 1); }

int lbm_step(lbm_ctx* c, int64_t n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (c->latched) return c->latched;
    int st = set_device(c);
    if (st) return st;
    if ((st = lazy_init(c))) return st;
    for (int64_t k = 0; k < n; ++k) {
        void* src = c->f[c->cur];
        void* dst = c->f[1 - c->cur];
        const bool timed = c->prof > 0 && (c->step % c->prof) == 0;
        const Grad A = gradient_at(c, (double)c->step);
        if (!c->model.periodic) {
            cudaEvent_t a = nullptr, b = nullptr;
            if (timed) {
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                cudaEventRecord(a, c->stream);
            }
            LBM_TRY(launch_ghost(c->prec, src, c->L, c->model, A, c->centre, c->d_err, c->stream));
            if (timed) {
                cudaEventRecord(b, c->stream);
                c->ev[1].push_back(a);
                c->ev[1].push_back(b);
            }
        }
        cudaEvent_t a = nullptr, b = nullptr;
        if (timed) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, c->stream);
        }
        LBM_TRY(launch_stream_collide(c->prec, src, dst, c->L, c->model, c->shape, A, c->centre, c->d_err, c->stream));
        if (timed) {
            cudaEventRecord(b, c->stream);
            c->ev[0].push_back(a);
            c->ev[0].push_back(b);
        }
        c->cur = 1 - c->cur;
        c->step += 1;
    }
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    int st = set_device(c);
    if (st) return st;
    return sync_and_check(c);
}

int lbm_moments(lbm_ctx* c, double m[10]) {
    if (!c || !m) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    LBM_TRY(launch_moments(c->prec, c->f[c->cur], c->L, c->d_partials, c->red_blocks, c->d_result, c->stream));
    LBM_TRY(cudaMemcpyAsync(c->h_result, c->d_result, sizeof(double) * 26, cudaMemcpyDeviceToHost, c->stream));
    if ((st = sync_and_check(c))) return st;
    memcpy(m, c->h_result, sizeof(double) * 10);
    return LBM_OK;
}

int lbm_deformation(lbm_ctx* c, double* D, double axes[9], double lambda[3], double centre[3]) {
    if (!c || !D) return LBM_EINVAL;
    double m[10];
    int st = lbm_moments(c, m);
    if (st) return st;
    *D = c->h_result[10];
    if (axes) memcpy(axes, c->h_result + 11, sizeof(double) * 9);
    if (lambda) memcpy(lambda, c->h_result + 20, sizeof(double) * 3);
    if (centre) memcpy(centre, c->h_result + 23, sizeof(double) * 3);
    return LBM_OK;
}

int lbm_get_fields(lbm_ctx* c, double* rho_A, double* rho_B, double* u) {
    if (!c) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    const size_t N = (size_t)c->box[0] * c->box[1] * c->box[2];
    double* d = nullptr;
    LBM_TRY(cudaMallocAsync(&d, sizeof(double) * 5 * N, c->stream));
    cudaError_t e = launch_fields(c->prec, c->f[c->cur], c->L, c->model, d, d + N, d + 2 * N, c->stream);
    if (e == cudaSuccess && rho_A) e = cudaMemcpyAsync(rho_A, d, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && rho_B) e = cudaMemcpyAsync(rho_B, d + N, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, d + 2 * N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return sync_and_check(c);
}

int lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    const size_t E = 38ull * c->box[0] * c->box[1] * c->box[2];
    double* d = nullptr;
    LBM_TRY(cudaMallocAsync(&d, sizeof(double) * E, c->stream));
    cudaError_t e = launch_pack(c->prec, c->f[c->cur], c->L, c->model, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, sizeof(double) * E, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return sync_and_check(c);
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return LBM_EINVAL;
    const size_t E = 38ull * c->box[0] * c->box[1] * c->box[2];
    if (!finite_all(f, (int)std::min<size_t>(E, (size_t)INT32_MAX))) return LBM_EINVAL;
    int st = set_device(c);
    if (st) return st;
    double* d = nullptr;
    // deviation storage needs the float32 densities of all nodes first
    const size_t scratch = is_dev(c->prec) ? 2 * E / 38 : 0;
    LBM_TRY(cudaMallocAsync(&d, sizeof(double) * E + sizeof(float) * scratch, c->stream));
    cudaError_t e = cudaMemcpyAsync(d, f, sizeof(double) * E, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_unpack(c->prec, c->f[c->cur], c->L, c->model, d, scratch ? (float*)(d + E) : nullptr, c->stream);
    if (e == cudaSuccess) e = launch_centre(c->prec, c->f[c->cur], c->L, c->centre, c->stream);
    cudaFreeAsync(d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    c->initialised = true;
    return LBM_OK;
}

int lbm_checksums(lbm_ctx* c, double mass[2], double mom[3]) {
    if (!c) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    LBM_TRY(launch_checksums(c->prec, c->f[c->cur], c->L, c->model, c->d_partials, c->red_blocks, c->d_result,
                             c->stream));
    LBM_TRY(cudaMemcpyAsync(c->h_result, c->d_result, sizeof(double) * 5, cudaMemcpyDeviceToHost, c->stream));
    if ((st = sync_and_check(c))) return st;
    if (mass) memcpy(mass, c->h_result, sizeof(double) * 2);
    if (mom) memcpy(mom, c->h_result + 2, sizeof(double) * 3);
    return LBM_OK;
}

int lbm_components(lbm_ctx* c, double threshold, int64_t min_nodes, int32_t* count, int64_t* sizes,
                   int32_t max_sizes) {
    if (!c || !count || !std::isfinite(threshold) || max_sizes < 0 || (max_sizes > 0 && !sizes)) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    const long long N = (long long)c->box[0] * c->box[1] * c->box[2];
    if (N > INT32_MAX) return LBM_EINVAL;
    // scratch: labels and sizes (N ints each), the change flag and root counter,
    // and the root sizes (N 64-bit)
    char* d = nullptr;
    const size_t bytes = sizeof(int) * (2 * N + 2) + sizeof(long long) * N + 16;
    LBM_TRY(cudaMallocAsync((void**)&d, bytes, c->stream));
    int* label = (int*)d;
    int* size = label + N;
    int* flags = size + N;  // [0] changed, [1] root count
    long long* out = (long long*)(((uintptr_t)(flags + 2) + 15) & ~(uintptr_t)15);
    int h_flags[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(size, 0, sizeof(int) * (N + 2), c->stream);
    if (e == cudaSuccess) e = launch_cc_init(c->prec, c->f[c->cur], c->L, threshold, label, c->stream);
    // propagation sweeps until no label changes; bounded (a component's
    // labels settle within its node count of sweeps)
    const long long max_sweeps = std::min<long long>(N + 8, 1LL << 22);
    bool converged = false;
    for (long long it = 0; e == cudaSuccess && it < max_sweeps; it += 4) {
        e = cudaMemsetAsync(flags, 0, sizeof(int), c->stream);
        for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = launch_cc_sweep(c->L, c->model.periodic, label, flags, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess && h_flags[0] == 0) {
            converged = true;
            break;
        }
    }
    std::vector<long long> roots;
    if (e == cudaSuccess && converged) e = launch_cc_sizes(c->L, label, size, flags + 1, out, (int)N, c->stream);
    if (e == cudaSuccess && converged) e = cudaMemcpyAsync(h_flags, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && converged) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && converged) {
        try { roots.resize((size_t)h_flags[1]); } catch (...) { e = cudaErrorMemoryAllocation; }
        if (e == cudaSuccess && !roots.empty())
            e = cudaMemcpyAsync(roots.data(), out, sizeof(long long) * roots.size(), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    cudaFreeAsync(d, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (!converged) return LBM_ETIMEOUT;
    std::vector<long long> kept;
    for (long long v : roots)
        if (v >= min_nodes) kept.push_back(v);
    std::sort(kept.begin(), kept.end(), [](long long a, long long b) { return a > b; });
    *count = (int32_t)kept.size();
    for (int32_t k = 0; k < max_sizes; ++k) sizes[k] = k < (int32_t)kept.size() ? kept[k] : 0;
    return sync_and_check(c);
}

int lbm_surface_deformation(lbm_ctx* c, double* D_lbm, double* area, double* volume) {
    if (!c || !D_lbm) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    const long long N = (long long)c->box[0] * c->box[1] * c->box[2];
    double* phi = nullptr;
    LBM_TRY(cudaMallocAsync(&phi, sizeof(double) * N, c->stream));
    cudaError_t e = launch_surface_stats(c->prec, c->f[c->cur], c->L, phi, c->d_partials, c->red_blocks, c->d_result,
                                         c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_result, c->d_result, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(phi, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if ((st = sync_and_check(c))) return st;
    const double sum = c->h_result[0], lo = c->h_result[1], hi = c->h_result[2], grad = c->h_result[3];
    const double span = hi - lo;
    if (!(span > 0.0)) {  // a uniform state has no interface
        *D_lbm = 0.0;
        if (area) *area = 0.0;
        if (volume) *volume = 0.0;
        return LBM_OK;
    }
    // Eq. 17: Omega = sum |grad phi| / span (co-area), V = sum (phi - min) / span
    const double A = grad / span, V = (sum - (double)N * lo) / span;
    const double A0 = std::cbrt(36.0 * M_PI * V * V);
    *D_lbm = std::sqrt(std::max(0.0, 1.0 - A0 / A));
    if (area) *area = A;
    if (volume) *volume = V;
    return LBM_OK;
}

int lbm_reinject_mass(lbm_ctx* c, double target, double* factor) {
    if (!c || !(target > 0.0) || !std::isfinite(target)) return LBM_EINVAL;
    if (is_dev(c->prec)) return LBM_EINVAL;
    int st = set_device(c);
    if (st || (st = lazy_init(c))) return st;
    LBM_TRY(launch_mass_split(c->prec, c->f[c->cur], c->L, c->d_partials, c->red_blocks, c->d_result, c->stream));
    LBM_TRY(cudaMemcpyAsync(c->h_result, c->d_result, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    if ((st = sync_and_check(c))) return st;
    const double m_in = c->h_result[0], m_out = c->h_result[1];
    if (!(m_in > 0.0)) return LBM_EINVAL;  // no droplet phase to rescale
    const double k = (target - m_out) / m_in;
    if (!(k > 0.0) || !std::isfinite(k)) return LBM_EINVAL;
    LBM_TRY(launch_reinject(c->prec, c->f[c->cur], c->L, k, c->stream));
    LBM_TRY(launch_centre(c->prec, c->f[c->cur], c->L, c->centre, c->stream));
    if (factor) *factor = k;
    return sync_and_check(c);
}

int lbm_get_step(lbm_ctx* c, int64_t* step) {
    if (!c || !step) return LBM_EINVAL;
    *step = c->step;
    return LBM_OK;
}

int lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    const size_t E = ckpt_pop_words(c);
    std::vector<double> pop;
    try { pop.resize(E, 0.0); } catch (...) { return LBM_ENOMEM; }
    int st;
    if (is_dev(c->prec)) {
        if ((st = set_device(c)) || (st = lazy_init(c))) return st;
        LBM_TRY(cudaMemcpyAsync(pop.data(), c->f[c->cur], (size_t)c->L.total * c->elem, cudaMemcpyDeviceToHost,
                                c->stream));
        if ((st = sync_and_check(c))) return st;
    } else if ((st = lbm_get_populations(c, pop.data()))) {
        return st;
    }
    // the frame origin of the next step is part of the state
    std::vector<double> cparts((size_t)4 * c->centre.n + 8);
    LBM_TRY(cudaMemcpy(cparts.data(), c->centre.p, sizeof(double) * cparts.size(), cudaMemcpyDeviceToHost));
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "LBMGB300", 8);
    h.version = 2;  // 2: row-interleaved device layout (raw buffers of deviation storage)
    for (int a = 0; a < 3; ++a) h.box[a] = c->box[a];
    h.prec = c->prec;
    h.bc = c->model.periodic;
    h.R = c->R; h.xi = c->xi; h.rho_hi = c->rho_hi; h.rho_lo = c->rho_lo;
    h.tau[0] = c->model.tau[0]; h.tau[1] = c->model.tau[1];
    h.G = c->model.G;
    h.rho_b[0] = c->model.rho_b[0]; h.rho_b[1] = c->model.rho_b[1];
    h.step = c->step;
    h.nknots = (int64_t)c->kt.size();
    h.npop = (int64_t)E;
    h.ncentre = (int64_t)c->centre.n;
    uint64_t sum = fnv1a(&h, sizeof(h));
    sum = fnv1a(c->kt.data(), sizeof(double) * c->kt.size(), sum);
    sum = fnv1a(c->kA.data(), sizeof(double) * c->kA.size(), sum);
    sum = fnv1a(pop.data(), sizeof(double) * E, sum);
    sum = fnv1a(cparts.data(), sizeof(double) * cparts.size(), sum);
    FILE* fp = fopen(path, "wb");
    if (!fp) return LBM_EIO;
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
    ok = ok && fwrite(c->kt.data(), sizeof(double), c->kt.size(), fp) == c->kt.size();
    ok = ok && fwrite(c->kA.data(), sizeof(double), c->kA.size(), fp) == c->kA.size();
    ok = ok && fwrite(pop.data(), sizeof(double), E, fp) == E;
    ok = ok && fwrite(cparts.data(), sizeof(double), cparts.size(), fp) == cparts.size();
    ok = ok && fwrite(&sum, sizeof(sum), 1, fp) == 1;
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : LBM_EIO;
}

int lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    FILE* fp = fopen(path, "rb");
    if (!fp) return LBM_EIO;
    CkptHeader h;
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "LBMGB300", 8) != 0 || h.version != 2) {
        fclose(fp);
        return LBM_EIO;
    }
    const size_t E = ckpt_pop_words(c);
    if (h.box[0] != c->box[0] || h.box[1] != c->box[1] || h.box[2] != c->box[2] || h.prec != c->prec ||
        h.bc != c->model.periodic || h.npop != (int64_t)E || h.nknots < 0 || h.nknots > (1LL << 32) ||
        h.ncentre < 0 || h.ncentre > (1LL << 30)) {
        fclose(fp);
        return LBM_EINVAL;
    }
    std::vector<double> kt, kA, pop, cparts;
    try {
        kt.resize((size_t)h.nknots);
        kA.resize((size_t)h.nknots * 9);
        pop.resize(E);
        cparts.resize((size_t)h.ncentre * 4 + 8);
    } catch (...) {
        fclose(fp);
        return LBM_ENOMEM;
    }
    uint64_t stored = 0;
    bool ok = fread(kt.data(), sizeof(double), kt.size(), fp) == kt.size();
    ok = ok && fread(kA.data(), sizeof(double), kA.size(), fp) == kA.size();
    ok = ok && fread(pop.data(), sizeof(double), E, fp) == E;
    ok = ok && fread(cparts.data(), sizeof(double), cparts.size(), fp) == cparts.size();
    ok = ok && fread(&stored, sizeof(stored), 1, fp) == 1;
    fclose(fp);
    if (!ok) return LBM_EIO;
    uint64_t sum = fnv1a(&h, sizeof(h));
    sum = fnv1a(kt.data(), sizeof(double) * kt.size(), sum);
    sum = fnv1a(kA.data(), sizeof(double) * kA.size(), sum);
    sum = fnv1a(pop.data(), sizeof(double) * E, sum);
    sum = fnv1a(cparts.data(), sizeof(double) * cparts.size(), sum);
    if (sum != stored) return LBM_EIO;
    int st = set_device(c);
    if (st) return st;
    LBM_TRY(cudaStreamSynchronize(c->stream));
    c->R = h.R; c->xi = h.xi; c->rho_hi = h.rho_hi; c->rho_lo = h.rho_lo;
    c->model.tau[0] = h.tau[0]; c->model.tau[1] = h.tau[1];
    c->model.G = h.G;
    c->model.rho_b[0] = h.rho_b[0]; c->model.rho_b[1] = h.rho_b[1];
    c->kt.swap(kt);
    c->kA.swap(kA);
    if (is_dev(c->prec)) {
        LBM_TRY(cudaMemcpyAsync(c->f[c->cur], pop.data(), (size_t)c->L.total * c->elem, cudaMemcpyHostToDevice,
                                c->stream));
        LBM_TRY(launch_centre(c->prec, c->f[c->cur], c->L, c->centre, c->stream));
        c->initialised = true;
    } else if ((st = lbm_set_populations(c, pop.data()))) {
        return st;
    }
    // restore the saved frame origin partials when the launch shape matches
    // (otherwise the ones just recomputed from the populations stay)
    float fr[3];  // the frame origin's float32 copy, as the reduction writes it (alive until the sync below)
    if (h.ncentre == c->centre.n) {
        LBM_TRY(cudaMemcpyAsync(c->centre.p, cparts.data(), sizeof(double) * cparts.size(), cudaMemcpyHostToDevice,
                                c->stream));
        const size_t o = (size_t)4 * c->centre.n + 4;
        for (int q = 0; q < 3; ++q) fr[q] = (float)cparts[o + q];
        LBM_TRY(cudaMemcpyAsync(c->centre.frame, fr, sizeof(fr), cudaMemcpyHostToDevice, c->stream));
    }
    c->step = h.step;
    LBM_TRY(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_profile_enable(lbm_ctx* c, int enable) {
    if (!c) return LBM_EINVAL;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k) {
        for (cudaEvent_t ev : c->ev[k]) cudaEventDestroy(ev);
        c->ev[k].clear();
        c->prof_n[k] = 0;
    }
    c->prof = enable > 0 ? enable : 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx* c, int kernel, double* total_ms, int64_t* launches) {
    if (!c || kernel < 0 || kernel > 1 || !total_ms || !launches) return LBM_EINVAL;
    cudaSetDevice(c->device);
    LBM_TRY(cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    const std::vector<cudaEvent_t>& v = c->ev[kernel];
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        float ms = 0.0f;
        LBM_TRY(cudaEventElapsedTime(&ms, v[i], v[i + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = (int64_t)(v.size() / 2);
    return LBM_OK;
}

int lbm_launch_shape(lbm_ctx* c, int32_t* tile_y, int32_t* z_chunk, int32_t* ctas) {
    if (!c) return LBM_EINVAL;
    if (tile_y) *tile_y = c->shape.ty;
    if (z_chunk) *z_chunk = c->shape.zchunk;
    if (ctas) *ctas = (int32_t)(c->shape.grid.x * c->shape.grid.y * c->shape.grid.z);
    return LBM_OK;
}

int lbm_launch_variant(lbm_ctx* c, int32_t* variant) {
    if (!c || !variant) return LBM_EINVAL;
    if (!c->shape.rows) *variant = 0;
    else *variant = c->shape.variant == kRowStaged ? 2 : (c->shape.variant == kRowWs ? 3 : 1);
    return LBM_OK;
}

}  // extern "C"
