// Internal declarations shared by the host ABI (lbm_abi.cu) and the kernel
// translation units (lbm_step.cu, lbm_reduce.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace lbmgb {

// Padded, row-interleaved structure-of-arrays population layout in device
// memory:
//
//   element (s, i, z, y, x) at  (z + 1) * plane + (y + 1) * row + (s*19 + i) * pitch + x0 + x
//
// for fluid nodes x in [0, Lx), y in [0, Ly), z in [0, Lz), with row = 38 *
// pitch (all populations of one row of nodes) and plane = ny * row.  Within a
// row block the 38 populations are rows of `pitch` elements, so the offset
// between any two populations of one node, and between the populations a
// node pulls from its neighbours (x - c_i), is a constant fixed by Lx alone
// except for the z plane: the row kernels address every access as one of
// three per-plane pointers plus a compile-time immediate.  One ghost layer
// surrounds the box: x = -1 .. Lx, y = -1 .. Ly, z = -1 .. Lz all have
// storage.  x0 puts the first fluid node of every row on a 32-byte boundary,
// and pitch (a multiple of 32 bytes) keeps every row on that boundary.
//
// 16-bit deviation storage uses the same geometry in 2-byte units with row =
// 44 * pitch: per row block first a row of `pitch` float4 blocks
// {rho*_A, rho*_B, f*_0A, f*_0B} (8 units per entry), then for each direction
// i = 1..18 a row of `pitch` 32-bit words, one per node, holding the
// deviations of both components {A, B} (see dev_node / dev_word / dev_at).
struct Layout {
    int Lx, Ly, Lz;
    int x0;           // elements before x = 0 in a row
    int pitch;        // elements per population row
    int ny, nz;       // Ly + 2, Lz + 2
    long long row;    // elements per row block (all populations of one row of nodes)
    long long plane;  // elements per z plane (ny row blocks)
    long long total;  // nz * plane
    __host__ __device__ long long at(int s, int i, int x, int y, int z) const {
        return (long long)(z + 1) * plane + (long long)(y + 1) * row + (long long)(s * 19 + i) * pitch + x0 + x;
    }
    // 16-bit deviation storage: float4 index of node (x, y, z)'s block
    __host__ __device__ long long dev_node(int x, int y, int z) const {
        return (long long)(z + 1) * (plane >> 3) + (long long)(y + 1) * (row >> 3) + x0 + x;
    }
    // 16-bit deviation storage: 32-bit word index of the deviation pair
    // {A, B} of direction i >= 1 of node (x, y, z)
    __host__ __device__ long long dev_word(int i, int x, int y, int z) const {
        return (long long)(z + 1) * (plane >> 1) + (long long)(y + 1) * (row >> 1) + (long long)(3 + i) * pitch + x0 +
               x;
    }
    // 16-bit deviation storage: 2-byte index of deviation (s, i >= 1) of node (x, y, z)
    __host__ __device__ long long dev_at(int s, int i, int x, int y, int z) const {
        return 2 * dev_word(i, x, y, z) + s;
    }
};

// Precision codes of the kernels (the values of lbm_precision).
enum { kFP64 = 0, kFP32 = 1, kFP16Dev = 2, kBF16Dev = 3 };
inline bool is_dev(int prec) { return prec == kFP16Dev || prec == kBF16Dev; }
// Bytes of one layout element: 8, 4 or 2 (the 16-bit unit of deviation storage).
inline int elem_bytes_of(int prec) { return prec == kFP64 ? 8 : (prec == kFP32 ? 4 : 2); }

Layout make_layout(int Lx, int Ly, int Lz, int prec);

// Scalars of the model that every kernel needs.
struct Model {
    double tau[2];     // relaxation times (Eq. 10)
    double G;          // Shan-Chen coupling (Eq. 7)
    double rho_b[2];   // ghost densities of A and B (Sec. 3)
    int periodic;      // 1: periodic test mode, no ghosts
    double mach2;      // guard on |u_ghost|^2 (lattice units)
    int droplet_frame; // 1: ghost flow A (x - x_c), x_c the droplet's centre of mass
    int mrt;           // 1: MRT collision with the free rates below (row kernel for float32 storage, else generic)
    double mrt_rates[5];  // s_e, s_eps, s_q, s_pi, s_m
};

// Per-CTA partial sums {sum w, sum w x, sum w y, sum w z} of the droplet
// indicator w = max(phi, 0) of the current state, written by the
// stream-collide kernel (one row per CTA) or by launch_centre.  The last CTA
// to finish sums the rows in CTA order into `sum` (deterministic) and resets
// `counter`; the ghost kernel of the next step reads `sum`.
//
// The partials are kept in the reduction's own type (float32 for the float32
// and 16-bit storage kernels, float64 for the float64 kernel: `p` is then
// read as float[n][4]), so that float32 kernels execute no FP64 instruction,
// which the FP64 pipe of this GPU runs at 1/64 of the float32 rate.
struct CentreParts {
    double* p;          // [n][4] partials of the reduction type
    int n;              // CTAs of the stream-collide launch
    double* sum;        // [8]: the four sums, then the frame origin x_c, y_c, z_c
    unsigned* counter;  // CTAs finished, 0 between launches
    float* frame;       // [3]: x_c, y_c, z_c rounded to float32 (read by the float32 ghost kernels)
};

// A velocity gradient passed by value, row-major A[3a+b] = d u_a / d x_b.
struct Grad {
    double a[9];
};

// Launch shape of the stream-collide kernel.
struct Shape {
    int rows;       // 1: the row-tiled cluster kernel (lbm_fast.cu), 0: the generic tile kernel
    int tx, ty;     // tile of the x-y plane per CTA
    int zchunk;     // z planes marched per CTA
    int variant;    // row kernel: kRowDirect, kRowStaged or kRowWs
    dim3 grid;
    int threads;
    size_t smem;
};

// Rows per thread-block cluster of the row kernels (lbm_fast.cu).
constexpr int kRowClusterRows = 8;

// Variants of the row kernel: per-thread loads of the pulled populations
// (each plane read twice, the second time from L2), whole pulled rows staged
// in shared memory by bulk copies, or loader and collider threads per row
// (warp-specialised, each population read once).
enum { kRowDirect = 0, kRowStaged = 1, kRowWs = 2 };

// ---- launchers (lbm_step.cu) ----
// variant_req: the row_variant of lbm_opts (1 direct loads, 2 staged,
// 3 warp-specialised, 0 automatic); mrt: the MRT collision (the row kernel's
// direct variant for float32 storage, the generic kernel otherwise)
Shape choose_shape(const Layout& L, int prec, int periodic, int mrt, int ty_req, int zchunk_req, int variant_req,
                   int num_sms);
cudaError_t launch_init(int prec, void* f, const Layout& L, double R, double xi, double rho_hi, double rho_lo,
                        Grad A0, cudaStream_t s);
cudaError_t launch_ghost(int prec, void* f, const Layout& L, const Model& m, Grad A, CentreParts cp, int* d_err,
                         cudaStream_t s);
// A: the boundary gradient of this step (the kernels read the ghost shell
// written by launch_ghost; A is passed for kernels that may compute it).
cudaError_t launch_stream_collide(int prec, const void* src, void* dst, const Layout& L, const Model& m,
                                  const Shape& sh, const Grad& A, CentreParts cp, int* d_err, cudaStream_t s);
// Centre-of-mass partials of the stored populations f (cp.n CTAs, grid-stride).
cudaError_t launch_centre(int prec, const void* f, const Layout& L, CentreParts cp, cudaStream_t s);

// ---- row-tiled cluster kernel (lbm_fast.cu): fp32 or 16-bit deviations, ghost boundary,
//      Lx in {32, 64, 128, 256}, Ly % 8 == 0 ----
// variant: kRowDirect, kRowStaged or kRowWs.
bool rows_kernel_applies(const Layout& L, int prec, int periodic);
// One warp waits on an mbarrier with the kernels' bounded wait (limit_ns of
// wall time); nothing arrives unless arrive.  *gave_up = 1 when the wait gave
// up.  Synchronises s.
cudaError_t launch_wait_selftest(unsigned long long limit_ns, int arrive, cudaStream_t s, int* gave_up);
int rows_kernel_resident_ctas(const Layout& L, int prec, int variant, int mrt);
cudaError_t launch_stream_collide_rows(int prec, int variant, const void* src, void* dst, const Layout& L,
                                       const Model& m, const Grad& A, int zchunk, CentreParts cp, int* d_err,
                                       cudaStream_t s);

// ---- the batched ensemble on the row kernel (lbm_fast.cu) ----
// Every box of the ensemble is laid out with the row geometry of width
// kRowsBatchWidth (rows padded to that width: Lx <= kRowsBatchWidth, Ly a
// multiple of kRowClusterRows), float32.  One launch runs the staged row
// kernel over the row groups of all boxes, stacked along grid y, with z chunks
// along grid z (boxes with fewer chunks leave the extra clusters idle); each
// box's centre of mass is reduced by the last of its CTAs, and the last CTA
// of the launch advances the device step counter.
constexpr int kRowsBatchWidth = 64;
struct RowsBatchBox {
    float* f[2];  // the two population buffers
    Layout L;     // make_layout_rows
    int ctas;     // CTAs of the box: Ly x its z chunks
    int part0;    // its first slot of centre partials
};
struct RowsBatch {
    const int4* group;          // per row group: {box, first row in the box, z chunks of the box, 0}
    const RowsBatchBox* box;
    float* parts;               // [slots][4] centre partials (float32)
    unsigned* box_done;         // [box] CTAs finished, 0 between launches
    double* box_sums;           // [box][8]: the four sums, then x_c, y_c, z_c
    float* box_frame;           // [box][4]: x_c, y_c, z_c in float32
    unsigned* ctas_done;        // CTAs of the launch finished, 0 between launches
    long long* d_step;          // advanced by the launch's last CTA
    int parity;                 // the boxes' f[parity] is read, f[1 - parity] written
};
// The layout of an Lx x Ly x Lz box with rows padded to kRowsBatchWidth.
Layout make_layout_rows(int Lx, int Ly, int Lz);
bool rows_batch_applies(int Lx, int Ly, int Lz);
// groups: total row groups (grid y / kRowClusterRows); max_chunks: grid z.
cudaError_t launch_rows_batch(const RowsBatch& rb, int groups, int max_chunks, int zchunk, const Model& m,
                              int* d_err, cudaStream_t s);
// Dynamic shared memory of a batched launch (bytes).
size_t rows_batch_smem();

// ---- launchers (lbm_reduce.cu) ----
// Ten moments of w = max(phi, 0) and the deformation: result[0..9] moments,
// [10] D, [11..19] axes (column-major by axis), [20..22] lambda,
// [23..25] centre.  partials: nblocks * 10 doubles of scratch.
int moments_blocks(const Layout& L, int num_sms);
cudaError_t launch_moments(int prec, const void* f, const Layout& L, double* partials, int nblocks,
                           double* result, cudaStream_t s);
// m: the ghost densities and boundary mode, which 16-bit deviation storage
// needs to rebuild the populations that leave the box.
cudaError_t launch_fields(int prec, const void* f, const Layout& L, const Model& m, double* rho_a, double* rho_b,
                          double* u, cudaStream_t s);
cudaError_t launch_checksums(int prec, const void* f, const Layout& L, const Model& m, double* partials,
                             int nblocks, double* result5, cudaStream_t s);
cudaError_t launch_pack(int prec, const void* f, const Layout& L, const Model& m, double* out, cudaStream_t s);
// Connected components of phi > threshold (6-connectivity): label init, one
// propagation sweep (sets *changed), component sizes of the roots (first cap).
cudaError_t launch_cc_init(int prec, const void* f, const Layout& L, double threshold, int* label, cudaStream_t s);
cudaError_t launch_cc_sweep(const Layout& L, int periodic, int* label, int* changed, cudaStream_t s);
// Eq. 17 statistics of phi: {sum phi, min, max, sum |grad phi|}; mass of A
// split at phi = 0; droplet-component scaling at phi > 0 (fp64 / fp32 only).
cudaError_t launch_surface_stats(int prec, const void* f, const Layout& L, double* phi, double* partials, int nblocks,
                                 double* out, cudaStream_t s);
cudaError_t launch_mass_split(int prec, const void* f, const Layout& L, double* partials, int nblocks, double* out,
                              cudaStream_t s);
cudaError_t launch_reinject(int prec, void* f, const Layout& L, double k, cudaStream_t s);
cudaError_t launch_cc_sizes(const Layout& L, const int* label, int* size, int* count, long long* out, int cap,
                            cudaStream_t s);
// scratch: 2 N floats (16-bit deviation storage only; may be NULL otherwise)
cudaError_t launch_unpack(int prec, void* f, const Layout& L, const Model& m, const double* in, float* scratch,
                          cudaStream_t s);

}  // namespace lbmgb
