/*
 * lbm.h -- C ABI of the GB300 (sm_103a) two-component Shan-Chen lattice
 * Boltzmann solver for a droplet in an exact linear flow.
 *
 * The method is the multiscale scheme of Milan, Biferale, Sbragaglia and
 * Toschi, "Sub-Kolmogorov droplet dynamics in isotropic turbulence using a
 * multiscale Lattice Boltzmann scheme" (arXiv:2112.09972):
 *   - two fluid components sigma = A (droplet) and B (solvent), D3Q19 lattice,
 *     densities and momentum of Sec. 2, Eq. 6;
 *   - Shan-Chen interaction force F^sigma of Sec. 2, Eq. 7 (psi = rho,
 *     G_AB = G_BA = G, G_AA = G_BB = 0);
 *   - ghost nodes one lattice layer outside the box that hold the equilibrium
 *     of Eq. 8 at the boundary density rho_b and the linear flow u = A(t) x of
 *     Sec. 3, Eq. 14, with x measured from the droplet's centre of mass (the
 *     droplet frame, lbm_frame) or from the box centre;
 *   - pull streaming and BGK collision (Eq. 9) with nu = (tau - 1/2)/3
 *     (Eq. 10), forcing by the Shan-Chen velocity shift;
 *   - droplet deformation D = (L - W)/(L + W) (Sec. 2, Eq. 4), with L, W from
 *     the principal second moments of the droplet indicator max(phi, 0),
 *     phi = (rho_A - rho_B)/(rho_A + rho_B).
 *
 * Conventions for every call:
 *   - Return value: an lbm_status (0 = LBM_OK).  No exception or abort ever
 *     crosses this interface.
 *   - Invalid arguments return LBM_EINVAL and leave the context unchanged.
 *   - Work is enqueued on the context's CUDA stream and runs asynchronously;
 *     a device-side fault condition (non-finite density, Mach guard) is latched
 *     on the device and reported by the next call that synchronises
 *     (lbm_sync, lbm_deformation, lbm_get_*, lbm_checksums, lbm_save).
 *   - Host arrays are owned by the caller, copied in or out during the call and
 *     never retained.  Device memory is owned by the context.
 *   - Population layout exchanged with the host (lbm_get/set_populations):
 *     float64 [component][direction][z][y][x], component 0 = A, 1 = B, x
 *     fastest; directions in the D3Q19 order
 *       0 (0,0,0); 1 (+1,0,0) 2 (-1,0,0) 3 (0,+1,0) 4 (0,-1,0) 5 (0,0,+1)
 *       6 (0,0,-1); 7 (+1,+1,0) 8 (-1,-1,0) 9 (+1,-1,0) 10 (-1,+1,0)
 *       11 (+1,0,+1) 12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1)
 *       15 (0,+1,+1) 16 (0,-1,-1) 17 (0,+1,-1) 18 (0,-1,+1).
 *   - Gradients are row-major 3x3, A[3*a + b] = d u_a / d x_b.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* invalid argument */
    LBM_ENOMEM = -2,     /* device or host allocation failed */
    LBM_ECUDA = -3,      /* a CUDA runtime call failed */
    LBM_ENONFINITE = -4, /* a non-finite density appeared on the device */
    LBM_EMACH = -5,      /* a ghost velocity exceeded the Mach guard */
    LBM_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
    LBM_EIO = -7         /* checkpoint file missing, short or corrupt */
} lbm_status;

typedef enum {
    LBM_FP64 = 0,     /* populations stored and collided in float64 */
    LBM_FP32 = 1,     /* populations stored and collided in float32 */
    /* 16-bit deviation storage, float32 collision.  Per node and component
       the post-collision density rho* and the rest population f*_0 are kept
       in float32; each moving population f*_i (i = 1..18) is kept as the
       16-bit deviation d_i = f*_i - w_i rho(x + c_i) from the equilibrium
       weight of the density of the node it streams to (the writer holds that
       density on chip for the force of Eq. 7, and the reader rebuilds the
       pulled value from its own rho*).  The rest population closes the mass
       of the node exactly, so mass is conserved to float32 rounding.  88
       bytes per node and copy (float64: 608, float32: 304).  Boxes with
       box[0] in {32, 64, 128, 256} and box[1] a multiple of 8, ghost
       boundary; other shapes use the generic kernel. */
    LBM_FP16_DEV = 2, /* deviations in IEEE binary16 */
    LBM_BF16_DEV = 3  /* deviations in bfloat16 */
} lbm_precision;

typedef enum {
    LBM_BC_GHOST_LINEAR = 0, /* the paper's ghost nodes with u = A(t) x (Sec. 3) */
    LBM_BC_PERIODIC_TEST = 1 /* periodic box with no boundary: a test mode */
} lbm_bc;

typedef enum {
    /* x in the ghost flow A(t) x is measured from the droplet's centre of
       mass, recomputed before every step from the current state (the frame
       of Sec. 3, Eq. 14, in which the droplet's centre stays fixed); the box
       centre when there is no droplet (sum of max(phi, 0) is zero) */
    LBM_FRAME_DROPLET = 0,
    /* x is measured from the box centre */
    LBM_FRAME_BOX = 1
} lbm_frame;

typedef enum {
    LBM_COLLISION_BGK = 0, /* single relaxation time 1/tau per component (Eqs. 9, 10) */
    /* multi-relaxation-time collision (Sec. 2), d'Humieres et al. (2002)
       D3Q19 moment basis: g* = g - M^-1 S M (g - g_eq); stress and momentum
       moments relax at 1/tau (Eq. 10; the velocity-shift forcing), the others
       at opts->mrt_rates.  Runs in the row kernel for LBM_FP32 storage on
       boxes with box[0] in {32, 64, 128, 256} and box[1] a multiple of 8
       (ghost boundary), on the generic kernel otherwise. */
    LBM_COLLISION_MRT = 1
} lbm_collision;

typedef struct {
    int32_t precision;   /* lbm_precision, default LBM_FP32 */
    int32_t bc;          /* lbm_bc, default LBM_BC_GHOST_LINEAR */
    double rho_hi;       /* majority density of either phase; <= 0: 1.0 */
    double rho_lo;       /* minority density; also the ghost density of A.
                            <= 0: the flat-interface value ln(h/l) = G (h - l) */
    double xi;           /* width of the initial tanh profile; <= 0: 1.0 */
    double mach_limit;   /* guard on |u_ghost| / c_s; <= 0: 0.9 */
    void* cuda_stream;   /* cudaStream_t to run on; NULL: the context creates
                            its own non-blocking stream */
    int32_t device;      /* CUDA device ordinal; < 0: the current device */
    int32_t tile_y;      /* rows per CTA of the stream-collide kernel; 0: auto */
    int32_t z_chunk;     /* z planes per CTA of the stream-collide kernel; 0: auto */
    int32_t frame;       /* lbm_frame, default LBM_FRAME_DROPLET */
    int32_t row_variant; /* row-tiled kernel: 1 per-thread loads of the pulled
                            populations (each plane read twice, the second
                            time from L2), 2 the pulled rows of each plane
                            staged in shared memory by bulk copies
                            (cp.async.bulk, two planes ahead, one read; each
                            node's populations carried in registers to its
                            collision), 3 loader and collider threads per row (warp-
                            specialised: each population read once, staged in
                            shared memory for the collision); 0: automatic
                            (2 for every storage form; 1 when the MRT
                            collision is selected); LBM_EINVAL outside 0..3 */
    int32_t collision;   /* lbm_collision, default LBM_COLLISION_BGK */
    double mrt_rates[5]; /* MRT rates of the energy, energy-square, energy-flux,
                            stress-partner and third-order moments (s_e, s_eps,
                            s_q, s_pi, s_m), each in (0, 2); <= 0: 1.19, 1.4,
                            1.2, 1.4, 1.98 */
} lbm_opts;

/* Fill *opts with the defaults above. */
void lbm_opts_default(lbm_opts* opts);

/*
 * Create a context: a box of box[0] x box[1] x box[2] fluid nodes (x, y, z),
 * each >= 4, with a droplet of component A of radius R (0 < R, 2R <=
 * min(box) - 2 for the ghost boundary) at the box centre, kinematic
 * viscosities visc = {nu_A, nu_B} > 0 in lattice units (tau = 3 nu + 1/2,
 * Eq. 10) and coupling G >= 0 (Eq. 7).  The populations start at the
 * equilibrium of the tanh density profile rho_A = lo + (hi - lo)(1 -
 * tanh((r - R)/xi))/2, rho_B = lo + (hi - lo)(1 + tanh((r - R)/xi))/2 and the
 * flow u = A(0) x of the gradient table (zero until lbm_set_gradient).  The
 * ghost densities are rho_b^A = rho_lo and rho_b^B = rho_hi (density ratio 1,
 * Sec. 3).  Device memory: two population buffers of
 * 38 (box[2]+2)(box[1]+2) pitch elements (float64 / float32), pitch >=
 * box[0] + 2, or 88 (box[2]+2)(box[1]+2) pitch bytes (16-bit deviations).
 * On success *out receives the context; on failure *out is NULL.
 */
int lbm_create(lbm_ctx** out, const int32_t box[3], double R, const double visc[2], double G,
               const lbm_opts* opts);

/*
 * Add a knot (t, A) to the context's velocity-gradient table.  Step n of the
 * simulation drives the ghost nodes with A(t_n), t_n = n, linearly
 * interpolated between knots and held constant before the first and after
 * the last knot (the gradient "sampling time" of Sec. 4: one tracer sample
 * every Delta t steps).  A must be traceless: |tr A| <= 1e-12 max(1, max|A_ij|),
 * otherwise LBM_EINVAL; t must exceed the previous knot's t.  If the first
 * knot is added before any step, the initial flow is re-initialised to
 * A(0) x (it is the flow of the paper's initial condition).
 */
int lbm_set_gradient(lbm_ctx* ctx, const double A[9], int64_t t);

/* Add n knots at once: t[k], A[9k .. 9k+8]; same rules as lbm_set_gradient. */
int lbm_set_gradient_table(lbm_ctx* ctx, const int64_t* t, const double* A, int64_t n);

/*
 * Advance n >= 0 time steps.  Each step runs the ghost-boundary kernel
 * (ghost equilibria from A(t_n) (x - x_c), Eq. 8/14, x_c the frame origin of
 * lbm_frame) and then the fused pull-stream + Shan-Chen force + collision
 * kernel (Eqs. 6, 7, 9, 10), which also accumulates the droplet's centre of
 * mass of the state it writes for the next step's frame.
 * Asynchronous: returns once the work is enqueued.
 */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* Wait for the context's stream and report any latched device error. */
int lbm_sync(lbm_ctx* ctx);

/*
 * Droplet deformation of the current state (Eq. 4): D = (sqrt(l1) - sqrt(l3))
 * / (sqrt(l1) + sqrt(l3)) with l1 >= l2 >= l3 the eigenvalues of the central
 * second-moment tensor of w = max(phi, 0).  axes (may be NULL) receives the
 * unit principal axes as columns, axes[3*a + k] = component a of axis k, each
 * signed so its largest-magnitude component is positive; lambda (may be NULL)
 * receives l1, l2, l3; centre (may be NULL) the centre of mass of w.
 * When no node has phi > 0 (no droplet phase) the tensor is undefined: D,
 * axes, lambda and centre are NaN and the call still returns LBM_OK.
 * Synchronises.
 */
int lbm_deformation(lbm_ctx* ctx, double* D, double axes[9], double lambda[3], double centre[3]);

/*
 * The ten float64 moments of w = max(phi, 0) over the box:
 * {sum w, sum w x, sum w y, sum w z, sum w xx, sum w xy, sum w xz, sum w yy,
 *  sum w yz, sum w zz}, coordinates from the box centre.  Synchronises.
 */
int lbm_moments(lbm_ctx* ctx, double m[10]);

/*
 * Copy the fields of the current (post-collision) populations to the host
 * (Eq. 6): rho_A[n], rho_B[n], u[3n + a] = sum_s sum_i g_i^s c_ia / (rho_A +
 * rho_B), n = (z * box[1] + y) * box[0] + x.  Any pointer may be NULL.
 * Synchronises.
 */
int lbm_get_fields(lbm_ctx* ctx, double* rho_A, double* rho_B, double* u);

/* Copy all populations to / from the host (float64, layout above).  With
 * 16-bit deviation storage the values read back are w_i rho*(x + c_i) + d_i
 * (the ghost density where x + c_i lies outside the box), and values written
 * are converted to that form: rho* is their float32 sum, each d_i is rounded
 * to 16 bits and the rest population closes the node's mass. */
int lbm_get_populations(lbm_ctx* ctx, double* f);
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* float64 sums over the box: mass[s] = sum rho_s, mom[a] = sum rho u_a. */
int lbm_checksums(lbm_ctx* ctx, double mass[2], double mom[3]);

/*
 * Breakup detection: the connected components (6-connected nodes) of the
 * droplet phase phi > threshold of the current state, phi = (rho_A - rho_B) /
 * (rho_A + rho_B) (0 is the interface).  *count receives the number of
 * components with at least min_nodes nodes and sizes[0 .. max_sizes-1] their
 * node counts, largest first (0 past the last).  A droplet that broke up
 * has count >= 2.  Periodic images connect in the periodic test mode.
 * Synchronises; allocates 16 bytes per node of scratch for the call
 * (LBM_ETIMEOUT if the labelling did not settle within its sweep bound).
 */
int lbm_components(lbm_ctx* ctx, double threshold, int64_t min_nodes, int32_t* count, int64_t* sizes,
                   int32_t max_sizes);

/*
 * Surface-area deformation of Sec. 5, Eq. 17: D_lbm = sqrt(1 - Omega_0 /
 * Omega), Omega the droplet's surface area and Omega_0 that of the sphere of
 * its volume.  The diffuse interface's area is the mean area of the level
 * sets of phi between its extremes (co-area formula): Omega = sum |grad phi| /
 * (phi_max - phi_min), central differences at interior nodes; the volume
 * V = sum (phi - phi_min) / (phi_max - phi_min); Omega_0 = (36 pi V^2)^(1/3).
 * area and volume (may be NULL) receive Omega and V.  Synchronises;
 * allocates 8 bytes per node of scratch for the call.
 */
int lbm_surface_deformation(lbm_ctx* ctx, double* D_lbm, double* area, double* volume);

/*
 * Mass reinjection (the reading adopted for the method Sec. 2 cites): the
 * droplet component's populations at the nodes with phi > 0 are multiplied
 * by one factor k so that the component's total mass becomes target (> 0);
 * *factor (may be NULL) receives k.  float64 and float32 storage only
 * (LBM_EINVAL for 16-bit deviations, or without a droplet phase).
 * Synchronises.
 */
int lbm_reinject_mass(lbm_ctx* ctx, double target, double* factor);

/* Step counter n of the next step (the number of steps taken so far). */
int lbm_get_step(lbm_ctx* ctx, int64_t* step);

/*
 * Checkpoint: lbm_save writes the parameters, the step counter, the gradient
 * table and the populations (float64; the raw device buffer for 16-bit
 * deviation storage) with a 64-bit FNV-1a checksum;
 * lbm_load restores them into a context created with the same box, precision
 * and boundary mode (LBM_EINVAL otherwise, LBM_EIO for a missing, short or
 * corrupt file).  A resumed run is bit-identical to an uninterrupted one.
 */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/*
 * Kernel timing: lbm_profile_enable(ctx, k) with k > 0 brackets the launches
 * of every k-th step (step counter divisible by k) of the stream-collide
 * kernel (kernel 0) and of the ghost kernel (kernel 1) with CUDA events on
 * the context's stream; k = 0 turns it off.  lbm_profile_read synchronises
 * and returns the summed device time in milliseconds and the number of timed
 * launches since the last enable.
 */
int lbm_profile_enable(lbm_ctx* ctx, int enable);
int lbm_profile_read(lbm_ctx* ctx, int kernel, double* total_ms, int64_t* launches);

/* Launch shape of the stream-collide kernel in use: rows per CTA, z planes
 * per CTA, CTAs. */
int lbm_launch_shape(lbm_ctx* ctx, int32_t* tile_y, int32_t* z_chunk, int32_t* ctas);

/* The stream-collide kernel in use: *variant = 0 the generic tile kernel
 * (k_stream_collide), or the row-tiled cluster kernel's variant as in
 * lbm_opts.row_variant (1 per-thread loads and 2 shared-memory staging, both
 * k_stream_collide_rows; 3 loader and collider threads, k_stream_collide_ws).
 * LBM_EINVAL for a NULL context or pointer. */
int lbm_launch_variant(lbm_ctx* ctx, int32_t* variant);

/*
 * Allocation-free droplet moments (an addition of this library; the paper has
 * no counterpart).  For callers that cannot allocate device memory when they
 * need the droplet's shape: code recording into a CUDA graph (no cudaMalloc
 * inside a capture), loops that must not touch the allocator, hosts with a
 * fixed memory budget.  Computes the same result as lbm_moments and
 * lbm_deformation from populations the caller already holds on the device:
 *   f          device pointer to float64 (precision LBM_FP64) or float32
 *              (LBM_FP32) populations in the dense layout of
 *              lbm_get_populations: [2][19][box[2]][box[1]][box[0]];
 *   box        box extents (x, y, z), each >= 1, at most 2^31/38 nodes in all
 *              (larger boxes return LBM_EINVAL);
 *   out        device pointer to 26 doubles receiving, in order, the ten
 *              moments of lbm_moments, D, the axes (as in lbm_deformation,
 *              axes[3*a + k]), the three eigenvalues and the centre of mass;
 *   cuda_stream the stream to run on (NULL: the legacy default stream).
 * Asynchronous; no device or host memory is allocated and no synchronising
 * call is made.  Scratch lives in one fixed 80 KB device array of the library
 * (1024 blocks x 10 doubles), held by every GPU that loads the library until
 * the process exits.  Its device address is looked up on the first call on
 * each device (with that device current): make that first call before any
 * stream capture starts.  After cudaDeviceReset of a device the cached
 * address is stale: do not call this entry point on that device again in the
 * same process.  All calls share the array, so calls whose kernels may run
 * concurrently on the GPU (unordered streams) race and give wrong results;
 * calls ordered on one stream are safe.  Returns LBM_ECUDA when one of the
 * call's own two launches fails (an error left by an earlier, unrelated call
 * is neither reported nor cleared).
 */
int lbm_moments_static(const void* f, int32_t precision, const int32_t box[3], double* out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched ensemble: many independent droplet boxes (for deformation
 * statistics over many tracer trajectories, Sec. 6), each a full copy of the
 * single-box method above with its own size, radius and per-step gradient
 * history, advanced together: one ghost launch and one stream-collide launch
 * per step, replayed from a captured CUDA graph.  When every box has
 * Lx <= 64 and Ly a multiple of 8 (and opts->tile_y is 0), the stream-collide
 * launch is the staged row kernel over the row groups of all boxes, with
 * rows padded to 64 (lbm_batch_launch_kind 1); otherwise a persistent launch
 * of the generic tile march over a work list of (box, tile, z chunk) items
 * (kind 0).  fp32 populations, ghost boundary, the frame of opts->frame.
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque */

/*
 * Create an ensemble of nbox boxes: boxes[3k .. 3k+2] = (Lx, Ly, Lz) of box k
 * (each 4 .. 1024), R[k] its droplet radius (2 R <= min extent - 2).
 * visc, G as for lbm_create.  opts must ask for LBM_FP32 and the ghost
 * boundary and must give rho_lo > 0 (the ghost density of the droplet
 * component); rho_hi <= 0 means 1.  opts->z_chunk (0: 32 for the row kernel,
 * 16 for the tile march) sets the initial z planes per work item; opts->tile_y
 * > 0 keeps the tile march.  Each box starts, on first use, at the equilibrium
 * tanh droplet in the flow of its gradient at step 0.
 */
int lbm_batch_create(lbm_batch** out, int32_t nbox, const int32_t* boxes, const double* R, const double visc[2],
                     double G, const lbm_opts* opts);

/*
 * Per-step gradients of every box: A[(t * nbox + k) * 9 .. + 8] drives box k at
 * step t, t = 0 .. nsteps-1 (row-major, traceless, see lbm_set_gradient);
 * steps beyond the table use its last row.  Stored on the device in float32.
 */
int lbm_batch_set_gradients(lbm_batch* batch, int64_t nsteps, const double* A);

/* Advance every box n steps (asynchronous; pairs of steps replay a CUDA graph). */
int lbm_batch_step(lbm_batch* batch, int64_t n);

/* Wait for the ensemble's stream and report any latched device error. */
int lbm_batch_sync(lbm_batch* batch);

/*
 * D of every box (as lbm_deformation): D[k]; axes[9k ..] and centre[3k ..]
 * may be NULL.  Synchronises.
 */
int lbm_batch_deformation(lbm_batch* batch, double* D, double* axes, double* centre);

/*
 * The ten float64 moments of w = max(phi, 0) of every box (as lbm_moments):
 * m[10k .. 10k+9] for box k, coordinates from the box's centre.  Synchronises.
 */
int lbm_batch_moments(lbm_batch* batch, double* m);

/* Populations of one box to / from the host (float64, lbm_get_populations layout). */
int lbm_batch_get_populations(lbm_batch* batch, int32_t box, double* f);
int lbm_batch_set_populations(lbm_batch* batch, int32_t box, const double* f);

/*
 * Time trial_steps steps for each candidate work-list shape (tile march: z
 * planes per item in {8, 16, 32, 64}, CTAs per SM in {all that fit, 2, 4};
 * row kernel: z planes per chunk in {16, 22, 32, 43, 64}) and keep the
 * fastest.  Only before the first step: the trials run from the initial
 * state, which is restored afterwards (LBM_EINVAL once stepping started).
 * The chosen values are returned in *zchunk and *ctas_per_sm (0 = all that fit).
 */
int lbm_batch_autotune(lbm_batch* batch, int32_t trial_steps, int32_t* zchunk, int32_t* ctas_per_sm);

/* Work-list shape in use: z planes per item, CTAs of the stream-collide
 * launch, work items (tile march: (box, tile, z chunk) items; row kernel:
 * row groups of 8 rows). */
int lbm_batch_shape(lbm_batch* batch, int32_t* zchunk, int32_t* ctas, int32_t* items);

/* The stream-collide launch of the ensemble: *kind = 0 the generic tile
 * march, 1 the row kernel over padded rows.  LBM_EINVAL for NULL. */
int lbm_batch_launch_kind(lbm_batch* batch, int32_t* kind);

/* Free the ensemble (NULL is allowed). */
void lbm_batch_destroy(lbm_batch* batch);

/* Free the context and its device memory (NULL is allowed). */
void lbm_destroy(lbm_ctx* ctx);

/* Static description of a status code. */
const char* lbm_strerror(int code);

/*
 * Diagnostic of the failure path of the device-side waits (the paper has no
 * counterpart).  Every kernel that waits on an mbarrier (the row kernels'
 * density exchange and plane staging, the tensor-core GEMM's pipeline) bounds
 * each wait by wall time; a wait that gives up raises a flag that the next
 * synchronising call reports as LBM_ETIMEOUT, and the kernel returns without
 * blocking.  This call runs one warp on `device` (< 0: the current device)
 * that waits, with the same bounded wait as the row kernels, on an mbarrier
 * with limit limit_ns (1e3 .. 1e10 ns): with arrive = 0 nothing arrives, the
 * wait gives up after limit_ns and the call returns LBM_ETIMEOUT; with
 * arrive = 1 the barrier completes first and the call returns LBM_OK.  Either
 * way the device stays usable.  LBM_EINVAL for other arguments.
 * Synchronises (its own stream).
 */
int lbm_selftest_wait(int64_t limit_ns, int32_t arrive, int32_t device);

/*
 * Maffettone-Minale model (Sec. 2, Eqs. 1, 2, 4, 5) for n gradient histories
 * at once, one GPU thread per trajectory: the morphology tensor M starts at the
 * identity (a sphere) and follows
 *   dM/dt = [f2(chi, Ca) tau_d (S M + M S) + tau_d (W M - M W)
 *            - f1(chi) (M - 3 III_M / II_M I)] / tau_d
 * in LBM time, with S, W the symmetric / antisymmetric parts of A(t),
 * Ca = tau_d max|A_ij| (Eq. 3), II_M = ((tr M)^2 - M:M)/2, III_M = det M.
 *   A       device float64 [T][n][9]: A of trajectory k at LBM step t (row-major,
 *           lattice units), linear in t between rows;
 *   tau_d   the droplet time eta_s R / sigma in LBM steps (> 0); chi the
 *           viscosity ratio (> 0);
 *   substeps classical RK4 steps per LBM step (>= 1);
 *   record_every  D (Eq. 4) is written at t = 0, r, 2r, ... <= T - 1 into
 *           D [floor((T - 1) / r) + 1][n] (device float64);
 *   precision LBM_FP64 or LBM_FP32 arithmetic;
 *   M       device float64 [n][6] (xx, xy, xz, yy, yz, zz) at t = T - 1, or NULL.
 * Asynchronous on cuda_stream; allocates nothing.
 */
int lbm_mm_integrate(const double* A, int64_t T, int64_t n, double tau_d, double chi, int32_t substeps,
                     int32_t record_every, int32_t precision, double* D, double* M, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Learned surrogate (an addition of this library; the paper compares the
 * LBM droplet with the Maffettone-Minale model of Sec. 2, Eqs. 1, 2, 5, and
 * names statistics over many trajectories as its next step, Sec. 6): a
 * multilayer perceptron that maps a window of the velocity gradient A(t) to
 * the droplet's conformation tensor M = I / det(I)^(1/3), I the central
 * second-moment tensor of Eq. 4 (M = identity for a sphere).
 *
 * Layers z_l = h_{l-1} W_l^T + b_l, h_l = max(z_l, 0) for l < L, output layer
 * linear.  Inputs are normalised as (x - x_mean) x_scale and outputs returned
 * as y_hat / y_scale + y_mean.  Training minimises the mean over samples and
 * outputs of (y_hat - (t - y_mean) y_scale)^2 with Adam (beta 0.9, 0.999,
 * eps 1e-8).  Matrix products run on bfloat16 tensor cores with float32
 * accumulation; inputs, weights, hidden activations and back-propagated
 * gradients are stored in bfloat16, parameters and Adam moments in float32.
 * ------------------------------------------------------------------------- */
typedef struct lbm_mlp lbm_mlp; /* opaque */

/*
 * sizes[0 .. nlayers]: input width, hidden widths (all multiples of 32, at
 * most 8192) and output width (1 .. 32).  max_batch (a multiple of 32, at
 * most 2^22) bounds the samples of one training step and the chunk of a
 * forward pass.  Weights start He-normal from seed (std::mt19937_64), biases
 * at zero; normalisation starts as the identity.  cuda_stream NULL: the
 * network creates its own stream; device < 0: the current device.
 */
int lbm_mlp_create(lbm_mlp** out, int32_t nlayers, const int32_t* sizes, int32_t max_batch, uint64_t seed,
                   void* cuda_stream, int32_t device);

/* Input (sizes[0] entries each) and output (sizes[nlayers] entries, scale != 0) normalisation. */
int lbm_mlp_set_normalisation(lbm_mlp* mlp, const float* x_mean, const float* x_scale, const float* y_mean,
                              const float* y_scale);

/* Number of parameters and their flat host layout: W_1 [sizes[1], sizes[0]]
 * row-major, b_1 [sizes[1]], W_2, b_2, ...  set_params resets Adam. */
int lbm_mlp_param_count(lbm_mlp* mlp, int64_t* n);
int lbm_mlp_get_params(lbm_mlp* mlp, float* params);
int lbm_mlp_set_params(lbm_mlp* mlp, const float* params);

/* Outputs y [n, sizes[nlayers]] (device, float32) of inputs x [n, sizes[0]]
 * (device, float32), any n >= 0 (processed in chunks of max_batch; x and y
 * may be NULL when n = 0).  Async. */
int lbm_mlp_forward(lbm_mlp* mlp, const float* x, float* y, int64_t n);

/* For a network with 6 outputs read as M (xx, xy, xz, yy, yz, zz): the
 * outputs into m6 [n, 6] and D of Eq. 4 of each predicted M into D [n]
 * (device float64), any n >= 0 (n = 0 launches nothing and accepts NULL
 * buffers).  Async. */
int lbm_mlp_deformation(lbm_mlp* mlp, const float* x, int64_t n, float* m6, double* D);

/* Loss and gradients of n samples (32 <= n <= max_batch, n % 32 == 0;
 * x, t device float32) without updating: *loss (host, may be NULL) and grads
 * (host, the flat parameter layout, may be NULL).  Synchronises. */
int lbm_mlp_gradients(lbm_mlp* mlp, const float* x, const float* t, int64_t n, double* loss, float* grads);

/* One Adam step with learning rate lr on n samples (as lbm_mlp_gradients);
 * loss (host) NULL keeps the call asynchronous. */
int lbm_mlp_train_step(lbm_mlp* mlp, const float* x, const float* t, int64_t n, float lr, double* loss);

/* Wait for the network's stream; LBM_ETIMEOUT if a bounded tensor-core wait gave up. */
int lbm_mlp_sync(lbm_mlp* mlp);

/* Matrix products: path 0 (default) runs tcgen05 tensor cores on every
 * product whose M and N are multiples of 128, K of 64, and whose operand,
 * output, bias and mask rows start on 16-byte boundaries (inputs x that are
 * not 16-byte aligned still run, through the scalar normalisation); warp-level
 * mma.sync takes the rest.  Path 1 runs mma.sync only.  Both accumulate in
 * float32.  LBM_EINVAL for a path other than 0 or 1. */
int lbm_mlp_set_tensor_path(lbm_mlp* mlp, int32_t path);
void lbm_mlp_destroy(lbm_mlp* mlp);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
