/*
 * nopcs.h -- C ABI of the GB300 (sm_103a) NOHAP/OUCS3 compressible Navier-Stokes
 * hot path.
 *
 * The method is that of Sundaram, Sengupta & Sengupta, "Ultrasound triggering of
 * Rayleigh-Taylor instability: solution of compressible Navier-Stokes equation
 * by a non-overlapping parallel compact scheme" (arXiv 2203.00879):
 *   - OUCS3 compact first derivative [A]{f'} = [B]{f} (Sec. 3, Eq. CS:AfpBf and
 *     the interior coefficients printed after it), solved per non-overlapping
 *     sub-domain with the NOHAP closure: sub-domain end points from the
 *     equivalent explicit scheme f'_i = sum_k C_ik f_{i+k}, C = A^-1 B
 *     (Eqs. CS:fpCf, CS:fpCf_i), interior points by the Thomas algorithm;
 *   - the nondimensional compressible Navier-Stokes right-hand side with bulk
 *     viscosity (Sec. 2, Eqs. ge1-ge20, reg, bv1-bv3), gravity source (Eq. ge8a),
 *     classical RK4 and the implicit filter with coefficient 0.135 every 50 steps
 *     (Sec. 4, first paragraph).
 *
 * Conventions (all entry points):
 *   - Every call returns a nopcs_status and never aborts or throws.  On an error
 *     other than NOPCS_ECUDA the context stays usable; nopcs_last_error() gives a
 *     message.  Arguments are validated before any device work.
 *   - Fields are SoA, x fastest: element (i, j, k) of an nx x ny x nz box is at
 *     i + nx * (j + ny * k).  A state is 5 such fields in the order
 *     rho, rho u, rho v, rho w, E (total energy per unit volume), nondimensional.
 *   - Caller-owned buffers passed to an entry point are only read or written
 *     during the work that call enqueues; the library keeps no pointer to them.
 *     The library owns the state registers, scratch, operator tables and CUDA
 *     graphs of a context and frees them in nopcs_destroy().
 *   - Streams are cudaStream_t values passed as void* (NULL = legacy default).
 *   - The library runs on the CUDA device current at nopcs_init().  Every
 *     later call on the context must be made with that device current, else
 *     it returns NOPCS_EINVAL and enqueues nothing; nopcs_destroy() switches
 *     to the context's device itself and switches back.
 *   - Device memory: nopcs_init allocates a context's registers, scratch and
 *     tables; nopcs_derivative(order = 2) allocates its scratch on first use.
 *     An allocation that fails, or that would take the context beyond the
 *     limit of nopcs_set_memory_limit, is NOPCS_ENOMEM, and a failed
 *     nopcs_init frees everything it had allocated.
 */
#ifndef NOPCS_H
#define NOPCS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nopcs_ctx nopcs_ctx; /* opaque, library-owned */

typedef enum {
    NOPCS_OK = 0,
    NOPCS_EINVAL = 1,      /* bad argument; nothing was enqueued                */
    NOPCS_ENOMEM = 2,      /* device or host allocation failed                  */
    NOPCS_ECUDA = 3,       /* a CUDA call failed; the context should be destroyed */
    NOPCS_EUNSTABLE = 4,   /* non-finite values found in the state              */
    NOPCS_ETIMEOUT = 5,    /* a bounded device wait gave up                     */
    NOPCS_EUNSUPPORTED = 6 /* valid request that is not implemented             */
} nopcs_status;

typedef enum {
    NOPCS_FP64 = 0, /* fluxes, derivatives, viscous terms and state in FP64      */
    NOPCS_MIXED = 1 /* FP32 fluxes/derivatives/viscous terms on the state minus its
                       hydrostatic base; FP64 state and RK accumulation          */
} nopcs_precision;

typedef enum {
    NOPCS_FORM_AUTO = 0,   /* per box and axis, the fastest form for FP32       */
                           /* derivatives, measured at nopcs_init               */
    NOPCS_FORM_THOMAS = 1, /* per-sub-domain Thomas sweeps                      */
    NOPCS_FORM_GEMM_3XTF32 = 2, /* FP32 derivatives on the tensor cores (tcgen05, */
                                /* split TF32); FP64 ones keep the Thomas form    */
    NOPCS_FORM_GEMM_BF16X3 = 3, /* FP32 derivatives on the tensor cores in three  */
                                /* BF16 parts per operand (tcgen05 kind::f16, six */
                                /* products); FP64 ones keep the Thomas form      */
    NOPCS_FORM_BANDED = 4  /* FP32 derivatives as the equivalent explicit scheme */
                           /* (Eq. CS:fpCf_i) at every row: rows of the global  */
                           /* C = A^-1 B truncated at 1e-8, no Thomas; FP64     */
                           /* ones keep the Thomas form.  The flux sweeps of    */
                           /* the RK step use Thomas under every form.          */
} nopcs_form;

/*
 * One box of the two-temperature Rayleigh-Taylor problem (Sec. 2, Fig. 1).
 * Caller-owned; copied by nopcs_init.  Nondimensionalisation of Eqs. ge14/ge15:
 * lengths by L, velocity by U_s = sqrt(gL), time by L/U_s, density by rho_s,
 * pressure and energy by rho_s U_s^2 (so p = rho T / (gamma M^2)), temperature
 * by T_s.
 */
typedef struct {
    int n[3];              /* grid points per axis, >= 5, product < 2^31; nodes    */
                           /* lie on the walls                                      */
    double len[3];         /* box lengths; spacing h = len / (n - 1)                */
    int gravity_axis;      /* 0, 1 or 2: gravity points along -axis; the interface  */
                           /* is the mid-plane normal to it                          */
    int sub_n[3];          /* NOHAP sub-domain length per axis (>= 3); 0 or >= n:   */
                           /* one sub-domain; -1: the autotuner picks 32, 64 or 128 */
                           /* by timing this GPU at nopcs_init                      */
    double Re, M, Pr, gamma;
    double suth_S;         /* Sutherland constant / T_s                             */
    double mub_scale;      /* factor on the bulk-viscosity law, Eq. reg             */
    double mu_s_si;        /* dimensional viscosity at T_s, Pa s (mu_b / mu_s)      */
    double Ts_kelvin;      /* T_s in kelvin (Eq. reg takes T* in kelvin)            */
    double T_upper, T_lower; /* nondimensional temperatures of the two halves       */
    double g;              /* nondimensional gravity g L / U_s^2 (1)                 */
    double dt;             /* nondimensional time step                              */
    int filter_every;      /* filter after every this many steps; 0 = never         */
    double filter_alpha;   /* filter coefficient (0.135)                            */
    int base_subtract;     /* 1: differentiate p - p_h, source -(rho - rho_h) g.    */
                           /* Forced to 1 under NOPCS_MIXED.                         */
    unsigned long long seed; /* seed of the initial velocity perturbation           */
    double perturb_amp;    /* amplitude of the uniform velocity perturbation        */
    int visc_compact;      /* 0: the paper's second-order explicit viscous terms    */
                           /* (Sec. 4).  1: the gradients of u, v, w, T and the     */
                           /* divergence of the viscous fluxes by the NOHAP/OUCS3   */
                           /* operator of the convective terms, with the same wall  */
                           /* rows and sub-domains -- an option beyond the paper;   */
                           /* it holds 12 more fields of scratch (FP32 under        */
                           /* NOPCS_MIXED, FP64 under NOPCS_FP64) per box           */
} nopcs_box_desc;

typedef struct {
    double mass;           /* sum of rho times h_x h_y h_z                          */
    double momentum[3];
    double energy_total;   /* sum of E + rho g z, times the cell volume             */
    double max_speed;      /* max |V|                                               */
    double max_dp;         /* max |p - p_h| (disturbance pressure, Sec. 4)          */
    double max_mach;       /* max |V| M / sqrt(T)                                   */
    long long step;        /* RK steps taken by this box                            */
    int nonfinite;         /* 1 if any state value is NaN or Inf                    */
} nopcs_diag;

/*
 * Create a context for `nboxes` independent boxes, build the operator tables
 * (Sec. 3: global C rows for sub-domain ends, Thomas factors), allocate the
 * three FP64 RK registers plus scratch per box on the current device, and set
 * every box to its initial state (quiescent hydrostatic two-temperature box
 * with a SplitMix64 velocity perturbation on interior nodes).
 * `stream` (cudaStream_t or NULL) is the stream of all later state work.
 * Errors: EINVAL (n < 5, nboxes < 1, bad enum, sub_n in 1..2, ...), ENOMEM,
 * ECUDA.  On error *out is NULL.
 */
nopcs_status nopcs_init(const nopcs_box_desc *boxes, int nboxes, nopcs_precision prec,
                        nopcs_form form, void *stream, nopcs_ctx **out);

/* Free everything the context owns (waits for its stream).  NULL is a no-op. */
void nopcs_destroy(nopcs_ctx *ctx);

/*
 * Cap, in bytes, on the device memory that each context created afterwards
 * may hold (its state registers, scratch and operator tables); 0 (the
 * default) removes the cap.  Process-wide.  A nopcs_init that would exceed it
 * returns NOPCS_ENOMEM with nothing left allocated; so does a later order-2
 * nopcs_derivative whose scratch would exceed it.  The paper has no
 * counterpart: this serves callers with a fixed memory budget per job.
 */
nopcs_status nopcs_set_memory_limit(unsigned long long bytes);

/* Message of the last failed call on this context (or of the last failed
 * nopcs_init when ctx is NULL); never NULL. */
const char *nopcs_last_error(const nopcs_ctx *ctx);

/*
 * Copy a state (5 FP64 fields, np = nx*ny*nz each) into / out of box `box`.
 * `q` may be host (pageable or pinned) or device memory; the copy is enqueued
 * on the context stream and the call returns after it completes.
 */
nopcs_status nopcs_set_state(nopcs_ctx *ctx, int box, const double *q);
nopcs_status nopcs_get_state(nopcs_ctx *ctx, int box, double *q);

/*
 * Staged state upload, for callers that stream a sequence of states through a
 * box (ensemble members, restarts): the copy of the next state overlaps the
 * work on the current one.  The paper has no counterpart.
 *
 * nopcs_stage_state enqueues the copy of a state (5 FP64 fields, np each, the
 * layout of nopcs_set_state; host memory -- pinned for full speed -- or device
 * memory) into the box's staging buffer on the context's copy stream and
 * returns without waiting.  The copy starts once the previous commit of the
 * box has read the staging buffer.  `q` must stay valid and unchanged until
 * the state has been committed and a later nopcs_diagnostics or
 * nopcs_synchronize call has returned.
 *
 * nopcs_commit_state makes the staged state the box's current state, ordered
 * on the context stream after the work already enqueued there: the stream
 * waits for the staging copy, the staged state replaces Q_n (a device copy)
 * and the derived fields are refreshed, as nopcs_set_state does.  It returns
 * without waiting; the step counter is unchanged.
 *
 * The staging buffer (5 np doubles) is allocated by the first
 * nopcs_stage_state of a box and counted against nopcs_set_memory_limit; it is
 * freed with the context.  Errors: EINVAL (bad box, q NULL, a commit with no
 * staged state), ENOMEM (the staging buffer), ECUDA.
 */
nopcs_status nopcs_stage_state(nopcs_ctx *ctx, int box, const double *q);
nopcs_status nopcs_commit_state(nopcs_ctx *ctx, int box);

/* Reset box `box` to its initial state and its step counter to 0. */
nopcs_status nopcs_reset_state(nopcs_ctx *ctx, int box);

/*
 * Set box `box`'s RK step counter (the count the filter cadence of Sec. 4,
 * every filter_every steps, is taken from), e.g. to resume from a checkpoint
 * written with nopcs_get_state and the `step` of nopcs_diagnostics: after
 * nopcs_set_state and nopcs_set_step the box continues exactly as the run
 * that wrote the checkpoint.  Errors: EINVAL (step < 0, bad box).
 */
nopcs_status nopcs_set_step(nopcs_ctx *ctx, int box, long long step);

/*
 * NOHAP compact derivative of one field of box `box`'s shape along `axis`
 * (0 = x, 1 = y, 2 = z).  order 1: the OUCS3 first derivative (Sec. 3),
 * scaled by 1/h.  order 2: the first-derivative operator applied twice
 * (the paper prints no compact second derivative; this reading is stated in the
 * design notes).  order NOPCS_ORDER_D2_COMPACT (3): the sixth-order tridiagonal
 * compact second derivative of Lele (alpha 2/11, a 12/11, b 3/11), scaled by
 * 1/h^2, with its own NOHAP closure (end rows of its global C = A^-1 B) and the
 * wall rows stated in the design notes; always the Thomas form.
 * dtype 0: f and df are FP64 and the arithmetic is FP64 with C
 * rows truncated at |C| < 1e-16 (48 taps each side, Sec. 3); dtype 1: FP32 with
 * C rows truncated at |C| < 1e-8 (24 taps each side).  f and df are device
 * pointers of np elements, must not overlap; the work is enqueued on `stream`
 * and the call does not wait.  order 2 uses library-owned scratch of np
 * elements.  Errors: EINVAL, ECUDA.
 */
enum { NOPCS_ORDER_D2_COMPACT = 3 };
nopcs_status nopcs_derivative(nopcs_ctx *ctx, int box, int axis, int order, int dtype,
                              const void *f, void *df, void *stream);

/*
 * Allocation-free form of nopcs_derivative(order = 2).  The paper has no
 * counterpart: this is a service for callers that cannot let the library
 * allocate device memory during a call (their device memory belongs to their
 * own pool allocator, or the implicit synchronisation of cudaMalloc/cudaFree
 * is not acceptable in their loop), whereas nopcs_derivative allocates its
 * order-2 scratch on first use.  Same arguments, result and arithmetic as
 * nopcs_derivative with order 2, including the form of each axis's FP32
 * derivative (Thomas, banded or tensor-core, as chosen at nopcs_init), so the
 * two give identical bits; the intermediate first derivative lives in a fixed
 * 16 MiB array in the library's device image.  Limits and behaviour:
 *   - the array becomes resident on a device when the first context is
 *     created there (nopcs_init looks up its device address, with that
 *     device current) and stays until the process exits; no call of this
 *     entry point loads a module or looks the address up again;
 *   - fields of at most 2^21 FP64 or 2^22 FP32 points; larger ones return
 *     NOPCS_EINVAL with a message (nothing is enqueued);
 *   - all calls share the one array, so two calls whose work overlaps on the
 *     GPU (different streams, no ordering between them) race on it; the array
 *     keeps the last call's contents, and each call overwrites every element
 *     it reads before reading it;
 *   - no cudaMalloc, cudaFree or other allocating routine is called.
 * Errors: EINVAL (as nopcs_derivative, plus the size limit), ECUDA.
 */
nopcs_status nopcs_derivative2_noalloc(nopcs_ctx *ctx, int box, int axis, int dtype, const void *f, void *df,
                                       void *stream);

/*
 * Advance every box by `nsteps` classical RK4 steps of dt (Sec. 4), applying
 * the no-slip adiabatic wall conditions after every stage and the filter after
 * every filter_every steps (counted per box from its initial state).  Enqueued
 * on the context stream; the call returns without waiting.  Errors: EINVAL
 * (nsteps < 0), ECUDA.
 */
nopcs_status nopcs_rk_step(nopcs_ctx *ctx, int nsteps);

/*
 * How nopcs_rk_step launches a step of the context's boxes (profiling off):
 *   NOPCS_LAUNCH_GRAPH (default): one CUDA graph per step, captured at the
 *     first step, one branch per box;
 *   NOPCS_LAUNCH_PERSISTENT: one persistent kernel per step that runs every
 *     box's phases (flux sweeps, viscous/source/RK stage, walls) from a device
 *     work list, each phase of a box after the box's previous phase, every
 *     wait bounded by wait_limit_s; results are identical to the graph's;
 *   NOPCS_LAUNCH_PERSISTENT_WITHHOLD: as PERSISTENT, but box 0's first
 *     dependency is never satisfied -- for testing the bounded wait: the
 *     kernel gives up after wait_limit_s and returns, nopcs_synchronize
 *     returns NOPCS_ETIMEOUT, and the boxes' states are undefined (reset or
 *     set them before stepping again).
 * The persistent modes need every box in NOPCS_MIXED with visc_compact = 0
 * (else NOPCS_EUNSUPPORTED).  The paper has no counterpart: it runs one box
 * per MPI job.  Errors: EINVAL (mode, wait_limit_s not in (0, 3600]),
 * EUNSUPPORTED, ENOMEM, ECUDA.
 */
enum { NOPCS_LAUNCH_GRAPH = 0, NOPCS_LAUNCH_PERSISTENT = 1, NOPCS_LAUNCH_PERSISTENT_WITHHOLD = 2 };
nopcs_status nopcs_set_launch(nopcs_ctx *ctx, int mode, double wait_limit_s);

/*
 * Evaluate the right-hand side of Eq. ge17 for the FP64 state `q` (device, 5
 * fields) of box `box` into `r` (device, 5 fields, FP64 under NOPCS_FP64 and
 * FP32 under NOPCS_MIXED), with exactly the arithmetic one RK stage uses.  The
 * momentum right-hand side is zero on wall nodes (no-slip).  Waits for
 * completion.  Does not change the box state.
 */
nopcs_status nopcs_rhs(nopcs_ctx *ctx, int box, const double *q, void *r);

/* Apply the filter (Sec. 4) to box `box`'s state now.  Enqueued; no wait. */
nopcs_status nopcs_filter(nopcs_ctx *ctx, int box);

/*
 * Reduce box `box`'s state to the diagnostics above (FP64 accumulation in a
 * fixed order, so repeated calls on the same state give identical bits).
 * Waits for the context stream.  Returns NOPCS_EUNSTABLE (with *out filled) if
 * the state holds a non-finite value.
 */
nopcs_status nopcs_diagnostics(nopcs_ctx *ctx, int box, nopcs_diag *out);

/*
 * Plane diagnostics of Sec. 4 from box `box`'s current FP64 state, on the
 * plane normal to `axis` (0, 1, 2) at node `index`:
 *   what = NOPCS_PLANE_DP (0): the disturbance pressure p - p_h, 1 field;
 *   what = NOPCS_PLANE_VORTICITY_TERMS (1): the three right-hand-side terms
 *     of the inviscid vorticity transport equation (Eq. eqn12_1) -- vortex
 *     stretching (omega . grad) V, dilatation -omega (div V) and the
 *     baroclinic term (grad rho x grad p) / rho^2 -- x, y, z components each,
 *     9 fields in that order; omega = curl V and every gradient is the
 *     second-order explicit difference of the viscous terms (central inside,
 *     one-sided on a wall).
 * out: caller-owned device array of nfields x n_b x n_a doubles, where a < b
 * are the two other axes and a runs fastest.  Enqueued on the context stream
 * (nopcs_synchronize waits).  Errors: EINVAL for a bad axis, index or `what`.
 */
enum { NOPCS_PLANE_DP = 0, NOPCS_PLANE_VORTICITY_TERMS = 1 };
nopcs_status nopcs_plane_fields(nopcs_ctx *ctx, int box, int axis, int index, int what, double *out);

/*
 * Choices in force for box `box` (caller arrays of 3 ints, any may be NULL):
 * the sub-domain length per axis (the autotuner's pick where the descriptor
 * asked for -1), the form of the FP32 derivative per axis (NOPCS_FORM_THOMAS,
 * NOPCS_FORM_GEMM_3XTF32, NOPCS_FORM_GEMM_BF16X3 or NOPCS_FORM_BANDED) and the
 * flux sweeps' tile width per axis (grid lines per CUDA block; 0 = the
 * precision's default, untuned for small boxes).
 */
nopcs_status nopcs_box_info(nopcs_ctx *ctx, int box, int *sub_n, int *deriv_form, int *tile_lines);

/* Wait for all work enqueued on the context stream. */
nopcs_status nopcs_synchronize(nopcs_ctx *ctx);

/*
 * Per-kernel timing.  With profiling on, nopcs_rk_step launches its kernels
 * directly (no CUDA graph) between pairs of CUDA events on the context stream;
 * nopcs_profile_read waits for the stream and returns, per kernel kind, the
 * summed event time in milliseconds and the launch count since the last reset
 * (arrays of NOPCS_NUM_KERNELS entries).  nopcs_kernel_name gives the kind's
 * name (static string; NULL for an out-of-range id).
 */
#define NOPCS_NUM_KERNELS 12
nopcs_status nopcs_set_profiling(nopcs_ctx *ctx, int on);
nopcs_status nopcs_profile_read(nopcs_ctx *ctx, double *ms, long long *launches, int reset);
const char *nopcs_kernel_name(int kind);

/*
 * Host-side operator tables, for inspection and tests; needs no GPU.
 * For a line of N points split into sub-domains of sub_n (kind 0: OUCS3 first
 * derivative, dimensionless, i.e. times h; kind 1: filter with coefficient
 * `alpha_f`), C rows truncated at |C| < thresh:
 *   starts[0..nsub]      sub-domain starts and N (caller array of N+1 ints),
 *   end_j0[2*nsub], end_len[2*nsub]  first column and tap count of the end row
 *                        of each sub-domain (start, then end),
 *   coef[]               the concatenated taps (capacity max_coef doubles).
 * Returns EINVAL on bad sizes or too small buffers; *nsub is set on success.
 */
nopcs_status nopcs_operator_rows(int N, int sub_n, int kind, double alpha_f, double thresh,
                                 int *nsub, int *starts, int *end_j0, int *end_len,
                                 double *coef, int max_coef);

/*
 * Host evaluation of the same line operator, FP64, the arithmetic of the line
 * kernels (end rows from C, Thomas with tabulated factors), for inspection and
 * tests; needs no GPU.  f and g are host arrays of N doubles; g = L f
 * (dimensionless: divide by h for a derivative).  Errors: EINVAL.
 */
nopcs_status nopcs_operator_apply(int N, int sub_n, int kind, double alpha_f, double thresh, const double *f,
                                  double *g);

/*
 * Host evaluation of the banded explicit form of the same line operator
 * (NOPCS_FORM_BANDED): the equivalent explicit scheme g_i = sum_j C_ij f_j of
 * Sec. 3 (Eqs. CS:fpCf, CS:fpCf_i), applied at every row instead of at the
 * sub-domain ends only, with the rows of the global C = A^-1 B truncated at
 * |C| < thresh.  Rows in [*interior_lo, *interior_hi] use one stencil of
 * offsets -*half_width .. *half_width; the rows near the walls use their own
 * tabulated windows.  FP64, needs no GPU; f and g are host arrays of N
 * doubles, g dimensionless as for nopcs_operator_apply.  The three outputs may
 * be NULL.  Errors: EINVAL.
 */
nopcs_status nopcs_band_apply(int N, int kind, double alpha_f, double thresh, const double *f, double *g,
                              int *half_width, int *interior_lo, int *interior_hi);

/*
 * ---- One box split into z-slabs across ranks (Sec. 3; the rank grid of Sec. 4)
 *
 * A rank that owns the planes [z0, z1) of a box -- whole NOHAP sub-domains of
 * the z lines -- computes the derivative of its planes from them plus the
 * halo planes [lo, z0) and [z1, hi) that the sub-domain end rows (rows of the
 * global C = A^-1 B, Eqs. CS:fpCf, CS:fpCf_i, reaching n_b = 48 points in FP64
 * and 24 in FP32) and the interior stencil reach.  The caller receives those
 * halo planes from the neighbouring ranks into its own memory (e.g. NCCL
 * send/recv; no remote loads); the result on [z0, z1) is then that of the
 * single-domain solve of the whole box, bit for bit.  A slab holds operator
 * tables only (a few KB), no field.
 *
 * nopcs_slab_create: `box` is the whole box (its n, len and sub_n are used;
 * sub_n must be 0 or >= 3, no tuning); z0 and z1 must be sub-domain
 * boundaries of the z partition.  Tables go to the current device.  Errors:
 * EINVAL (sizes, unaligned slab), ENOMEM, ECUDA.  On error *out is NULL and
 * nopcs_slab_last_error(NULL) has the message.
 */
typedef struct nopcs_slab nopcs_slab; /* opaque, library-owned */
nopcs_status nopcs_slab_create(const nopcs_box_desc *box, int z0, int z1, nopcs_slab **out);
void nopcs_slab_destroy(nopcs_slab *slab);
const char *nopcs_slab_last_error(const nopcs_slab *slab);

/* Planes [*lo, *hi) of the box that a slab's local field of `dtype` (0 f64,
 * 1 f32) holds: own planes plus halo, lo <= z0 < z1 <= hi. */
nopcs_status nopcs_slab_extent(const nopcs_slab *slab, int dtype, int *lo, int *hi);

/*
 * NOHAP first derivative along `axis` of a slab's field: f (device) holds the
 * planes [lo, hi) of nopcs_slab_extent (nx*ny values each, x fastest), the
 * halo planes already received; df (device) receives the own planes [z0, z1)
 * only, nx*ny*(z1 - z0) values.  Along x and y only the own planes of f are
 * read.  FP64 (dtype 0) or FP32 (dtype 1) as nopcs_derivative order 1,
 * Thomas form.  Enqueued on `stream`; no wait.  Must be called with the
 * slab's device current.  Errors: EINVAL, ECUDA.
 */
nopcs_status nopcs_slab_derivative(nopcs_slab *slab, int axis, int dtype, const void *f, void *df, void *stream);

/*
 * Host FP64 evaluation of the same restricted line operator, for inspection
 * and tests (needs no GPU): a line of N points with sub-domains of sub_n and
 * end-row taps truncated at `thresh`; f holds points [*lo, *hi) (set on
 * return; pass f = g = NULL to query them only), g receives points
 * [z0, z1), dimensionless (times h).  Errors: EINVAL.
 */
nopcs_status nopcs_slab_line_apply(int N, int sub_n, double thresh, int z0, int z1, const double *f, double *g,
                                   int *lo, int *hi);

#ifdef __cplusplus
}
#endif
#endif /* NOPCS_H */
