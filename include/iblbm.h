/*
 * iblbm.h -- C ABI of the B300 (sm_103a) immersed-boundary lattice Boltzmann
 * library (libiblbm.so).
 *
 * The library advances D2Q9 lattice Boltzmann flows coupled to rigid bodies
 * given as Lagrangian marker sets, following H. Jo, "Mechanism-Resolved
 * Interface Momentum Transfer in Immersed-Boundary Lattice Boltzmann
 * Simulations":
 *   - stream + collide with BGK (Eq. 1-3), TRT or central-moment MRT (Eq. 5,
 *     Sec. 2.2) and Guo forcing with the half-force velocity of Eq. 4;
 *   - marker interpolation (Eq. 7) and spreading (Eq. 8) with the hat (Eq. 9)
 *     or Peskin 4-point (Eq. 10) kernel;
 *   - direct forcing (Eq. 11), multi-direct forcing (Eq. 12-14) and
 *     distribution-function correction (Eq. 15-20);
 *   - FP64 rigid-body Velocity-Verlet (Eq. 21-23) with the internal-mass
 *     correction of Eq. A3.
 *
 * Conventions shared by every call:
 *   Units      lattice units, dx = dt = 1, rho_f = 1 (Sec. 2.1, App. A.1).
 *   Layout     host population arrays are double, unshifted, one plane per
 *              direction: f[(i*ny + y)*nx + x], i in 0..8 with
 *              e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1)
 *              e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1).
 *              The state between steps is the post-collision field.
 *   Ownership  inputs are copied in; the caller keeps its arrays.  Outputs go
 *              to caller-allocated host buffers of the documented size.
 *              Device memory belongs to the context; it comes from the
 *              allocator installed with iblbm_set_allocator (else cudaMalloc).
 *   Streams    all device work of a context is ordered on the stream given in
 *              its lattice descriptor (NULL = legacy default stream).
 *              Calls documented as "syncs" wait for that stream.
 *   Errors     every int-returning call returns IBLBM_OK (0) on success, a
 *              negative IBLBM_ERR_* on error (the context stays usable unless
 *              stated), or a positive IBLBM_WARN_* for a completed call with a
 *              warning.  iblbm_strerror() names each code.
 *   Threads    a context is not thread-safe; use one host thread per context.
 */
#ifndef IBLBM_H
#define IBLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------- */
#define IBLBM_OK 0
#define IBLBM_WARN_MDF_NOT_CONVERGED 1   /* an MDF loop hit N_max or its divergence guard */
#define IBLBM_ERR_INVALID_ARG (-1)
#define IBLBM_ERR_OOM (-2)
#define IBLBM_ERR_UNSTABLE (-3)           /* non-finite or non-positive density seen */
#define IBLBM_ERR_MARKER_OUT_OF_DOMAIN (-4)
#define IBLBM_ERR_BODY_OVERLAP (-5)
#define IBLBM_ERR_TIMEOUT (-6)
#define IBLBM_ERR_NOT_ADMITTED (-7)
#define IBLBM_ERR_BUSY (-8)
#define IBLBM_ERR_CUDA (-9)
#define IBLBM_ERR_NOT_FOUND (-10)
#define IBLBM_ERR_CAPACITY (-11)          /* a buffer given by the caller is too small */

typedef struct iblbm_ctx iblbm_ctx;

/* Collision operator, Sec. 2.2.  IBLBM_STREAM_ONLY is the identity collision
 * (pure streaming), a verification mode with no counterpart in the paper. */
typedef enum { IBLBM_BGK = 0, IBLBM_TRT = 1, IBLBM_CMMRT = 2, IBLBM_STREAM_ONLY = 3 } iblbm_collision;
/* Regularised delta kernel, Sec. 2.4 (Eq. 9, Eq. 10). */
typedef enum { IBLBM_HAT = 0, IBLBM_PESKIN4 = 1 } iblbm_kernel;
/* Boundary-enforcement scheme, Sec. 2.5. */
typedef enum { IBLBM_DF = 0, IBLBM_MDF = 1, IBLBM_DFC = 2 } iblbm_scheme;
/* Population storage: FP64, FP32 shifted (f - w), FP16 shifted with FP32 compute. */
typedef enum { IBLBM_F64 = 0, IBLBM_F32 = 1, IBLBM_F16S = 2 } iblbm_storage;
/* Domain side condition.  VELOCITY is the Zou-He closure at the prescribed
 * velocity (inflow, far-field and no-slip walls of Sec. 2.9); NEUMANN copies
 * the nine post-streaming populations of the adjacent interior node (zero
 * gradient).  PERIODIC must be set on both sides of an axis or on neither. */
typedef enum { IBLBM_BC_PERIODIC = 0, IBLBM_BC_VELOCITY = 1, IBLBM_BC_NEUMANN = 2 } iblbm_bc;
/* Body motion: fixed (or moved by the caller with iblbm_move_body), prescribed
 * in-line oscillation x_c(t) = x_c0 - A sin(2 pi t / T) (Sec. 2.9.2), or free
 * rigid-body dynamics (Sec. 2.7). */
/* IBLBM_FREE_TRANSLATION: free in translation (Eq. 23), rotation held at rest; the paper
 * calls the disks' rotational contribution negligible, and with MDF the torque-only rotation
 * of a free light disk can go unstable (explicit coupling) */
typedef enum { IBLBM_FIXED = 0, IBLBM_PRESCRIBED = 1, IBLBM_FREE = 2, IBLBM_FREE_TRANSLATION = 3 } iblbm_motion;

typedef struct {
    int nx, ny;                 /* lattice nodes, each >= 3 */
    int storage;                /* iblbm_storage */
    int bc[4];                  /* iblbm_bc for the west, east, south, north sides */
    double u_bc[4][2];          /* velocity of each VELOCITY side */
    double trt_lambda;          /* TRT magic parameter Lambda_eo (e.g. 3/16 or 1/4) */
    double cm_sq, cm_se;        /* CM-MRT third/fourth-order rates (paper: 1.2, 1.4) */
    double force[2];            /* uniform body-force density on the fluid (usually 0) */
    double init_rho, init_u[2]; /* initial state: equilibrium at this density/velocity */
    void* cuda_stream;          /* cudaStream_t, NULL = legacy default stream */
    int wall_closure;           /* IBLBM_BC_VELOCITY sides with zero velocity: 0 = the Zou-He
                                   closure with its tangential correction (Sec. 2.9.3 names Zou
                                   and He); 1 = on-node bounce-back of the unknown populations,
                                   the same closure at u = 0 without the tangential correction,
                                   which stays stable with BGK below tau ~ 0.6.  A side takes
                                   the bounce-back form when its u_bc is exactly (0, 0) in FP64;
                                   any other value is INVALID_ARG */
} iblbm_lattice_desc;

typedef struct {
    double xc, yc;              /* body centre (lattice units) */
    double radius;              /* for the masses m_s = rho_s pi r^2, I_s = m_s r^2 / 2 */
    double rho_ratio;           /* rho_s / rho_f */
    int motion;                 /* iblbm_motion */
    double gx, gy;              /* gravity (lattice units), Eq. 22 */
    int internal_mass;          /* 1: scheme (B-2), Eq. A3; 0: scheme (A) */
    int mdf_nmin, mdf_nmax;     /* MDF iteration bounds (paper: 5, 20) */
    double mdf_tol;             /* MDF L_inf slip tolerance (paper: 1e-4) */
    double mdf_omega;           /* MDF relaxation; <= 0 selects 1/||A||_inf */
    double osc_amp, osc_period; /* PRESCRIBED: A and T of x_c(t) */
    int history_cap;            /* force-history ring capacity in steps (<= 0: 65536) */
} iblbm_body_desc;

/* ---- memory --------------------------------------------------------------------- */
/* Installs the device allocator used by every later context (process-wide).
 * alloc(bytes, stream, user) returns a device pointer or NULL; free(ptr, stream,
 * user) releases it.  Pointers should be at least 16-byte aligned (256 like
 * cudaMalloc is best); the bulk-staged stream-collide variant is skipped for a
 * lattice whose population buffers are not.  Passing NULL functions restores
 * cudaMalloc/cudaFree. */
typedef void* (*iblbm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*iblbm_free_fn)(void* ptr, void* stream, void* user);
int iblbm_set_allocator(iblbm_alloc_fn alloc, iblbm_free_fn free_fn, void* user);

/* ---- lattice ---------------------------------------------------------------------- */
/* Creates a lattice context on the current CUDA device (Sec. 2.1-2.2).
 * tau > 1/2 is the relaxation time (nu = (tau - 1/2)/3); BGK/TRT/CM-MRT share it
 * as the viscous rate.  Initialises every node to the equilibrium at
 * (init_rho, init_u).  *out receives the context.  Errors: INVALID_ARG, OOM, CUDA. */
int iblbm_create(const iblbm_lattice_desc* desc, int collision, double tau, iblbm_ctx** out);
/* Frees the context and all its device memory (syncs).  NULL is ignored. */
void iblbm_destroy(iblbm_ctx* ctx);

/* Adds a rigid body given by n markers xy[2*n] (x0,y0,x1,y1,...) with arc
 * length ds (Eq. 8), delta kernel and scheme (Sec. 2.3-2.5).  The markers are
 * rigidly attached to the centre (xc, yc).  For MDF with mdf_omega <= 0 the
 * relaxation 1/||A||_inf is computed here once (Sec. 2.5.2); for DFC the
 * factors lambda_k of Eq. 17 are computed on the device.  Every kernel
 * footprint must lie inside the lattice.  *body_id receives the index (0, 1,
 * ...).  A second MDF body in a lattice switches its MDF bodies to the coupled
 * iteration (iblbm_mdf_relaxation) and allocates a lattice-wide scratch of three
 * values per node.  Errors: INVALID_ARG, MARKER_OUT_OF_DOMAIN, OOM.
 * (IBLBM_ERR_BODY_OVERLAP is no longer returned: MDF bodies may share nodes.) */
int iblbm_add_body(iblbm_ctx* ctx, const double* xy, int n, double ds, int kernel, int scheme,
                   const iblbm_body_desc* body, int* body_id);

/* Advances nsteps IB-LBM steps, asynchronously on the context stream (replays
 * a captured CUDA graph).  One step: stream with domain conditions, IB stage of
 * every body, collide, body forces and motion update.  Device-side errors
 * (instability, markers leaving the lattice) are reported by the next syncing
 * call.  Errors: INVALID_ARG, CUDA. */
int iblbm_step(iblbm_ctx* ctx, int nsteps);

/* Waits for the context stream and returns the first device-side error seen,
 * IBLBM_WARN_MDF_NOT_CONVERGED if an MDF loop stopped early, else IBLBM_OK. */
int iblbm_sync(iblbm_ctx* ctx);

/* Steps seen so far. */
long long iblbm_steps_done(const iblbm_ctx* ctx);

/* Force (x, y) and torque on body body_id from the last step, FP64, following
 * the sign rules of Sec. 2.7 (DF/MDF: -sum F_L ds; DFC: sum F_s).  Syncs. */
int iblbm_body_forces(iblbm_ctx* ctx, int body_id, double out[3]);
/* Body centre, velocity and rotation after the last step: xc, yc, vx, vy,
 * omega, theta.  Syncs. */
int iblbm_body_state(iblbm_ctx* ctx, int body_id, double out[6]);
/* Copies the last min(cap, steps) entries of the force history (3 doubles per
 * step, oldest first) into out[3*cap]; *n receives the count.  Syncs. */
int iblbm_force_history(iblbm_ctx* ctx, int body_id, double* out, int cap, int* n);
/* FIXED bodies only: replaces the marker positions (xy[2*n], or NULL to keep
 * them) and sets the rigid velocity uvw = (vx, vy, omega) used for
 * U_d = v + omega x (X - X_c).  Errors: INVALID_ARG (not FIXED), MARKER_OUT_OF_DOMAIN. */
int iblbm_move_body(iblbm_ctx* ctx, int body_id, const double* xy, const double uvw[3]);

/* FIXED bodies only: sets the desired velocity U_d,k of every marker, ud[2*n] =
 * (U_d,x, U_d,y) per marker in lattice units (|component| < 1), used by the IB
 * stage (Eq. 13) from the next step on instead of v + omega x (X - X_c), until
 * the next call, iblbm_move_body with uvw, or ud = NULL (back to the rigid
 * velocity).  App. D.1 drives markers this way with the analytical Taylor-Green
 * field.  The setting is not part of a checkpoint.  Errors: INVALID_ARG (bad
 * body, not FIXED, a component out of range).  Syncs. */
int iblbm_set_marker_velocity(iblbm_ctx* ctx, int body_id, const double* ud);
/* Per-marker data of the last step into out[7*n]: X, Y, U_d,x, U_d,y, force x,
 * force y (DF: F_L, MDF: F_total, DFC: F_s), lambda_k (DFC, else 0).  Syncs. */
int iblbm_marker_data(iblbm_ctx* ctx, int body_id, double* out);
/* Stencil origin (i0, j0) of each marker for the last step into ij[2*n]: the
 * footprint is i0..i0+S-1 x j0..j0+S-1, S = 2 (hat) or 4 (Peskin).  Syncs. */
int iblbm_marker_stencils(iblbm_ctx* ctx, int body_id, int* ij);
/* Local boundary-fidelity diagnostics of Sec. 2.8 for body body_id on the state
 * after the last step, with the bilinear probe of Sec. 4.2.  The fluid fields
 * are the density and Eq. 4 velocity of the last collision (as iblbm_get_macro);
 * X_k, U_d,k and F_k are the marker data of iblbm_marker_data; u_ref > 0 is the
 * reference speed (U_inf), kappa >= 0 the buffer width in lattice units (the
 * paper takes 2).  out[8]:
 *   [0] mean over markers of |U(X_k) - U_d,k| / u_ref, U interpolated with the
 *       body's kernel (Eq. 7): the slip error eps_slip
 *   [1] max over markers of the same
 *   [2] max over markers of the same with U from the bilinear probe
 *   [3] leakage Phi_leak: sum_k rho(X_k) (U - U_d,k).n_k ds / (u_ref n ds), n_k the
 *       outward unit normal of the chord X_{k+1} - X_{k-1} (radial when n < 3);
 *       n ds is pi D for a circle
 *   [4] the same with |(U - U_d,k).n_k| (gross flux)
 *   [5] mean over nodes with |x - X_c| < R - kappa (strict; R the body radius) of
 *       |u(x) - (v + omega x (x - X_c))| / u_ref: the internal residual velocity
 *   [6] the number of those nodes
 *   [7] sum_k |F_k|
 * per_marker[5*n] (host, may be NULL): per marker [0] and the bilinear slip,
 * (U - U_d,k).n_k / u_ref, (rho_bilinear(X_k) - 1) c_s^2 and |F_k|.  Sums are
 * FP64.  Errors: INVALID_ARG, MARKER_OUT_OF_DOMAIN (a stencil or probe node
 * outside the lattice), OOM.  Syncs. */
int iblbm_local_diagnostics(iblbm_ctx* ctx, int body_id, double u_ref, double kappa, double out[8],
                            double* per_marker);
/* MDF diagnostics of the last step: increments applied, last L_inf residual
 * (FP64) and omega_MDF.  Syncs. */
int iblbm_mdf_info(iblbm_ctx* ctx, int body_id, int* iterations, double* residual, double* omega);
/* Relaxation factor in use when the body's last MDF iteration ended.  A lattice with
 * two or more MDF bodies iterates them coupled (Sec. 2.5.2): one fluid update per
 * iteration shared by every MDF body, omega starting at min(0.8, omega_MDF of the
 * bodies) and halved for every trial iteration whose L_inf residual (over all their
 * markers) grows by more than 20 %, the iteration ending at 0.125 of the start value;
 * iblbm_mdf_info then reports the trial iterations (rejected ones included) and the
 * joint residual, the same for every coupled body.  A single MDF body keeps omega_MDF
 * (this call returns it).  Syncs.  Errors: INVALID_ARG. */
int iblbm_mdf_relaxation(iblbm_ctx* ctx, int body_id, double* omega_end);

/* Post-collision populations into f[9*nx*ny] (layout above).  shifted = 0
 * returns f; shifted = 1 returns the stored values f - w_i exactly as held in
 * device memory, widened to double.  Syncs. */
int iblbm_get_populations(iblbm_ctx* ctx, double* f, int shifted);
/* Replaces the post-collision state with f[9*nx*ny] (unshifted, layout above);
 * values are rounded to the storage precision after the shift.  Syncs. */
int iblbm_set_populations(iblbm_ctx* ctx, const double* f);
/* Density and Eq. 4 velocity of the last collision into rho/ux/uy[nx*ny]
 * (row-major y, x), computed from the post-collision state.  Syncs. */
int iblbm_get_macro(iblbm_ctx* ctx, double* rho, double* ux, double* uy);

/* Whole-state checkpoint (populations, body state, markers) into host memory.
 * host may be NULL to query the size into *n.  Errors: CAPACITY.  Syncs. */
int iblbm_snapshot(iblbm_ctx* ctx, void* host, size_t cap, size_t* n);
/* Restores a checkpoint written by iblbm_snapshot of a context with the same
 * lattice and bodies.  Errors: INVALID_ARG.  Waits for this context's own stream
 * only (before the copies and after them, so host may be reused on return); work
 * queued on other contexts keeps running, which lets a caller copy one lattice
 * in while others step. */
int iblbm_restore(iblbm_ctx* ctx, const void* host, size_t n);

/* Device bytes held by the context. */
size_t iblbm_device_bytes(const iblbm_ctx* ctx);

const char* iblbm_strerror(int status);

/* ---- batched stepping (one launch sequence for many cases) ------------------------- */
/* Advances every context in ctxs[0..n) by nsteps steps with one launch per kernel
 * per storage type per step, over a case/tile table (uneven lattices allowed).
 * All contexts must live on the current device; the work is ordered on
 * ctxs[0]'s stream after the other contexts' streams.  Results are identical to
 * stepping each context alone.  Errors: INVALID_ARG, CUDA. */
int iblbm_step_batch(iblbm_ctx** ctxs, int n, int nsteps);

/* ---- stream-collide kernel variants (tuning control; no counterpart in the paper) ---- */
/* IBLBM_KERNEL_VARIANTS implementations of the fused stream-collide exist:
 * 0 keeps a 16-byte vector of nodes per lane, 1 one node per lane, 2 two nodes
 * per lane, 3 stages each tile's source rows in shared memory with bulk
 * asynchronous copies (needs 16-byte aligned population buffers, see
 * iblbm_set_allocator; otherwise variant 1 runs in its place and its tuning
 * time reads 0).  By default the first batch that needs a (storage, collision)
 * pair times all of them in place and keeps the fastest for the rest of the
 * process; groups sweeping fewer than 2^20 nodes per launch (latency-bound) are
 * tuned apart from larger ones, so a lattice runs the same kernel alone,
 * batched or served within its size class.
 * iblbm_set_kernel_variant fixes the choice for both classes (-1 = tune again);
 * iblbm_kernel_variant reports the large-class choice once tuned, else the small
 * one (-1 = not chosen) and, if ms is not NULL, writes the mean launch time of
 * each variant measured when it was tuned into ms[IBLBM_KERNEL_VARIANTS].
 * Errors: INVALID_ARG. */
#define IBLBM_KERNEL_VARIANTS 4
int iblbm_set_kernel_variant(int storage, int collision, int variant);
/* Test hook of the bounded device wait (no counterpart in the paper).  The bulk
 * variant's consumer warps wait for each staged tile for at most a fixed number
 * of polls and then give up: the launch raises IBLBM_ERR_TIMEOUT in the status
 * of the lattice it was sweeping, and its producer waits (bounded, unchanged by
 * this call) for the copies it still has in flight before the CTA exits.  This
 * call sets that consumer poll count process-wide (polls >= 0; 0 gives up at
 * the first wait) or restores the default bound (polls < 0), so a test can run
 * the give-up path without a copy that never lands.  A step taken while it is
 * lowered leaves the lattice's populations undefined.  Syncs the device.
 * Errors: CUDA. */
int iblbm_test_set_consumer_poll_limit(long polls);
/* Test hook: enable != 0 (the default) lets the IB stage of a fixed DF or DFC body with a
 * cached footprint take its fast path (static data in registers and shared memory, the
 * gathered state in shared memory); 0 sends every body through the general path.  Both
 * compute the same values in the same order, so the results are bitwise equal; tests
 * check that.  Process-wide.  Syncs the device.  Errors: CUDA. */
int iblbm_test_set_ib_fast(int enable);
int iblbm_kernel_variant(int storage, int collision, int* variant, double* ms);

/* ---- serving loop ---------------------------------------------------------------------- */
/* Continuous batching of simulation requests (no counterpart in the paper; it
 * serves the method of Sec. 2 to many callers).  A request is a lattice with
 * at most one body run for nsteps steps; its result is the body's force
 * history.  Requests are admitted in arrival order while a slot is free and
 * the estimated device bytes fit the budget; admitted cases stay resident and
 * every tick advances all of them with one batched launch sequence per step,
 * so a case's result is identical to running it alone.  Not thread-safe. */
typedef struct iblbm_server iblbm_server;
/* hbm_budget: device bytes the resident cases may hold; max_slots: resident
 * cases at most; stream: cudaStream_t the cases order their work after. */
int iblbm_server_create(size_t hbm_budget, int max_slots, void* stream, iblbm_server** out);
void iblbm_server_destroy(iblbm_server* srv);
/* Queues a request (copies every input).  body/xy may be NULL when n = 0.
 * *req_id receives its id.  Errors: INVALID_ARG. */
int iblbm_server_submit(iblbm_server* srv, const iblbm_lattice_desc* desc, int collision, double tau,
                        const iblbm_body_desc* body, const double* xy, int n, double ds, int kernel,
                        int scheme, int nsteps, long long* req_id);
/* One tick: advances every resident case by min(max_steps, fewest steps left)
 * steps, admits queued requests while the device works, retires finished
 * cases (their memory is freed at once).  Returns the number of requests
 * completed in this tick (>= 0) or an error; *resident / *queued receive the
 * counts after the tick (either may be NULL). */
int iblbm_server_tick(iblbm_server* srv, int max_steps, int* resident, int* queued);
/* Result of a request: 1 when done (force history into forces_out[3*cap],
 * *n entries, *latency_s seconds from submission to completion), 0 while
 * pending, IBLBM_ERR_NOT_ADMITTED if it can never fit the budget, another
 * negative code if its case failed, IBLBM_ERR_NOT_FOUND for an unknown id. */
int iblbm_server_poll(iblbm_server* srv, long long req_id, double* forces_out, int cap, int* n,
                      double* latency_s);
/* Device bytes held by resident cases and the resident / queued counts. */
int iblbm_server_stats(const iblbm_server* srv, size_t* used_bytes, int* resident, int* queued);
/* Whether ticks replay the batch's captured CUDA graphs (1, the default: a new set
 * of resident requests captures its graphs on its first tick) or launch each step's
 * kernels one by one (0).  Results are the same either way.  Errors: INVALID_ARG. */
int iblbm_server_set_graphs(iblbm_server* srv, int enable);

/* ---- allocation-free lambda_k ------------------------------------------------------------ */
/* No counterpart in the paper.  For callers that cannot allocate device memory
 * where they need the DFC factors lambda_k of Eq. 17 (host code inside a
 * framework that owns every device allocation, a solver embedded in another
 * application's time loop where an allocation would synchronise the device or
 * could fail mid-run, real-time loops where an allocation could block), this
 * call computes lambda_k for one marker set without allocating:
 * no cudaMalloc, cudaFree or allocating library routine.  Its scratch (W_total
 * on the markers' bounding box) is a library-wide device array of 2^18 FP64
 * values, so the box -- (max - min stencil origin + S) in x times the same in y,
 * S = 2 (hat) or 4 (Peskin) -- may hold at most 262144 nodes (512 x 512).
 *   xy      device pointer, 2*n doubles (x0, y0, x1, y1, ...), lattice units
 *   n, ds   marker count and arc length (Eq. 17 uses ds; rho_f = 1)
 *   kernel  IBLBM_HAT or IBLBM_PESKIN4
 *   nx, ny  lattice size; every footprint must lie inside it
 *   lambda  device pointer, n doubles, written with lambda_k
 *   stream  cudaStream_t the work is ordered on (NULL = legacy default); the
 *           call syncs that stream to report errors.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture begins.
 * The array is shared by all calls and keeps the last call's contents; calls
 * that overlap on the GPU race and must be serialised by the caller.
 * Errors: INVALID_ARG, CAPACITY (box above 262144 nodes),
 * MARKER_OUT_OF_DOMAIN, CUDA. */
int iblbm_dfc_lambda_noalloc(const double* xy, int n, double ds, int kernel, int nx, int ny, double* lambda,
                             void* stream);

/* ---- timing of the stream-collide kernel ------------------------------------------ */
/* While enabled, steps launch their kernels one by one (no graph) and bracket
 * each stream-collide launch (one per collision operator and storage type in
 * the batch) and each lattice-edge launch (one per storage type) with CUDA
 * events on the launching stream; together they are the whole lattice sweep.
 * iblbm_kernel_timing returns the summed event time (ms) and the launch count
 * since the last reset, then resets.  Syncs. */
int iblbm_set_timing(iblbm_ctx* ctx, int enable);
int iblbm_kernel_timing(iblbm_ctx* ctx, double* stream_collide_ms, int* launches);
/* The same timed steps broken down by stage: ms[0] / launches[0] the IB stage (body
 * motion, interface coupling and body update: one launch per storage type with
 * bodies), [1] the stream-collide launches, [2] the lattice-edge launches, [3] the
 * step-counter launch; sums since the last reset, then resets (this call and
 * iblbm_set_timing reset; iblbm_kernel_timing resets only its own sums).  Either
 * pointer may be NULL.  Syncs.  Errors: INVALID_ARG. */
int iblbm_stage_timing(iblbm_ctx* ctx, double ms[4], int launches[4]);

#ifdef __cplusplus
}
#endif
#endif
