/*
 * ibl.h - C ABI of the GB300-native immersed-boundary lattice Boltzmann library.
 *
 * The library implements the per-time-step hot path of the implicit
 * velocity-correction IB-LBM of Kumar, De and Das, "Investigation of flow
 * field of clap & fling motion using immersed boundary coupled lattice
 * Boltzmann method" (arXiv 2102.01305):
 *
 *   - BGK collision (Eq. 1) with the Guo forcing term (Eqs. 7-8), fused with
 *     streaming and moment recovery (Eqs. 2, 9, 11), on D2Q9 (Sec. 2.1,
 *     weights Eq. 5) or D3Q19;
 *   - the implicit immersed-boundary exchange with Lagrangian markers
 *     (Sec. 2.2): 4-point cosine delta (Eqs. 13-14), interpolation (Eq. 17),
 *     the per-step system A X = B for the marker velocity corrections
 *     (Eqs. 18-19), spreading (Eq. 15), velocity correction (Eq. 16) and
 *     force density F = 2 rho du / dt (Eq. 26);
 *   - prescribed rigid kinematics of the wings (Eqs. 20-23, Sec. 3.3);
 *   - the body-force, lift/thrust/drag reduction (Sec. 3.7).
 *
 * Conventions shared by every call
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3.  Grid nodes sit at integer
 *     coordinates 0..n-1 on each axis; cell index (z*ny + y)*nx + x.
 *   - All pointer arguments are HOST pointers unless a call says otherwise.
 *     Inputs are copied before the call returns; the caller keeps ownership.
 *     Outputs go to caller-allocated buffers of the stated size.
 *   - Every call returns an ibl_status and never aborts the process.  On
 *     error the context keeps its previous state and ibl_last_error() gives
 *     a one-line reason.  A context is not thread-safe; distinct contexts are
 *     independent.  All device memory is owned by the context and released
 *     by ibl_destroy.
 *   - ibl_step is asynchronous with respect to the host: it enqueues work on
 *     the context's CUDA stream and returns.  Calls that return data
 *     (ibl_forces, ibl_get_*, ibl_mass) synchronise that stream first and
 *     then report any error the enqueued steps raised (divergence, solver
 *     non-convergence, a device wait that timed out).
 */
#ifndef IBL_H
#define IBL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibl_ctx ibl_ctx;   /* opaque */

typedef enum {
  IBL_OK = 0,
  IBL_EINVAL = 1,      /* invalid argument or configuration */
  IBL_ENOMEM = 2,      /* device allocation failed */
  IBL_ECUDA = 3,       /* CUDA runtime error (message in ibl_last_error) */
  IBL_EDIVERGED = 4,   /* NaN/Inf or runaway density detected; sticky until destroy */
  IBL_ENOTCONV = 5,    /* the implicit IB solve did not reach its tolerance */
  IBL_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  IBL_ESTATE = 7,      /* call out of order (e.g. step before the fluid is initialised) */
  IBL_ECANCELED = 8,   /* a serving run was cancelled (ibl_server_cancel) */
  IBL_EUNSTABLE = 9    /* a serving request lies outside the collision's stability range */
} ibl_status;

/* Lattice: D2Q9 (Sec. 2.1, Eq. 5) or D3Q19 (textbook weights 1/3, 1/18, 1/36). */
typedef enum { IBL_D2Q9 = 9, IBL_D3Q19 = 19 } ibl_lattice;

/* Face conditions (Sec. 2.1 bounce-back walls; Sec. 3.1 Zou-He inlet / outlet). */
typedef enum {
  IBL_PERIODIC = 0,     /* must be set on both faces of an axis */
  IBL_BOUNCEBACK = 1,   /* halfway bounce-back wall, at rest */
  IBL_VEL_INLET = 2,    /* Zou-He, velocity u_in prescribed */
  IBL_PRESS_OUTLET = 3  /* Zou-He, density rho_out prescribed, zero tangential velocity */
} ibl_bc;

/* Storage precision of the distributions.  FP64 computes in FP64; FP32
 * stores f_i - w_i in FP32 and collides in FP32.  FP16DEV / BF16DEV store
 * f_i - w_i in 16 bits and collide in FP32. */
typedef enum { IBL_FP64 = 0, IBL_FP32 = 1, IBL_FP16DEV = 2, IBL_BF16DEV = 3 } ibl_precision;

typedef struct {
  int32_t nx, ny, nz;        /* nz = 1 for D2Q9 */
  int32_t bc[6];             /* ibl_bc per face: -x, +x, -y, +y, -z, +z */
  double u_in[3];            /* inlet velocity (IBL_VEL_INLET faces) */
  double rho_out;            /* outlet density (IBL_PRESS_OUTLET faces) */
  double body_force[3];      /* uniform body force G added to F everywhere */
  int32_t precision;         /* ibl_precision */
} ibl_grid;

/* Prescribed wave form of a body's translation A(t) or rotation alpha(t).
 * theta(t) = 2 pi f t + phi with f and phi given to ibl_set_kinematics:
 *   IBL_WAVE_CONST    offset
 *   IBL_WAVE_COS      offset + amp cos(theta)       Eq. 20 (amp = A0/2)
 *   IBL_WAVE_SIN      offset + amp sin(theta)       Eq. 21, Eq. 23
 *   IBL_WAVE_ABS_SIN  offset + amp |sin(theta)|     opening 0..amp (clap-and-fling reading)
 *   IBL_WAVE_TABLE    table[n mod n_table] at step n; rate by central difference */
typedef enum {
  IBL_WAVE_CONST = 0, IBL_WAVE_COS = 1, IBL_WAVE_SIN = 2, IBL_WAVE_ABS_SIN = 3, IBL_WAVE_TABLE = 4
} ibl_wave_kind;

typedef struct {
  int32_t kind;            /* ibl_wave_kind */
  double amp, offset;
  const double* table;     /* IBL_WAVE_TABLE only: n_table samples, copied */
  int64_t n_table;
} ibl_wave;

/* Field selectors for ibl_get_field. */
typedef enum {
  IBL_FIELD_RHO = 0,   /* rho = sum_i f_i, N values */
  IBL_FIELD_U = 1,     /* u = (sum_i c_i f_i + G/2)/rho, d x N values (component-major) */
  IBL_FIELD_FORCE = 2  /* last step's IB force density 2 rho du (Eq. 26, without G), d x N */
} ibl_field;

/* ------------------------------------------------------------------ lifecycle */

/* Create a context on the current CUDA device.  tau > 1/2 is the BGK
 * relaxation time (Eq. 3: tau = 3 nu + 1/2).  Allocates both population
 * buffers; the fluid starts uninitialised (see ibl_init_fluid).
 * Errors: IBL_EINVAL (sizes <= 0, nz != 1 for D2Q9, unpaired periodic faces,
 * a Zou-He face whose lateral axes are not periodic, tau <= 1/2, unknown
 * precision), IBL_ENOMEM, IBL_ECUDA. */
ibl_status ibl_create(const ibl_grid* grid, double tau, int32_t lattice, ibl_ctx** out);

/* Release all device memory and the stream.  NULL is accepted. */
ibl_status ibl_destroy(ibl_ctx* ctx);

/* Set f_i = f_eq(rho, u) (Eq. 4) everywhere and reset the step counter.
 * rho: N host doubles or NULL (rho = 1); u: d x N host doubles
 * (component-major) or NULL (u = 0). */
ibl_status ibl_init_fluid(ibl_ctx* ctx, const double* rho, const double* u);

/* Set the populations directly: f is Q x N host doubles, direction-major in
 * the order of ibl_lattice_velocities.  Resets the step counter. */
ibl_status ibl_set_populations(ibl_ctx* ctx, const double* f);

/* ------------------------------------------------------------------ bodies */

/* Add a rigid body of m Lagrangian markers (Sec. 2.2, Fig. 1).
 * X0: m x d body-frame coordinates (marker-major); ds: m element sizes
 * (arc length in 2D, area in 3D, the ds_l of Eq. 15); hinge: rotation centre
 * in the body frame; axis: rotation axis (normalised internally; in 2D use
 * +/- z); origin: world position of the body-frame origin.  The world
 * position is X = origin + hinge + R(axis, alpha)(X0 - hinge) + A e_s.
 * Until ibl_set_kinematics is called the body is at rest (A = alpha = 0).
 * *body_id receives 0, 1, ... in order of creation.
 * Errors: IBL_EINVAL (m <= 0, ds <= 0, zero axis), IBL_ENOMEM. */
ibl_status ibl_set_markers(ibl_ctx* ctx, int32_t m, const double* X0, const double* ds,
                           const double hinge[3], const double axis[3],
                           const double origin[3], int32_t* body_id);

/* Prescribe a body's motion (Eqs. 20-23, Sec. 3.3): translation A(t) along
 * the stroke direction e_s = (cos beta, sin beta, 0) and rotation alpha(t)
 * about the hinge axis; phi is the body's phase and f its frequency in
 * cycles per step.  The wall velocity U_B = A' e_s + alpha' axis x r
 * includes the rotational velocity (Sec. 3.3).  J is the advance ratio
 * J = U_inf / U_tip (Eq. 24); it is recorded for reporting only, the
 * free stream itself is the grid's inlet velocity. */
ibl_status ibl_set_kinematics(ibl_ctx* ctx, int32_t body_id, const ibl_wave* A,
                              const ibl_wave* alpha, double beta, double phi, double f,
                              double J);

/* Override the kinematics for the NEXT step only: X and U are m x d host
 * doubles (marker-major), positions and wall velocities at that step. */
ibl_status ibl_set_marker_state(ibl_ctx* ctx, int32_t body_id, const double* X,
                                const double* U);

/* Lift direction of a body (unit vector, default +y); drag is along +x. */
ibl_status ibl_set_lift_axis(ibl_ctx* ctx, int32_t body_id, const double e[3]);

/* Reference values of the coefficients C = F / (rho_ref U_ref^2 L / 2):
 * L is a length in 2D and an area in 3D (Sec. 3.6 uses rho C S U_tip^2 / 2). */
ibl_status ibl_set_reference(ibl_ctx* ctx, double U_ref, double L_or_S, double rho_ref);

/* ------------------------------------------------------------------ stepping */

/* Advance n >= 0 time steps, each the whole hot path in the paper's order
 * (Sec. 2.2): kinematics -> moments -> interpolation (Eq. 17) -> implicit
 * solve (Eqs. 18-19) -> spreading and force density (Eqs. 15, 16, 26) ->
 * collision with forcing (Eqs. 7-8) and streaming with the face conditions
 * -> body-force reduction (Sec. 3.7).  Asynchronous; returns the first
 * sticky error already known (e.g. IBL_EDIVERGED) or IBL_OK. */
ibl_status ibl_step(ibl_ctx* ctx, int64_t n);

/* Block until the enqueued steps finish; returns their first error. */
ibl_status ibl_sync(ibl_ctx* ctx);

/* Coefficients of the last completed step for one body (Sec. 3.7):
 * C_D along +x, C_T = -C_D, C_L along the body's lift axis. */
ibl_status ibl_forces(ibl_ctx* ctx, int32_t body_id, double* C_L, double* C_T, double* C_D);

/* Up to max most recent (C_L, C_T, C_D) triples of a body, oldest first, into
 * out3 (3*max doubles); *n receives how many were written.  The device keeps
 * the last 65536 steps. */
ibl_status ibl_force_history(ibl_ctx* ctx, int32_t body_id, int64_t max, double* out3,
                             int64_t* n);

/* Copy a macroscopic field of the current populations to the host
 * (sizes in ibl_field). */
ibl_status ibl_get_field(ibl_ctx* ctx, int32_t what, double* out);

/* Copy the current (post-streaming) populations, Q x N doubles. */
ibl_status ibl_get_populations(ibl_ctx* ctx, double* f);

/* Marker state of the last completed step: X, U_B (wall velocity) and the
 * force each marker exerts on the fluid, 2 rho_l du_B^l ds_l; each m x d,
 * any pointer may be NULL. */
ibl_status ibl_get_markers(ibl_ctx* ctx, int32_t body_id, double* X, double* U, double* F);

/* Total mass sum_x rho(x) of the current populations, accumulated in FP64
 * in a fixed order. */
ibl_status ibl_mass(ibl_ctx* ctx, double* mass);

/* Periodic FP64 mass check (failure detection).  Every `every` steps
 * (default 500; 0 = off) ibl_step sums rho over all cells in FP64, in a fixed
 * order, into buffers the context owns, and compares the total with the
 * total taken when the fluid was initialised (ibl_init_fluid,
 * ibl_set_populations).  A non-finite total or - when no face is a Zou-He
 * inlet or outlet, so that the faces conserve mass - a relative change above
 * rel_tol (0 = default: 1e-9 for FP64 storage, 1e-4 FP32, 1e-2 FP16/BF16)
 * sets the sticky divergence status: the next synchronising call and every
 * later ibl_step return IBL_EDIVERGED.  The collision kernels flag a cell
 * whose density is non-finite or outside (0, 100) on every step as well. */
ibl_status ibl_set_mass_check(ibl_ctx* ctx, int32_t every, double rel_tol);

/* The mass check's reference total, its last checked total and the number
 * of checks so far.  Synchronises; a divergence already flagged is returned
 * as IBL_EDIVERGED after the values are written. */
ibl_status ibl_mass_check_read(ibl_ctx* ctx, double* m0, double* m_last, int64_t* checks);

/* Same total as ibl_mass, for callers that must not allocate device memory
 * after start-up: a solver embedded in a real-time control loop, where a
 * cudaMalloc can block for an unbounded time, or code whose device memory is
 * fully claimed by another allocator (a framework's caching allocator), where
 * a cudaMalloc fails.  ibl_mass allocates its partial sums per call; this call
 * allocates nothing: its partials live in a static device array of 4096
 * doubles (32 KB), which every GPU that loads the library holds until the
 * process exits.  The paper has no counterpart of this call.
 *   nparts  number of fixed chunks summed on the device, 1..4096 (IBL_EINVAL
 *           beyond); with nparts = 1024 the result equals ibl_mass bitwise.
 * The first call on a device looks up the array's device address (with that
 * device current), so make it before any stream capture.  All calls share
 * the array: calls from different contexts or threads that overlap on the
 * GPU race and must be serialised by the caller.  Synchronises the stream. */
ibl_status ibl_mass_noalloc(ibl_ctx* ctx, int32_t nparts, double* mass);

/* ------------------------------------------------------------------ point operators */

/* The two transfers of the IB step on an arbitrary cloud of m points, without
 * the implicit solve (for throughput sweeps and for callers that run their
 * own marker update).  All arrays are DEVICE pointers (e.g. tensor storage).
 * ibl_interpolate_points: U (m x d, point-major) and, if non-NULL, rho (m) =
 *   sum_x u*(x) D(x - X_l), sum_x rho(x) D(x - X_l) of the current
 *   populations (Eq. 17 with the velocity of Eq. 11 including G/2).
 * ibl_spread_points: out (d x N, component-major, overwritten) =
 *   sum_l V_l ds_l D(x - X_l) (Eq. 15).  The sums are accumulated in 64-bit
 *   fixed point (2^-46) inside `out` itself, so they do not depend on the
 *   order of the atomic additions; |V ds| must stay below 1.3e5.
 * X is m x 3 (point-major; z ignored in 2D).  Both synchronise the stream.
 * IBL_EINVAL if a stencil leaves a non-periodic axis. */
ibl_status ibl_interpolate_points(ibl_ctx* ctx, int32_t m, const double* d_X, double* d_U, double* d_rho);
ibl_status ibl_spread_points(ibl_ctx* ctx, int32_t m, const double* d_X, const double* d_V,
                             const double* d_ds, double* d_out);

/* ------------------------------------------------------------------ introspection */

/* Velocity set of a lattice: c is Q x 3 int32 (marker of direction order used by
 * every population array of this ABI), w is Q doubles; either may be NULL.
 * Returns Q in *q. */
ibl_status ibl_lattice_velocities(int32_t lattice, int32_t* q, int32_t* c, double* w);

/* Solver statistics of the last completed step: PCG iterations and the final
 * relative residual of the implicit IB system; number of preconditioner
 * rebuilds so far (scheduled ones plus early ones after a slow solve). */
ibl_status ibl_solver_stats(ibl_ctx* ctx, int32_t* iterations, double* rel_residual,
                            int64_t* refreshes);

/* Settings of the implicit IB solve (preconditioned conjugate gradients on
 * the system of Eqs. 18-19): the dense FP32 approximate inverse used as
 * preconditioner is rebuilt every refresh_every steps (default 384).  It is
 * also rebuilt early after a solve that did not converge, or once the
 * iterations spent beyond 40 and beyond the first solve after the last
 * rebuild, summed over the solves since, pass the rebuild's cost in
 * iterations (sum 2 m_b^3 / sum 6 m_b^2, at least 64).  tol is the relative
 * residual in the preconditioner's norm (0 = default: 1e-10 for FP64
 * storage, 1e-6 for FP32, FP16 and BF16).  extrapolate chooses each
 * solve's initial guess: 2 (or more) 3 w_{n-1} - 3 w_{n-2} + w_{n-3},
 * 1 (default) 2 w_{n-1} - w_{n-2}, 0 w_{n-1}, < 0 zero.  Changing these changes the iterates, not the system being
 * solved. */
ibl_status ibl_solver_config(ibl_ctx* ctx, int32_t refresh_every, double tol, int32_t extrapolate);

/* Thread blocks (one per SM, 1024 threads) of the cooperative implicit
 * solve; 0 (default) = half the SMs (all of them above 8192 markers unless
 * the split is forced), larger values are capped at the SM count.  The block count fixes the solve's reduction order: runs with the
 * same count are bitwise reproducible. */
ibl_status ibl_solver_blocks(ibl_ctx* ctx, int32_t blocks);

/* Preconditioner of the implicit IB solve (Eqs. 18-19).  Both kinds
 * approximate (G_b + sigma I)^-1 per body, sigma = 1e-6 (kind 0) or 2e-7
 * (kind 1) times G_b's largest absolute row sum, rebuilt every
 * refresh_every steps (ibl_solver_config):
 *   kind 0: the dense inverse, FP32, m_b^2 numbers per body;
 *   kind 1: separable factors, for bodies whose markers form a chord x span
 *           product mesh (a planform grid, possibly clipped) turning about
 *           the z axis: G_b is then a principal submatrix of a Kronecker
 *           product C (x) Z, and its shifted inverse follows from the
 *           factors' inverses and one Schur block over the mesh's bounding
 *           rectangle (n_k^2 + n_k n_i^2 + n_c^2 numbers; 3D only);
 *   kind -1 (default): kind 1 when every body qualifies and the largest has
 *           at least 4096 markers, else kind 0.
 * A change of kind takes effect at the next step and restarts the solver's
 * warm start.  IBL_EINVAL at the next step if kind 1 is asked for bodies
 * that do not qualify.
 * resident_rows (kind 0): -1 (default) each solve block keeps its
 * preconditioner rows in shared memory when they fit; 0 the rows are always
 * read from L2/HBM (the path every solve takes when they do not fit).  Both
 * paths multiply the same FP32 rows in the same order, so they give bitwise
 * the same results.  IBL_EINVAL for other values. */
ibl_status ibl_solver_preconditioner(ibl_ctx* ctx, int32_t kind, int32_t resident_rows);

/* How a step with markers schedules its collision: 0 = one kernel over all
 * cells after the IB chain; 1 = split: the cells outside the IB band collide
 * on a second stream while the IB chain (interpolation, solve, spreading)
 * runs, and the band tiles collide after the spreading; 2 = serial split:
 * after the IB chain, the cells outside the band collide in a kernel without
 * the band lookup on every SM, then the band tiles; -1 (default) = split on
 * grids of at least 2^20 cells with at most 8192 markers, else 0.  All give
 * bitwise the same populations and forces (every cell runs the same
 * arithmetic). */
ibl_status ibl_set_overlap(ibl_ctx* ctx, int32_t mode);

/* Launch shape of the one-kernel collide (the kernel of steps without the
 * split, see ibl_set_overlap): thread blocks of bx x by threads, bx in
 * {32, 64, 128, 256}, bx * by <= 256 (default 64 x 2).  With 16-bit storage
 * and nx even, each thread takes the two x-adjacent cells (x, x + 1), whose
 * collisions run as packed FP32 pairs: pairs = 3 (default) walks 8 z-planes
 * per thread, the next plane's loads in flight while the current one
 * collides; pairs = 1 one plane per thread; pairs = 2 blocks of 64 x 4
 * threads walk 16 z-planes of 128 x 4 cells, the next plane's source rows
 * arriving in shared memory by bulk asynchronous copies (D3Q19 with nx a
 * multiple of 8; otherwise as 1); pairs = 0 one cell per thread.  Every
 * cell runs the same rounded operations whatever the shape, so all shapes
 * give bitwise the same populations (a tuning knob, not a numerical one).
 * IBL_EINVAL for other values. */
ibl_status ibl_set_collide_shape(ibl_ctx* ctx, int32_t bx, int32_t by, int32_t pairs);

/* Phase timestamps (GPU global timer, ns, taken by block 0) of the last
 * implicit solve: [0] start, [1] after the optional preconditioner rebuild,
 * [2] after set-up, [3] end; [4]-[7] the four phases of the rebuild's first
 * pivot block (pivot inverse, row panel, trailing update, column panel);
 * iteration k (k < 26) at 8 + 9k: recurrence
 * scalars ready, search direction input staged, SpMV rows done, block
 * reduction done, grid barrier passed, step length ready, preconditioner
 * input staged, preconditioner rows done, grid barrier passed.  With the
 * separable preconditioner, [4]-[7] and [251]-[252] mark the ends of stages
 * A-F of the set-up's first application (from [250]) and [253] the end of
 * its stage G.  Unused slots are 0.  Copies min(max, 256) values into ns. */
ibl_status ibl_solver_trace(ibl_ctx* ctx, int64_t* ns, int32_t max, int32_t* n);

/* Enable (1 or 2) or disable (0) CUDA-event timing of the collide-stream
 * kernel(s) and of the IB chain (kinematics .. spreading and the force
 * reduction) of every step enqueued while enabled.  In a split step (see
 * ibl_set_overlap) the bulk collide is timed on its own stream, concurrently
 * with the IB chain.  Enabling resets the totals.  Adds events only; the
 * launch sequence is unchanged. */
ibl_status ibl_profile(ibl_ctx* ctx, int32_t enable);

/* With ibl_profile(ctx, 2): milliseconds per phase of the step on the
 * context's main stream since profiling was enabled, ms[0..n): 0 kinematics,
 * 1 band counters reset, 2 tile marking, 3 slot assignment (which also
 * resets the previous band), 4 marker lists,
 * 5 interpolation and system assembly (one kernel; 6 is kept for the
 * assembly and reads 0), 7 implicit solve and spreading (one kernel; 8 is
 * kept for the spreading and reads 0),
 * 9 collision (the band tiles' kernel in a split step; the bulk collide on
 * the second stream is in ibl_profile_read).  Each phase is the time from
 * the end of the previous one, so launch gaps are included.  Synchronises. */
ibl_status ibl_profile_phases(ibl_ctx* ctx, double* ms, int32_t n);

/* Totals since the last ibl_profile(ctx, 1): milliseconds in the
 * collide-stream kernel(s), milliseconds in the IB chain, steps timed.
 * Synchronises the stream. */
ibl_status ibl_profile_read(ibl_ctx* ctx, double* collide_ms, double* ib_ms, int64_t* steps);

/* Number of kernel launches the context has enqueued since creation. */
ibl_status ibl_launch_count(const ibl_ctx* ctx, int64_t* n);

/* The CUDA stream the context enqueues on (a cudaStream_t, as void*). */
ibl_status ibl_stream(const ibl_ctx* ctx, void** stream);

/* One-line description of the context's last error ("" if none).  With
 * ctx == NULL, the last error of a failed ibl_create. */
const char* ibl_last_error(const ibl_ctx* ctx);

/* ------------------------------------------------------------------ serving */

/* Serving form of the paper's parametric study (Sec. 3.3-3.7: clap-and-fling
 * runs over Re, f and J): requests arrive while others run, are admitted by
 * an HBM budget, and advance concurrently, each on its own stream, in
 * chunks of steps.  A run follows exactly the kernel sequence it would
 * follow alone, so its result does not depend on the mix. */
typedef struct ibl_server ibl_server;

typedef struct {
  int64_t hbm_budget_bytes;  /* device memory the active runs may use together */
  int32_t max_active;        /* runs advanced concurrently */
  int32_t chunk_steps;       /* steps enqueued per run between scheduling passes */
  int32_t tune;              /* 1: per-request launch tuning (see below); 0: library defaults */
} ibl_server_config;

/* One clap-and-fling run: D3Q19 box nx x ny x nz, two flat elliptic wings of
 * chord `chord` (span 5 chord, unit-spaced markers) hinged at the trailing
 * edge c/2 apart, opening angle (pi/3)|sin(2 pi t / period)| per wing;
 * Re = U_tip c / nu with U_tip = 2 Phi c / period, Phi = 120 degrees (Eq. 24,
 * Sec. 3.4), tau = 3 nu + 1/2 (Eq. 3); free stream J * U_tip along +x,
 * imposed by Zou-He inlet/outlet faces (faces = 1) or as the initial flow of
 * an x-periodic box (faces = 0). */
typedef struct {
  int32_t nx, ny, nz;
  double chord;
  double Re;
  double period;        /* steps per flapping period, T = 1/f */
  double J;
  int32_t precision;    /* ibl_precision */
  int32_t faces;
  int64_t steps;        /* 1 .. 65536 */
} ibl_run_request;

typedef struct {
  int32_t status;       /* ibl_status of the run */
  int32_t done;         /* 1 once finished (or failed) */
  int64_t steps_done;   /* steps enqueued so far */
  double submit_s, start_s, finish_s;   /* server clock, seconds since creation */
  double CL_max[2], CL_mean[2], CT_max[2], CT_mean[2];   /* per wing over the run */
  double CL_last[2], CT_last[2];
  /* launch configuration the run used (tune = 1): solve blocks, overlap
   * mode and collide shape after its tuning chunk (0 where not set) */
  int32_t solve_blocks, overlap, collide_bx, collide_by, collide_pairs, tuned;
} ibl_run_result;

/* Per-request tuning (tune = 1).  The solve's block count changes its
 * reduction order, so it is a function of the request alone: one block per
 * 64 markers, between 4 and half the SMs (small runs then leave SMs to the
 * others' kernels).  The overlap mode and the collide shape give bitwise the
 * same results whatever their values (ibl_set_overlap,
 * ibl_set_collide_shape), so they are measured: the first chunk of a run
 * whose shape (grid, chord, precision, faces) has not been seen is split
 * between the candidates (split step; one kernel with 64 x 2, 128 x 1 or
 * 64 x 4 blocks; staged 16-bit planes), each timed with CUDA events on the run's
 * stream, and the fastest is kept for that run and every later run of the
 * same shape.  A run's numbers therefore depend on its request only, alone
 * or in any mix. */
/* Create a server on the current device (starts its scheduling thread). */
ibl_status ibl_server_create(const ibl_server_config* cfg, ibl_server** out);
/* Queue a run; *run_id identifies it.  IBL_EINVAL for a malformed request or
 * wings that do not fit the box, IBL_ENOMEM if its footprint exceeds the
 * whole budget, IBL_EUNSTABLE if it lies outside the BGK collision's
 * stability range (tau = 3 nu + 1/2 below 0.505, a free stream J U_tip above
 * 0.05, a tip speed above 0.15 lattice units, or a tip speed above 0.05 with
 * U_tip / nu above 5), instead of diverging on the GPU.  The submission time is taken on entry.  Thread-safe. */
ibl_status ibl_server_submit(ibl_server* s, const ibl_run_request* req, int64_t* run_id);
/* Cancel a run: a queued run never starts; a running one stops after the
 * chunk of steps in flight and its memory returns to the budget.  Its result
 * then reports IBL_ECANCELED with the steps done.  No effect on a finished
 * run; IBL_EINVAL for an unknown id.  Thread-safe. */
ibl_status ibl_server_cancel(ibl_server* s, int64_t run_id);
/* Snapshot of a run's progress and, once done, its result.  Thread-safe. */
ibl_status ibl_server_poll(ibl_server* s, int64_t run_id, ibl_run_result* out);
/* Block until no run is queued or active; IBL_ETIMEOUT after timeout_s. */
ibl_status ibl_server_wait_all(ibl_server* s, double timeout_s);
ibl_status ibl_server_stats(ibl_server* s, int32_t* queued, int32_t* active, int32_t* finished,
                            int64_t* hbm_in_use);
/* Where the scheduling thread's time went since the server was created:
 * wall_s in total, busy_s in scheduling passes that did work (the rest it
 * slept), and of busy_s: enqueue_s enqueueing steps (ibl_step), build_s
 * creating run contexts, retire_s reading results and destroying contexts.
 * busy_s close to wall_s with the GPU not saturated means the host thread
 * bounds the throughput.  Any pointer may be NULL. */
ibl_status ibl_server_load(ibl_server* s, double* wall_s, double* busy_s, double* enqueue_s, double* build_s,
                           double* retire_s);
/* Stop the scheduler and release every run. */
ibl_status ibl_server_destroy(ibl_server* s);

#ifdef __cplusplus
}
#endif

#endif /* IBL_H */
