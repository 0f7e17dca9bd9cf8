/*
 * sdg.h -- C ABI of the GB300 library for the matrix-free pressure / viscous
 * solves and the time step of the spectral semi-implicit staggered DG scheme
 * for the incompressible Navier-Stokes equations (Fambri & Dumbser, Sec. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Periodic box [0,L_x] x [0,L_y] (x [0,L_z]) split into n[d] cells per
 *    direction; degree N (0 <= N <= 11), n1 = N + 1 Gauss-Legendre nodes per
 *    direction on every main and dual cell (Sec. 2.1).
 *  - A field is an array of ncell * n1^dim doubles (or floats where stated),
 *    element-major with the x node fastest:
 *        idx = (((k*ny + j)*nx + i) * n1^dim) + (l3*n1 + l2)*n1 + l1 .
 *    Velocity component d is stored on its own dual grid: the block at
 *    element (i,j,k) is the dual cell shifted by +1/2 along d (Sec. 2.1,
 *    T_{i+1/2,j,k}, T_{i,j+1/2,k}, T_{i,j,k+1/2}).
 *  - Pointers marked "device" are device pointers owned by the caller; the
 *    library never frees them.  Pointers marked "host or device" may be
 *    either (the copy uses unified addressing).  The handle owns all of its
 *    internal buffers and frees them in sdg_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it.  Calls that run an iterative solve synchronise the
 *    stream while they iterate (convergence is tested on the device and the
 *    flag is read back), so they return with the result complete.
 *  - Every entry point returns an sdg_status; on error nothing is guaranteed
 *    about the outputs.  sdg_strerror gives a message; sdg_last_error gives
 *    the text of the last failure in this thread.
 */
#ifndef SDG_H
#define SDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SDG_OK = 0,
  SDG_ERR_INVALID_ARG = 1,   /* bad size, degree, parameter or NULL pointer */
  SDG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  SDG_ERR_NOT_CONVERGED = 3, /* CG hit maxit or its true residual stopped improving
                                above the tolerance; x holds the last iterate */
  SDG_ERR_BREAKDOWN = 4,     /* p^T A p <= 0 or not finite */
  SDG_ERR_UNSUPPORTED = 5    /* a configuration this build does not handle */
} sdg_status;

typedef enum { SDG_FP64 = 0, SDG_MIXED = 1 } sdg_precision;

typedef struct {
  int dim;       /* 2 or 3 */
  int n[3];      /* cells per direction; n[2] ignored in 2D; each >= 1 */
  double L[3];   /* box lengths (> 0); L[2] ignored in 2D */
} sdg_grid;

typedef struct {
  int iters;          /* CG iterations (mixed: FP32 iterations; FP64
                         iterations of a finishing phase count in
                         applies_fp64) */
  int outer_iters;    /* mixed: FP64 residual replacements (0 in FP64) */
  int applies_fp64;   /* operator applications in FP64 */
  int applies_fp32;   /* operator applications in FP32 */
  double rel_res;     /* ||r|| / ||b||: recursive residual (FP64 mode) or
                         true FP64 residual (mixed mode) at exit */
  int status;         /* sdg_status of this solve */
  double true_res;    /* ||b - A x|| / ||b|| of the returned x, recomputed in
                         FP64 with the accurate operator (both modes; for the
                         singular pressure system the constant part of the
                         residual, round-off of a zero-mean b, is removed) */
  double floor_res;   /* estimate of the smallest true_res any FP64 vector
                         near x can have: ||A u|| / ||b|| for a perturbation
                         u of random sign and size ulp(x_i) / (2 sqrt 3) per
                         entry, the spread of rounding x to FP64 (0 when not
                         computed: FP64 mode without info, mixed mode that
                         met the tolerance) */
  double eval_res;    /* ||A x - A~ x|| / ||b||: two FP64 evaluations of the
                         operator at the returned x (accurate and direct
                         contraction), the size of the rounding of A x itself;
                         computed only when a solve stops improving (else 0) */
} sdg_cg_info;

typedef struct {
  sdg_cg_info pressure;    /* the pressure solve of the last step */
  sdg_cg_info viscous[3];  /* the viscous solves of the last step */
  double pressure_ms;      /* device time of the pressure solves, summed over
                              the nsteps of the call (CUDA events) */
  double step_ms;          /* device time of the whole call (CUDA events) */
  long long pressure_applies; /* operator applications in the pressure solves,
                                 summed over the nsteps of the call */
  long long kernel_launches;  /* CUDA kernels the call launched */
} sdg_step_info;

typedef struct sdg_handle sdg_handle;

/* ---------------------------------------------------------------- set-up */

/* Gauss-Legendre nodes xi[0..N] and weights w[0..N] on [0,1] (Sec. 2.1;
 * the nodal basis is the Lagrange interpolant through these points).
 * xi, w: host arrays of N+1 doubles.  Errors: INVALID_ARG. */
int sdg_nodes(int N, double* xi, double* w);

/* The 1D reference matrices of degree N, each (N+1)x(N+1) row-major, written
 * to host array `out` in this order: M (mass), R~, L~, R-bar, L-bar
 * (Eq. matrices), M^L, M^R (Sec. 2.2, L2 projections), H^R, H^L, H^C
 * (after Eq. pSyst).  `out` holds 10*(N+1)^2 doubles.  Errors: INVALID_ARG. */
int sdg_matrices(int N, double* out);

/* Orthogonal projector (row-major (N+1)x(N+1), host array `proj`) onto the
 * local patterns c with (R~ - L~) c = 0, and its dimension (host int, may be
 * NULL).  Repeated in every cell and multiplied over the directions, these
 * patterns span the kernel of the periodic pressure operator: the weak
 * solutions of grad p = 0 of Sec. 2.1 (the constants for even N; the
 * constants and one per-cell sawtooth-like pattern per direction for odd N).
 * Errors: INVALID_ARG. */
int sdg_kernel_projector(int N, double* proj, int* dim);

/* The 1D line operator the FP64 (fp32 = 0) or FP32 (fp32 != 0) kernels
 * apply with the accurate contraction, evaluated on the host in extended
 * precision from the coefficients they store: HL, HR the neighbour blocks
 * (stand-ins for H^L, H^R after Eq. pSyst) and Mc the centre block H^C
 * plus the symmetric correction that makes the stored operator vanish on
 * the local kernel (see sdg_kernel_projector).  Three host arrays of
 * (N+1)^2 doubles, row-major.  By construction HL = HR^T and Mc = Mc^T
 * (exactly, up to the extended-precision evaluation) and
 * (HL + Mc + HR) c = 0 for every kernel pattern c.  Every CG iteration
 * and true residual uses this form; the FP64 sdg_pressure_apply /
 * sdg_viscous_apply and the pressure right-hand side apply HL, H^C and HR
 * directly (the same operator in exact arithmetic).
 * Errors: INVALID_ARG. */
int sdg_line_operator(int N, int fp32, double* HL, double* Mc, double* HR);

/* Create a problem: grid, degree N, viscosity nu >= 0, implicitness
 * theta in [1/2, 1] (Sec. 2.1, P^{n+theta}), time step dt > 0.  Allocates
 * the state (U_d, P) and every work buffer on the current CUDA device.
 * Defaults: see sdg_set_options.
 * Errors: INVALID_ARG, CUDA. */
int sdg_create(const sdg_grid* grid, int N, double nu, double theta, double dt,
               sdg_handle** out);
int sdg_destroy(sdg_handle* h);

/* Precision mode and CG controls: relative tolerances on ||r||/||b|| for the
 * pressure and viscous solves, cap on CG iterations per solve.  Both modes
 * run the CG of Sec. 2.1 (no preconditioner) with the accurate operator (the
 * contraction that removes the local kernel patterns first and annihilates
 * them exactly, see sdg_line_operator), and both stop on the TRUE residual
 * ||b - A x|| recomputed in FP64 ("residual replacement": the recomputed
 * residual replaces the recursive one and the iteration continues in the
 * same direction).
 *   SDG_FP64:  iterations in FP64; the residual is replaced when the
 *              recursion reports the tolerance (a long FP64 recursion drifts:
 *              on 256 x 256 cells at N = 7 it reports 1e-12 when the true
 *              residual is 7e-10).
 *   SDG_MIXED: iterations and operator applications in FP32; the dot
 *              products are summed as compensated FP32 pairs per thread and
 *              block and finished in FP64; the FP32 correction is folded into
 *              the FP64 solution and the residual replaced whenever the FP32
 *              residual has dropped by the factor delta since the last
 *              replacement (or after max(2000, iterations/8) FP32
 *              iterations).
 * The tolerance actually used is max(rtol, 3 floor): floor (reported as
 * sdg_cg_info.floor_res) is the residual that rounding the solution to FP64
 * leaves, which no FP64 vector can beat (about 3e-12 on 256 x 256 cells at
 * N = 7); the solves measured here level off at 2.2-2.3 floor.  A true
 * residual that stops improving (FP64: two replacements, mixed: thirty,
 * without a 1.25x gain) within 10 max(floor, eval_res) also ends the solve
 * with OK (eval_res: the rounding of A x itself, which for high degrees lies
 * well above the representation floor).  Above
 * it, a mixed solve continues with FP64 iterations from its current x (FP32
 * rounding of the operator can keep it from resolving modes with tiny
 * eigenvalues; at most 1/8 of its FP32 iterations, counted in
 * applies_fp64) and an FP64 solve ends with SDG_ERR_NOT_CONVERGED; true_res
 * always holds the achieved value.  (Unpreconditioned CG at N = 10, 11 on
 * grids of 64^2 cells and more converges so slowly -- FP64 CG needs 244,000
 * iterations on 64 x 64 cells at N = 11 -- that such solves can end there
 * short of rtol = 1e-12.)
 * For the singular pressure system every replaced residual is projected onto
 * the range of the operator (its kernel part is round-off).
 * Defaults: SDG_FP64, 1e-12, 1e-12, 1000000.  Errors: INVALID_ARG. */
int sdg_set_options(sdg_handle* h, int precision, double rtol_p, double rtol_v,
                    int maxit);
/* Mixed mode: reliable-update factor delta in (0,1) (default 0.5: on the
 * 256 x 256, N = 7 workload it needs 30,100 FP32 iterations against 42,600
 * at 0.1 and 62,700 at 0.001), the cap on FP64 residual replacements per
 * solve (default 10000), and deflate != 0
 * to remove the kernel of the pressure operator (odd N: constants and
 * sawtooth patterns) from every FP32 search direction (default 0: the
 * operator kernel already annihilates those patterns exactly). */
int sdg_set_mixed_options(sdg_handle* h, double delta, int max_updates, int deflate);

/* Number of equal SSP-RK3 sub-steps (dt / nsub each) in which the explicit
 * convection of Sec. 2.2 advances over one time step; the pressure and
 * viscous solves still take the full dt.  The explicit stage is stable only
 * below the CFL limit of Eq. CFL1 (CFL < 1); a time step above it stays
 * stable with nsub >= CFL / 0.5.  nsub = 1 (default) is the scheme as the
 * paper states it.  Errors: INVALID_ARG unless 1 <= nsub <= 1000. */
int sdg_set_convection_substeps(sdg_handle* h, int nsub);

/* Form of a CG iteration on the device.  0: one launch per iteration --
 * the operator kernel of iteration k also applies the update of iteration
 * k-1 (r -= alpha Ap, x += alpha p) while it stages its input, and reduces
 * p.Ap, r.r, r.Ap and Ap.Ap, from which beta is formed one iteration ahead.
 * 1: two launches per iteration, the operator (p = r + beta p, Ap, p.Ap)
 * and the update (x += alpha p, r -= alpha Ap, r.r).  2 (default): two
 * launches, with x += alpha p moved into the next operator launch (which
 * reads p already), so that the update moves only r and Ap.  All are the CG
 * of Sec. 2.1 in exact arithmetic; the FP32 kernel deflation of
 * sdg_set_mixed_options always uses form 1.
 * Errors: INVALID_ARG unless form is 0, 1 or 2. */
int sdg_set_iteration_form(sdg_handle* h, int form);

/* Tile shape of the operator kernel.  2D FP32 (a CTA's box of elements):
 * 0 = base, 1 = twice as wide in x, 2 = twice as wide in y (fewer halo
 * loads per element, twice the threads per CTA).  3D: 0 = columns of 4 x 4
 * elements marching through z with a three-plane ring in shared memory
 * (N <= 4; default), 1 or 2 = boxes of elements with their face halo.  The
 * shape changes the summation order of the CG's dot products, so results
 * differ in the last bits between shapes (each is deterministic).  The
 * one-launch CG iteration (sdg_set_iteration_form) uses the base 2D shape.
 * Errors: INVALID_ARG. */
int sdg_set_tile(sdg_handle* h, int variant);
/* Times the FP32 operator of the handle's grid with every tile shape (10
 * launches each, CUDA events on `stream`), keeps the fastest and returns it
 * in *variant (may be NULL); us (may be NULL) receives the mean launch time
 * of each shape in microseconds (3 entries in 2D, 2 in 3D).  No counterpart
 * in the paper: a tuning aid.  Synchronises the stream. */
int sdg_autotune(sdg_handle* h, int* variant, double* us, void* stream);

/* Number of DOF of one field (ncell * n1^dim). */
long long sdg_ndof(const sdg_handle* h);

/* Copy the state in / out.  u, v (, w in 3D; NULL in 2D), p: host or device
 * arrays of sdg_ndof doubles.  The initial pressure is used as P^n of the
 * first step (Eq. pSyst).  Errors: INVALID_ARG, CUDA. */
int sdg_set_state(sdg_handle* h, const double* u, const double* v,
                  const double* w, const double* p, void* stream);
int sdg_get_state(sdg_handle* h, double* u, double* v, double* w, double* p,
                  void* stream);

/* ---------------------------------------------------------------- operators */

/* y = theta * A' x with A' = dt sum_d (1/dx_d^2) M^{perp d} (H^L x_{i-1} +
 * H^C x_i + H^R x_{i+1})_d : the left-hand side of Eq. pSyst, periodic.
 * x, y: device arrays of sdg_ndof elements, double (fp32 = 0) or float
 * (fp32 = 1); x and y must not overlap.  Errors: INVALID_ARG, CUDA. */
int sdg_pressure_apply(sdg_handle* h, const void* x, void* y, int fp32,
                       void* stream);

/* y = (M + nu H) x of Eq. implicitviscosity with the scales of Eqs. uSDG12
 * and Ux-Uz: M^{xyz} x + nu dt sum_d (1/dx_d^2) M^{perp d} H_d x.
 * Same arguments as sdg_pressure_apply. */
int sdg_viscous_apply(sdg_handle* h, const void* x, void* y, int fp32,
                      void* stream);

/* ---------------------------------------------------------------- solvers */

/* Solve theta A' x = b (Eq. pSyst) by matrix-free CG without
 * preconditioner (Sec. 2.1), in the handle's precision mode.  b: device,
 * sdg_ndof doubles, must be orthogonal to the kernel of the operator (see
 * sdg_kernel_projector; the solve does not project it).  x: device, in = x0,
 * out = solution; its kernel component stays that of x0 (in mixed mode it
 * is restored explicitly after the FP32 iterations).
 * info may be NULL.  Returns the solve status (OK, NOT_CONVERGED, BREAKDOWN)
 * or INVALID_ARG / CUDA. */
int sdg_pressure_cg(sdg_handle* h, const double* b, double* x,
                    sdg_cg_info* info, void* stream);

/* Solve (M + nu H) x = b (Eq. implicitviscosity) by CG; same conventions. */
int sdg_viscous_cg(sdg_handle* h, const double* b, double* x,
                   sdg_cg_info* info, void* stream);

/* ---------------------------------------------------------------- step stages */

/* L2 projection of a velocity component d (0..dim-1) from its dual grid to
 * the main grid (Eq. l2forward) or back (Eq. l2backward).  in, out: device
 * doubles, sdg_ndof, must not overlap. */
int sdg_dual_to_main(sdg_handle* h, int d, const double* in, double* out,
                     void* stream);
int sdg_main_to_dual(sdg_handle* h, int d, const double* in, double* out,
                     void* stream);

/* Explicit convection of a main-grid velocity V (dim device arrays) over one
 * dt by third-order SSP Runge-Kutta with the Rusanov-flux DG operator
 * (Eqs. Fu-Fw, Sec. 2.2), in sdg_set_convection_substeps sub-steps; writes
 * F (dim device arrays, disjoint from V). */
int sdg_convect(sdg_handle* h, const double* const* V, double* const* F,
                void* stream);

/* Pressure right-hand side from dual-grid velocities U* (dim device arrays)
 * and the old pressure: b = -sum_d (1/dx_d) M^{perp d} (R-bar U_{i+1/2} -
 * L-bar U_{i-1/2})_d - (1 - theta) A' P_old (Eqs. pSDG1, pSyst), then b is
 * shifted to zero mean.  b: device doubles. */
int sdg_pressure_rhs(sdg_handle* h, const double* const* Ustar,
                     const double* P_old, double* b, void* stream);

/* Velocity update of Eq. LOvelocityU-W with q = theta P_new +
 * (1 - theta) P_old: U_d = U*_d - (dt/dx_d) M^-1 (R~ q_{i+1} - L~ q_i)_d.
 * Ustar, U: dim device arrays each (U may alias Ustar). */
int sdg_velocity_update(sdg_handle* h, const double* const* Ustar,
                        const double* P_new, const double* P_old,
                        double* const* U, void* stream);

/* ---------------------------------------------------------------- time step */

/* Advance the handle's state by nsteps steps of the compact fractional-step
 * scheme (Eqs. LOdiffusionU-W, LOpressure, LOvelocityU-W): project to the
 * main grid, SSP-RK3 convection (in sdg_set_convection_substeps sub-steps),
 * implicit viscous CG per component, project back, pressure CG, velocity
 * update, pressure gauge (zero mean).
 * info may be NULL.  Returns the first non-OK solve status, or OK. */
int sdg_step(sdg_handle* h, int nsteps, sdg_step_info* info, void* stream);

/* ---------------------------------------------------------------- adjoint */

/* Adjoint (reverse-mode derivative) of one sdg_step, with respect to the
 * state and the viscosity, for gradient-based use of the scheme.  The step
 * is differentiated stage by stage as a map (U^n, P^n, nu) -> (U^{n+1},
 * P^{n+1}) with both linear systems solved exactly: transposed projections
 * (Eqs. l2forward, l2backward), the transposed velocity update and pressure
 * right-hand side (Eqs. LOvelocityU-W, pSDG1, pSyst), the pressure and
 * viscous solves (symmetric operators: one CG each with the same kernels),
 * the gauge and the kernel part of P (reading R3), and the Rusanov
 * convection (Eqs. Fu-Fw) linearised at the recomputed RK3 stages, with the
 * sub-gradient of the larger side of the flux speed 2 max(|v-|, |v+|).
 *   U:    dim device arrays, the dual-grid velocities at the start of the
 *         step (the checkpoint; the stages are recomputed from it).
 *   lamU: dim device arrays; in: d loss / d U^{n+1}; out: d loss / d U^n.
 *   lamP: device array; in: d loss / d P^{n+1}; out: d loss / d P^n.
 *   dnu:  host double; d loss / d nu of this step is ADDED to it.
 * The handle's state is not touched; its precision and tolerances apply to
 * the four CG solves.  The first call allocates a work arena of
 * (3 nsub + 7) dim + 5 fields.  Returns the first non-OK solve status. */
int sdg_step_adjoint(sdg_handle* h, const double* const* U, double* const* lamU,
                     double* lamP, double* dnu, void* stream);

/* ---------------------------------------------------------------- batches */

/* A batch of independent problems of uneven size and degree (each one the
 * scheme of Sec. 2 on its own grid), stepped together.  Every member is an
 * sdg_handle with its own non-blocking CUDA stream; sdg_batch_step advances
 * the members concurrently from a pool of host threads (largest first), so
 * that many small problems occupy the GPU at once. */
typedef struct sdg_batch sdg_batch;

/* nprob members: grids[i], degree N[i], viscosity nu[i] (host arrays), all
 * with the same theta and dt.  Argument rules and errors as sdg_create, per
 * member; on error no batch is returned. */
int sdg_batch_create(const sdg_grid* grids, const int* N, const double* nu,
                     int nprob, double theta, double dt, sdg_batch** out);
int sdg_batch_destroy(sdg_batch* b);
/* Number of members (0 for NULL). */
int sdg_batch_size(const sdg_batch* b);
/* Member i (owned by the batch: do not destroy it), for sdg_set_state,
 * sdg_get_state, sdg_set_options, sdg_set_convection_substeps and the other
 * per-handle calls.  Errors: INVALID_ARG. */
int sdg_batch_member(sdg_batch* b, int i, sdg_handle** h);
/* Host threads used by sdg_batch_step (default min(nprob, 16, cores)). */
int sdg_batch_set_threads(sdg_batch* b, int nthreads);
/* nsteps steps of every member (as sdg_step), ordered after the work queued
 * on `stream` before the call and before the work queued on it after.
 * info: host array of nprob entries, or NULL.  Returns the first non-OK
 * member status (by index); sdg_last_error names the member. */
int sdg_batch_step(sdg_batch* b, int nsteps, sdg_step_info* info, void* stream);

/* ---------------------------------------------------------------- instrumentation */

/* enable != 0: bracket every launch of the fused CG operator kernel with CUDA
 * events on the launch stream and accumulate its device time (costs a few
 * microseconds of host time per launch).  Resets the counters below. */
int sdg_set_profiling(sdg_handle* h, int enable);

/* Counters since sdg_create or the last sdg_set_profiling: kernels launched
 * by the handle, and (profiling on) the summed device time in ms and the
 * number of timed launches of the fused CG operator kernel, index 0 = FP64,
 * 1 = FP32.  Host outputs; any may be NULL. */
int sdg_counters(const sdg_handle* h, long long* launches, double* apply_ms,
                 long long* apply_launches);

/* ---------------------------------------------------------------- diagnostics */

/* Kinetic energy K = (1/|Omega|) int |v|^2/2 (Sec. 2.5) of the handle's
 * state, by GL quadrature on each dual grid; and the Euclidean norm of the
 * discrete divergence of Eq. pSDG1.  Host outputs; either may be NULL. */
int sdg_diagnostics(sdg_handle* h, double* kinetic_energy, double* div_norm,
                    void* stream);

/* ---------------------------------------------------------------- allocation-free */

/* Kinetic energy K = (1/|Omega|) int |v|^2 / 2 of caller-owned velocity
 * arrays, like the kinetic_energy output of sdg_diagnostics, for callers that
 * cannot allocate device memory: code whose device memory is owned by another
 * allocator or pool, and latency-critical loops where an allocation would
 * stall the device.  The paper has no counterpart; it is a
 * service of this library.
 *   - Needs no handle and calls no cudaMalloc, cudaFree or allocating
 *     library routine.  Its scratch (partial sums and a ticket counter) is a
 *     fixed 32 KB array compiled into the library, held by every GPU that
 *     loads it until the process exits.
 *   - grid, N: as for sdg_create (periodic box, 0 <= N <= 11).  u, v (, w in
 *     3D, ignored in 2D): device arrays of ncell * (N+1)^dim doubles in the
 *     layout above, each component on its own grid.  ke: device pointer to
 *     one double, written on `stream`.
 *   - At most 67,108,864 nodes per component; larger grids return
 *     SDG_ERR_INVALID_ARG with the limit in sdg_last_error.
 *   - The first call in each CUDA context of a device looks up the scratch
 *     array's device address (cudaGetSymbolAddress) with that device
 *     current, and keeps it for later calls in the same context (a new
 *     context, e.g. after cudaDeviceReset, repeats the look-up).
 *   - Every call shares the one scratch array: calls that can overlap on the
 *     GPU (different streams, or different host threads) race and must be
 *     ordered by the caller.  Each call clears the counter it relies on.
 * Errors: INVALID_ARG, CUDA. */
int sdg_kinetic_energy_noalloc(const sdg_grid* grid, int N, const double* u,
                               const double* v, const double* w, double* ke,
                               void* stream);

const char* sdg_strerror(int status);
const char* sdg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SDG_H */
