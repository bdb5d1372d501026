/* hweno.h -- C ABI of the GB300 (sm_103a) HWENO-I library (libhweno.so).
 *
 * The library advances the fifth-order finite-difference interpolation-based Hermite WENO scheme
 * (HWENO-I) of Xie, Tao, Jiao and Zhang (arXiv 2411.11229) on one GPU, in FP64:
 *   - the augmented system u_t + f(u)_x = 0, v_t + h(u,v)_x = 0 with v = u_x, h = f'(u) v
 *     (Sec. 2, Eq. EQ1) and its 2D form with w = u_y (Sec. 3, Eq. EQ3);
 *   - the conservative semi-discretisation L = -(F_{i+1/2} - F_{i-1/2})/dx (- the y difference)
 *     (Eqs. odeH, ode2H);
 *   - one HWENO interpolation per stencil for u^{+-}, v^{+-} and the modified derivative v~
 *     (Sec. 2.1, Eqs. Pxi, P'xi, limiter-p, GHYZ, nonlinear, interp, limiter);
 *   - Lax-Friedrichs fluxes with the central Hermite corrections D(f), D(h)
 *     (Eqs. flux-1d, flux-LF, Cd-1, DfDh) and the linear mixed fluxes (Eq. mixed);
 *   - local characteristic decomposition for the Euler equations (remarks closing Sec. 2 and
 *     Sec. 3): Roe-averaged eigenvectors at each face, cell eigenvectors for v~;
 *   - SSP-RK3 with the modified derivative in the update base (Eqs. fully-hweno, 2Dfully-hweno).
 *
 * Systems: linear advection (f = a_x u, g = a_y u), Burgers (f = g = u^2/2) and the Euler
 * equations with E = P/(gamma-1) + rho |vel|^2 / 2 (Eqs. euler1d, euler2d).
 *
 * STATE LAYOUT.  One state is a contiguous FP64 array [field][comp][ny][nx], x fastest.
 *   fields: 1D (U, V = U_x), 2D (U, V = U_x, W = U_y);
 *   comps : 1 (scalar), 3 (1D Euler: rho, rho*mu, E), 4 (2D Euler: rho, rho*mu, rho*nu, E).
 *   1D problems have ny = 1.  hweno_state_doubles() gives the element count.
 *
 * OWNERSHIP.  All device memory (the state and the workspace) belongs to the caller.  The library
 * borrows the pointers given to hweno_bind() until the next bind or hweno_destroy(), and owns only
 * the handle itself.  Device pointers must be 16-byte aligned.
 *
 * ERRORS.  Every call returns an int status (HWENO_OK = 0 or a negative code); no exception or
 * abort crosses the ABI.  Launches are asynchronous on the handle's stream: a device-side failure
 * (a non-physical state: rho <= 0, P <= 0 or a non-finite wavespeed) is recorded in a device status
 * word and reported as HWENO_ENONPHYS by the next synchronising call (hweno_sync,
 * hweno_last_dt, hweno_max_wavespeed).  CUDA errors are reported as HWENO_ECUDA.
 *
 * THREADS.  A handle is not thread-safe; distinct handles are independent.
 */
#ifndef HWENO_H
#define HWENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hweno_ctx hweno_t;

enum { HWENO_ADVECTION = 0, HWENO_BURGERS = 1, HWENO_EULER = 2 };
enum { HWENO_BC_PERIODIC = 0, HWENO_BC_TRANSMISSIVE = 1, HWENO_BC_REFLECTIVE = 2, HWENO_BC_FIXED = 3 };
/* scheme variants of hweno_create_ex */
enum {
  HWENO_FLAG_V_WEIGHTED = 1,
  HWENO_FLAG_CD2 = 2,
  HWENO_FLAG_R2 = 4,
  HWENO_FLAG_ALPHA_STEP = 8,
  HWENO_FLAG_ALPHA_LOCAL = 16
};
enum {
  HWENO_OK = 0,
  HWENO_EINVAL = -1,   /* invalid argument */
  HWENO_ECUDA = -2,    /* a CUDA runtime error */
  HWENO_ENOMEM = -3,   /* workspace too small / host allocation failed */
  HWENO_ENONPHYS = -4, /* rho <= 0, P <= 0 or non-finite wavespeed met on the device */
  HWENO_ESTATE = -5,   /* call out of order (e.g. no state bound) */
  HWENO_ETOOBIG = -6   /* grid larger than the fixed scratch of hweno_rhs_static */
};

/* Create a solver for a uniform grid of nx (x ny) cells with spacing dx (dy).
 * dim: 1 or 2.  system: HWENO_ADVECTION, HWENO_BURGERS or HWENO_EULER.  gamma: ratio of specific
 * heats (Euler only, > 1).  bc: boundary condition on every side (periodic, as in every accuracy
 * test of Sec. 4; transmissive = zero-order extrapolation of U and of its derivatives; reflective =
 * a wall at each end: ghost cell -1-k mirrors cell k with the sign tables of Eqs. RBC-1d, RBC-2d-x,
 * RBC-2d-y (normal velocity odd; the normal derivative of every other
 * primitive odd, of the normal velocity even), Euler only).
 * EINVAL: dim not 1 or 2, nx < 5 (ny < 5 in 2D), dx or dy <= 0, gamma <= 1 for Euler, unknown
 * system or bc, reflective with a scalar system.  ny and dy are ignored when dim == 1.
 * Defaults (Sec. 4): gamma0 = 0.95 (1D) / 0.99 (2D), d0 = 0.9, eps = 1e-10, CFL = 0.6, a = (1, 1). */
int hweno_create(int dim, int system, int64_t nx, int64_t ny, double dx, double dy, double gamma,
                 int bc, hweno_t **out);

/* Extensions of the scheme for hweno_create_ex.
 *   flags: any of
 *     HWENO_FLAG_V_WEIGHTED  v^+/- formed with the nonlinear weights of u^+/- (the same combination
 *                            of the candidates' derivatives, p1' and p2' being their slopes) instead
 *                            of the linear value p0' of Eq. (interp);
 *     HWENO_FLAG_CD2         the D-terms of Eq. (Cd-2) (Hermite data h_i, h_{i+1}, the alternative
 *                            the paper describes after Eq. D6) instead of Eq. (Cd-1);
 *     HWENO_FLAG_R2          characteristic decomposition with the eigenvectors of each stencil's
 *                            centre cell (U_i for u^-_{i+1/2}, U_{i+1} for u^+_{i+1/2}) instead of
 *                            the Roe average at the face (Euler; no effect on scalar laws).  Every
 *                            cell then interpolates both of its faces in its own characteristic
 *                            fields in one pass.
 *     HWENO_FLAG_ALPHA_STEP  the LF coefficients alpha of Eq. (flux-LF) taken from the input of the
 *                            step's first stage and held for its three stages (the paper does not
 *                            say when alpha is updated; the default recomputes it at every stage);
 *     HWENO_FLAG_ALPHA_LOCAL local LF: alpha at each face is the larger spectral radius of its two
 *                            cells (ghost cells through the boundary map) instead of one maximum
 *                            over the grid (the paper's alpha = max |f'(u)| is read as global).
 *   side[4]: boundary type of the sides x-low, x-high, y-low, y-high (side[2], side[3] unused in
 *     1D): HWENO_BC_PERIODIC (both ends of an axis or neither), _TRANSMISSIVE, _REFLECTIVE (Euler),
 *     or HWENO_BC_FIXED: the ghost cells hold the conserved state fixed[side] with zero derivatives
 *     (the fixed top and bottom states of Example 4.11).
 *   grav: g of the gravity source of Eq. (euler2d-s), (0, 0, g rho, g rho nu) on U and its
 *     derivatives g (0, 0, rho_x, (rho nu)_x) and g (0, 0, rho_y, (rho nu)_y) on the derivative
 *     equations, taken from the stage input (2D Euler only; 0 = none).
 *   fixed[side]: conserved state (rho, rho mu[, rho nu], E) or (u) of a HWENO_BC_FIXED side. */
typedef struct hweno_ext {
  int32_t flags;
  int32_t side[4];
  int32_t pad_;
  double grav;
  double fixed[4][4];
} hweno_ext;

/* hweno_create with the extensions above (ext is read during the call only).  A configuration
 * with no flag, no gravity and one non-fixed type on every side is exactly hweno_create with that
 * type.  EINVAL: as hweno_create, and an unknown flag or side type, periodic on one end of an axis
 * only, reflective with a scalar system, gravity outside 2D Euler, a non-finite or (Euler)
 * non-physical fixed state.  The adjoint entry points return EINVAL for a handle with
 * extensions. */
int hweno_create_ex(int dim, int system, int64_t nx, int64_t ny, double dx, double dy, double gamma,
                    const hweno_ext *ext, hweno_t **out);

/* Linear weights gamma = (gamma0, (1-gamma0)/2, (1-gamma0)/2) and d = (d0, (1-d0)/2, (1-d0)/2)
 * (Sec. 4), epsilon of Eq. (nonlinear), the CFL number, and the advection speeds.
 * EINVAL: gamma0 or d0 outside (0,1), eps <= 0, cfl <= 0. */
int hweno_set_params(hweno_t *h, double gamma0, double d0, double eps, double cfl, double adv_ax,
                     double adv_ay);

/* Stream for all launches and copies of this handle (a cudaStream_t; NULL = legacy default). */
int hweno_set_stream(hweno_t *h, void *cuda_stream);

/* Number of doubles in one state ([field][comp][ny][nx]). */
size_t hweno_state_doubles(const hweno_t *h);

/* Bytes of device workspace hweno_bind() needs (stage base, modified derivatives, nodal fluxes,
 * face fluxes, wavespeed slots and status words). */
size_t hweno_workspace_bytes(const hweno_t *h);

/* Borrow the caller's device state (updated in place by hweno_step) and workspace (at least
 * hweno_workspace_bytes() bytes).  Clears the device scalars (wavespeed slots, time, status, and
 * four slots the kernels read as zero to hold the units of their arithmetic in registers) with an
 * asynchronous memset on the handle's stream; the workspace belongs to the library until the
 * handle is destroyed or rebound.  EINVAL: NULL pointers or unaligned pointers. */
int hweno_bind(hweno_t *h, double *state_dev, void *workspace_dev);

/* One evaluation of the spatial operator at S: L(S) (Eq. odeH / ode2H, every field) and
 * M(S) = (U, V~, W~), the solution with the modified derivatives of Eq. (limiter).  The LF
 * coefficients alpha_x, alpha_y are the maxima of |f'(u)| (Euler: |mu|+c, |nu|+c) over the cells
 * of S.  S, L, M: device arrays of hweno_state_doubles() doubles; S must not alias L or M.
 * Uses the bound workspace (ESTATE if none). */
int hweno_rhs(hweno_t *h, const double *S_dev, double *L_dev, double *M_dev);

/* One SSP-RK3 step of the bound state in place (Eq. fully-hweno / 2Dfully-hweno):
 *   S1 = M(S^n) + dt L(S^n);  S2 = 3/4 B + 1/4 (M(S1) + dt L(S1));  S^{n+1} = 1/3 B + 2/3 (M(S2) + dt L(S2))
 * with B = M(S^n).  dt > 0: fixed step.  dt <= 0: CFL step computed on the device from the
 * wavespeeds of S^n: dt = CFL dx / alpha (1D), CFL / (alpha_x/dx + alpha_y/dy) (2D), clamped to the
 * end time set by hweno_set_time() if one was set; a CFL step issued once that end time is reached
 * has dt = 0 and leaves the state unchanged.  No host synchronisation. */
int hweno_step(hweno_t *h, double dt);

/* nsteps calls of hweno_step(h, dt). */
int hweno_steps(hweno_t *h, double dt, int nsteps);

/* Device time and end time used by CFL steps (t_end <= 0: no clamp); resets the count of steps
 * taken that hweno_run reports. */
int hweno_set_time(hweno_t *h, double t, double t_end);

/* CFL steps of the bound state from t = 0 to t_end (> 0), the last one clamped (the way every
 * example of Sec. 4 runs), or until max_steps steps.  steps_done (may be NULL) receives the number
 * of steps taken.  The steps are issued in chunks of 16 without host synchronisation, replayed from
 * a CUDA graph recorded on a private stream that is ordered after and before the handle's stream;
 * steps of a chunk beyond the end time change nothing.  Returns when the device time has reached
 * t_end, with HWENO_ENONPHYS if a non-physical state was met (the state is then that of the step
 * that met it, or later).  EINVAL: t_end not finite and positive, max_steps < 0; ESTATE: nothing
 * bound. */
int hweno_run(hweno_t *h, double t_end, int64_t max_steps, int64_t *steps_done);

/* Synchronise the stream; read the dt of the last step (and the device time). */
int hweno_last_dt(hweno_t *h, double *dt_host, double *t_host);

/* Synchronise; alpha_x, alpha_y of the bound state (ay = 0 in 1D). */
int hweno_max_wavespeed(hweno_t *h, double *ax, double *ay);

/* Synchronise the stream and report the device status (HWENO_OK or HWENO_ENONPHYS). */
int hweno_sync(hweno_t *h);

/* Copy a host state into the bound device state / the bound state to the host (asynchronous
 * cudaMemcpyAsync on the handle's stream; pinned host memory gives true asynchrony). */
int hweno_upload(hweno_t *h, const double *host_state);
int hweno_download(hweno_t *h, double *host_state);

/* Host-to-host pipeline (not in the paper: for callers whose inputs and results live in host
 * memory).  Bytes of device memory one slot of hweno_pipeline needs: a state and a workspace (each 256-byte
 * aligned within the slot). */
size_t hweno_pipeline_slot_bytes(const hweno_t *h);

/* Independent problems of this handle's grid and scheme, host memory to host memory: problem i is
 * uploaded from host_in[i], advanced by nsteps SSP-RK3 steps with the CFL dt computed on the
 * device (no end time), and downloaded to host_out[i] (host arrays of hweno_state_doubles()
 * doubles; pinned memory lets the copies overlap the steps; host_out[i] may equal host_in[i], the
 * arrays of different problems must not overlap unless i and j share a slot, i = j mod depth).
 * depth slots (1..8) in slot_mem (caller-owned device memory of depth * hweno_pipeline_slot_bytes()
 * bytes, 256-byte aligned), each with its own state, workspace and stream, take the problems in
 * turn (problem i on slot i mod depth), so that the uploads and downloads of some slots run on the
 * copy engines while another slot steps.  The slots start after the work queued on the handle's
 * stream and the handle's stream is ordered after them; the call returns when every result is in
 * host memory, with HWENO_ENONPHYS if any problem met a non-physical state.  The handle's own bound
 * state and workspace are not used.  EINVAL: NULL or unaligned pointers, count or nsteps < 0, depth
 * outside 1..8. */
int hweno_pipeline(hweno_t *h, int count, const double *const *host_in, double *const *host_out, int nsteps,
                   int depth, void *slot_mem);

/* Per-kernel timing (tracing aid).  When on, every stage records CUDA events on the handle's
 * stream around its three launches (cell, face, update kernels).  hweno_kernel_times()
 * synchronises, returns the summed milliseconds and launch counts per kernel kind in
 * ms3[0..2], n3[0..2] (cell, face, update) since the previous query, and resets them. */
int hweno_set_profiling(hweno_t *h, int on);
int hweno_kernel_times(hweno_t *h, double *ms3, long long *n3);

/* Free the handle (not the borrowed device memory). */
void hweno_destroy(hweno_t *h);

/* Static message for a status code. */
const char *hweno_strerror(int status);

/* Bounds-checked build only (libhweno_bounds.so, compiled with -DHWENO_BOUNDS_CHECK; a debugging
 * aid, not in the paper): every cell, face, ghost-line and batch-instance index the kernels form is checked against
 * the extent of the arrays it addresses; an index out of range is counted, the source line of the
 * first one recorded, and the access redirected to element 0 of its array.  Synchronises the
 * device and returns the number of such indices since the previous call (then clears it); *where
 * (may be NULL) receives the first one's source line plus 100000 x its translation unit (0: entry
 * points and stage kernels, 1: batched, 2: adjoint).  Returns -1 in a normal build, HWENO_ECUDA if
 * the synchronisation fails. */
long long hweno_bounds_status(int *where);

/* Bounds-checked build only: the check applied once to an index one past the end of a
 * two-element array in a one-thread kernel (whose one write goes to element 0 whatever the check
 * returns).  Reads and drops the record of earlier launches first, then returns what
 * hweno_bounds_status reports for the probe: 1 when the check works; -1 in a normal build. */
long long hweno_bounds_selftest(void);

/* Number of kernel launches issued by this handle since creation (for accounting). */
long long hweno_launch_count(const hweno_t *h);

/* ---------------------------------------------------------------------------------------------
 * Adjoint (Euler, 1D and 2D; periodic or transmissive).  Not in the paper: derivatives of the
 * scheme above for gradient-based use.  Conventions: the step size and the LF coefficient alpha
 * of every stage are held at the values recorded in the forward pass (the derivative of the
 * CFL rule and of the wavespeed maximum is not taken); d|x|/dx = sign(x) with sign(0) = 0 in the
 * nonlinear weights (Eq. nonlinear).  Everything else -- smoothness indicators, weights, the
 * characteristic projections with their Roe-averaged eigenvectors, fluxes, D-terms, mixed
 * fluxes, modified derivatives -- is differentiated exactly.  All arrays are device arrays in
 * the state layout unless stated; alpha arrays hold {alpha_x, alpha_y} per stage. */

/* Device workspace of the adjoint entry points (7 states, per-face and per-cell contributions). */
size_t hweno_adjoint_workspace_bytes(const hweno_t *h);

/* Record of the last hweno_step: rec7_dev[0] = dt, rec7_dev[1..6] = alpha of stages 1, 2, 3
 * (device to device copy on the stream; no synchronisation). */
int hweno_step_record(hweno_t *h, double *rec7_dev);

/* One SSP-RK3 step of the bound state with the given dt (> 0) and per-stage alpha6_dev instead of
 * the wavespeeds of the stage inputs (replay of a recorded step, as the adjoint assumes). */
int hweno_step_replay(hweno_t *h, double dt, const double *alpha6_dev);

/* lam_out = (dS^{n+1} / dS^n)^T lam_in for one SSP-RK3 step from S_n_dev with dt and alpha6_dev
 * (Eqs. fully-hweno / 2Dfully-hweno transposed: the three stage operators' vector-Jacobian
 * products in reverse order, the stage inputs recomputed from S^n).  Uses the bound workspace as
 * scratch (its stage base and wavespeed slots are overwritten; the bound state and time are not)
 * and adj_ws_dev (hweno_adjoint_workspace_bytes, 256-byte aligned).  S_n, lam_in and lam_out must
 * not alias each other.  All three boundary types of hweno_create (a reflective wall reads its
 * mirrored neighbours through the sign tables, and their adjoints go back through the same
 * tables).  EINVAL for scalar systems, handles of hweno_create_ex with extensions, or dt <= 0. */
int hweno_adjoint_step(hweno_t *h, const double *S_n_dev, double dt, const double *alpha6_dev,
                       const double *lam_in_dev, double *lam_out_dev, void *adj_ws_dev);

/* The same adjoint step when the caller already holds the stage inputs S1, S2 of the step (as
 * hweno_step_replay_stages leaves them): no forward recomputation. */
int hweno_adjoint_step_stages(hweno_t *h, const double *S_n_dev, const double *S1_dev, const double *S2_dev,
                              double dt, const double *alpha6_dev, const double *lam_in_dev,
                              double *lam_out_dev, void *adj_ws_dev);

/* hweno_step (Eq. fully-hweno / 2Dfully-hweno; dt > 0 fixed, dt <= 0 CFL on the device) that also
 * copies the stage inputs S1 (after stage 1) and S2 (after stage 2) of the step to S1_out_dev and
 * S2_out_dev (device arrays of hweno_state_doubles() doubles, 16-byte aligned, not the bound
 * state): with the step's input and hweno_step_record, everything hweno_adjoint_step_stages needs,
 * so that a rollout that keeps them needs no forward recomputation in its backward pass.  EINVAL:
 * NULL or unaligned outputs, dt not finite; ESTATE: nothing bound. */
int hweno_step_stages(hweno_t *h, double dt, double *S1_out_dev, double *S2_out_dev);

/* hweno_step_replay that also copies the stage inputs S1 (after stage 1) and S2 (after stage 2)
 * of the step to S1_out_dev and S2_out_dev. */
int hweno_step_replay_stages(hweno_t *h, double dt, const double *alpha6_dev, double *S1_out_dev,
                             double *S2_out_dev);

/* lam = (dM/dS)^T muM + (dL/dS)^T muL at S with alpha2_dev held fixed: the transpose of one
 * evaluation of hweno_rhs (the building block of hweno_adjoint_step). */
int hweno_stage_vjp(hweno_t *h, const double *S_dev, const double *alpha2_dev, const double *muM_dev,
                    const double *muL_dev, double *lam_dev, void *adj_ws_dev);

/* ---------------------------------------------------------------------------------------------
 * Batched problems (not in the paper: many independent Euler problems of uneven sizes advanced
 * together).  Every instance is an independent HWENO-I problem exactly as above (its own grid,
 * boundary, wavespeeds and CFL step); the batch only changes how the work is launched:
 * hweno_batch_step runs every Runge-Kutta stage over a work-list of tiles of all instances, either
 * as one persistent cooperative launch (cell work, grid barrier, face work, grid barrier, update)
 * or as three persistent launches (one per phase; the default and usually the autotuner's
 * choice), the stages of a step recorded once in a CUDA graph and replayed;
 * hweno_batch_step_plain launches the three kernels of every instance separately (the comparison
 * path).  Both give the same results up to rounding.
 * Only the Euler system is accepted (1D and 2D may be mixed). */
typedef struct hweno_batch hweno_batch_t;

typedef struct {
  int dim, system, bc, pad_;
  int64_t nx, ny;
  double dx, dy, gamma;
} hweno_desc;

/* EINVAL: n <= 0, a non-Euler system, or any instance hweno_create would reject. */
int hweno_batch_create(int n, const hweno_desc *descs, hweno_batch_t **out);
/* Stream for all launches and copies (a non-default stream lets the steps replay a CUDA graph). */
int hweno_batch_set_stream(hweno_batch_t *b, void *cuda_stream);
/* Total doubles of the packed state (instances back to back, each in the state layout) and the
 * offset (in doubles) of instance i. */
size_t hweno_batch_state_doubles(const hweno_batch_t *b);
size_t hweno_batch_state_offset(const hweno_batch_t *b, int i);
/* Bytes of device workspace: the per-instance workspaces plus the batch tables. */
size_t hweno_batch_workspace_bytes(const hweno_batch_t *b);
/* Borrow the packed device state and the workspace (caller-owned); uploads the work-list. */
int hweno_batch_bind(hweno_batch_t *b, double *state_dev, void *workspace_dev);
/* Every instance: t = 0 and end time t_end (<= 0: no clamp) for the CFL steps. */
int hweno_batch_set_time(hweno_batch_t *b, double t_end);
/* nsteps SSP-RK3 steps of every instance with its own CFL step (no host synchronisation). */
int hweno_batch_step(hweno_batch_t *b, int nsteps);
int hweno_batch_step_plain(hweno_batch_t *b, int nsteps);
/* Synchronise; the last dt and the time of every instance (arrays of n doubles; t may be NULL).
 * HWENO_ENONPHYS if any instance met a non-physical state. */
int hweno_batch_dts(hweno_batch_t *b, double *dt_host, double *t_host);
/* Autotuner: times one step of each launch shape (tiles per work item 1, 2, 4; three phase
 * launches, or one cooperative launch with 1 .. occupancy resident blocks per SM) on the bound
 * state, keeps the fastest, and restores the state and the instance times from backup_dev
 * (caller-owned device buffer of hweno_batch_state_doubles() doubles).  Returns the chosen tiles
 * per item and resident blocks per SM (0 = three phase launches).  Results are cached per
 * instance list for the process.  Synchronises. */
int hweno_batch_tune(hweno_batch_t *b, double *backup_dev, int *tiles_per_item, int *blocks_per_sm);
long long hweno_batch_launch_count(const hweno_batch_t *b);
void hweno_batch_destroy(hweno_batch_t *b);

/* hweno_rhs without any allocation.  The paper has no counterpart: this is a convenience for
 * callers that cannot allocate device memory for a workspace, such as host programs whose own
 * framework or memory pool owns every device allocation and passes a library nothing but the
 * input and output buffers, or latency-sensitive loops that cannot afford a cudaMalloc (which can
 * synchronise the whole device).  It evaluates exactly what hweno_rhs evaluates (L(S) and
 * M(S) = (U, V~, W~) with alpha taken from S), with the same kernels, launched on `stream`.
 *   Arguments: the grid as in hweno_create (dim, system, nx, ny, dx, dy, gamma, bc; the same
 *   EINVAL rules); params5 = {gamma0, d0, eps, adv_ax, adv_ay} or NULL for the defaults of
 *   hweno_create; S, L, M: caller-owned device arrays of nfield*ncomp*ny*nx doubles in the state
 *   layout, S not aliasing L or M.
 *   Scratch: a fixed 16 MiB device array inside the library, present on every GPU that loads it
 *   until the process exits.  The grid must fit: about 480 bytes per cell for 2D Euler (roughly
 *   34 000 cells, e.g. 180 x 180) and 144 bytes per cell for 1D Euler; larger grids return
 *   HWENO_ETOOBIG before any device work.
 *   It calls no cudaMalloc, cudaFree or other allocating routine.  The first call on a device looks
 *   up the array's device address (cudaGetSymbolAddress) with that device current; make that first
 *   call before any stream capture.  All calls share the one array, which keeps the previous call's
 *   contents (the wavespeed slot and status word are cleared on the stream at every call), so calls
 *   whose work overlaps on the GPU (other streams, other host threads) race and must be
 *   serialised by the caller.  Device-side failures are reported by later synchronising calls only
 *   through the CUDA error state; use hweno_rhs with a handle to read the status word. */
int hweno_rhs_static(int dim, int system, int64_t nx, int64_t ny, double dx, double dy, double gamma, int bc,
                     const double *params5, const double *S_dev, double *L_dev, double *M_dev, void *stream);

/* Self-test of the library's FP64 reciprocal (the hardware approximation refined by one
 * third-order step, r (1 + e + e^2) with e = 1 - x r; within one unit in the last place; used for
 * every normalisation of the nonlinear weights and every 1/rho):
 * r_dev[i] = 1/x_dev[i] for i < n, launched on `stream`.  Device arrays; EINVAL on NULL/n < 0. */
int hweno_selftest_rcp(const double *x_dev, double *r_dev, int64_t n, void *stream);

/* Probe of the FP64 issue rate of the current GPU, the peak of the stage kernels' ALU roofline
 * (they are bound by the FP64 pipe, not by memory; Sec. 4's CFL-0.6 SSP-RK3 stepping of the
 * scheme is FP64 arithmetic throughout).  Launches, on `stream`, eight resident blocks of 256
 * threads per SM, each thread running eight independent chains of fused multiply-adds whose three
 * operands are thread registers, once untimed and then `reps` times between CUDA events; reports
 * the best rate in fused multiply-adds per second (2 floating-point operations each) in
 * *dfma_per_s and the DFMAs of one launch in *dfma_per_launch (may be NULL).
 *   scratch_dev: caller-owned device array of 4 doubles (the operands and a sink the kernel
 *   writes only in a case that does not occur); reps in 1..100.  Synchronises the stream.
 *   EINVAL on NULL scratch or result pointer or reps out of range, ECUDA on a CUDA error. */
int hweno_selftest_fp64_peak(double *scratch_dev, int reps, void *stream, double *dfma_per_s,
                             double *dfma_per_launch);

#ifdef __cplusplus
}
#endif
#endif /* HWENO_H */
