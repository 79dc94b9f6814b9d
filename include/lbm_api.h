/*
 * lbm_api.h -- C ABI of the GB300 library for the coupled, locally
 * volume-conserving lattice Boltzmann step of Xiong, Wang & Liu,
 * "Local volume-conserving lattice Boltzmann model for incompressible
 * multiphase flows" (arXiv 2505.10899).
 *
 * One time step couples
 *   - the interface-capturing MRT-LB for the modified Cahn-Hilliard equation
 *     (Sec. 3.2, Eqs. 30-37; target PDE Eq. 17), whose source carries the
 *     level-set sharpening flux (lambda/W)[1 - tanh^2(2 psi/W)] grad(psi)/|grad(psi)|
 *     (Eq. 32), and
 *   - the hydrodynamic MRT-LB for incompressible two-phase flow
 *     (Sec. 3.1, Eqs. 20-29; target PDE Eq. 18) driven by F_s = hbar grad(phi),
 * with the isotropic gradient/Laplacian stencils of Sec. 3.2 for grad(phi),
 * lap(phi) and grad(psi), on the D2Q9 lattice of Eq. 19.  Lattice units:
 * dt = dx = 1, c_s^2 = 1/3.  The grid is periodic in x; in y it is
 * periodic, or bounded by moving walls (lbm_params.walls).
 *
 * Conventions shared by every entry point
 *   - Return value: LBM_OK (0) or a negative LBM_ERR_* code.  No C++
 *     exception crosses the ABI.  lbm_last_error() gives a message for the
 *     last failing call of the calling thread.
 *   - Device memory: the library never allocates device memory.  The caller
 *     passes one device buffer (the workspace) of lbm_workspace_bytes()
 *     bytes, 256-byte aligned, which must outlive the handle.  All
 *     simulation state lives there.
 *   - Host memory: every host array is owned by the caller; the library
 *     copies in or out during the call and keeps no host pointer.  Host
 *     fields are always FP64, whatever the device precision.  Layout of a
 *     2-D field: [y][x], x fastest; of populations: [i][y][x] with i the
 *     D2Q9 index of Eq. 19; of phi*u: [component][y][x].
 *   - Streams: every call enqueues its work on the CUDA stream given to
 *     lbm_init (NULL = legacy default stream).  Calls that return host data
 *     (lbm_volume, lbm_fields, lbm_get_state, lbm_save, lbm_status)
 *     synchronise that stream; lbm_step does not.
 *   - Batches: one handle advances ncases >= 1 independent grids of
 *     possibly different sizes in the same kernel launches.  Fields that
 *     define the launch (precision, flow, W, sigma, lambda, xi, tau_g, the
 *     free MRT rates, vortex_U, vortex_T) must be equal across the batch;
 *     nx, ny, rho_l, rho_g, tau_f_l, tau_f_g may differ per case.
 *   - Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef LBM_API_H
#define LBM_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 2

typedef struct lbm_handle lbm_handle; /* opaque; freed by lbm_destroy */

enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,           /* invalid argument or parameter set */
  LBM_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  LBM_ERR_WORKSPACE = -3,     /* workspace missing, too small or misaligned */
  LBM_ERR_NONFINITE = -4,     /* a NaN/Inf appeared in the macroscopic fields */
  LBM_ERR_TIMEOUT = -5,       /* a bounded device wait gave up (lbm_set_wait_limit) */
  LBM_ERR_UNIMPLEMENTED = -6, /* entry point declared but not built */
  LBM_ERR_BOUNDS = -7         /* the library built with index checks found an
                                 index out of range (liblbm_gb300_checked.so) */
};

/* Storage and arithmetic precision.  Under LBM_F32 the rest population g_0
 * is kept as an unevaluated sum of two FP32 values, formed exactly from phi
 * minus the stored movers, so that the populations of every node sum to the
 * phi that entered it to ~2^-48 and FP32 rounding does not drift the phase
 * volumes (Sec. 4.1 measures exactly these volumes). */
enum { LBM_F64 = 0, LBM_F32 = 1 };
enum { LBM_FLOW_COUPLED = 0, LBM_FLOW_VORTEX = 1 }; /* see lbm_params.flow */

/* Parameters of one case (one grid, periodic in x; in y periodic or closed
 * by moving walls). */
typedef struct {
  int32_t abi_version; /* must be LBM_ABI_VERSION */
  int32_t nx, ny;      /* nodes in x and y, each >= 1 */
  int32_t precision;   /* LBM_F64 or LBM_F32 */
  /* LBM_FLOW_COUPLED: both LB equations, u from Eq. 28.
   * LBM_FLOW_VORTEX: the phase-field LB alone under the prescribed
   * time-reversed single vortex of Eqs. 43-44 (Sec. 4.2):
   *   u = -U sin^2(pi X) sin(2 pi Y) cos(pi t/T),
   *   v =  U sin^2(pi Y) sin(2 pi X) cos(pi t/T),
   * X = (x + 1/2)/nx, Y = (y + 1/2)/ny, t the step index; U < 0 gives the
   * sign printed in Eqs. 43-44. */
  int32_t flow;
  /* 0: periodic in y.  1: walls half a node below y = 0 and above y = ny-1,
   * moving along x at u_wall_bottom and u_wall_top (the sheared cavity of
   * Sec. 4.4; the paper gives no boundary scheme, so the reading is):
   * halfway bounce-back; a returning f_i gains 2 w_i rho (c_i . u_w)/c_s^2
   * with rho = rho(phi) of the receiving node; g bounces back without a
   * term (no flux of phi through a wall: the phase volume is kept); the
   * stencils see a ghost row mirroring the wall row (zero normal gradient
   * of phi and psi: neutral wetting, 90-degree contact angle).
   * LBM_FLOW_COUPLED only. */
  int32_t walls;
  double W;         /* interface width (Eq. 4) */
  double sigma;     /* surface tension; beta = 12 sigma/W, kappa = 3 sigma W/2 (Sec. 2) */
  double lambda;    /* penalty constant (Eq. 6; 0.5 in the paper); 0 = classical C-H */
  double xi;        /* regulariser of psi (Eq. 37; 1e-10 in the paper) */
  double tau_g;     /* phase-field relaxation time; mobility M = (tau_g - 1/2)/3 (Eq. 34) */
  double rho_l, rho_g;     /* densities of the phi = 1 and phi = 0 fluids */
  double tau_f_l, tau_f_g; /* f relaxation times in each bulk; viscosity from Eq. 27 */
  /* MRT rates of Eq. 26 in the moment order of Eq. 24.  s_f[7], s_f[8] are
   * replaced by 1/tau_f(phi) and s_g[3], s_g[5] by 1/tau_g (Eqs. 27, 34);
   * the other entries are free (the paper does not fix them; 1.0 is the
   * usual choice) and must lie in (0, 2). */
  double s_f[9], s_g[9];
  double vortex_U, vortex_T; /* flow == LBM_FLOW_VORTEX only */
  double u_wall_top, u_wall_bottom; /* walls == 1 only: wall velocities along x */
} lbm_params;

/* Device bytes the caller must provide for this batch (0 on bad params). */
size_t lbm_workspace_bytes(const lbm_params* cases, int32_t ncases);

/* Create a handle and set the initial state of every case (Sec. 4 set-ups):
 *   phi = h_phi0[c] ([ny][nx], FP64), u = h_u0[c] ([2][ny][nx], FP64; the
 *   array pointer or an entry may be NULL for a fluid at rest), p = 0;
 *   hbar0 = Eq. 2 on phi0; g = g_eq(phi0, hbar0, u0) (Eq. 31);
 *   f = f_eq(p = 0, rho(phi0), u0) (Eq. 22); phi*u at t-1 := phi0 u0.
 * rho(phi) = rho_g + phi (rho_l - rho_g) and mu(phi) linear likewise;
 * tau_f(x) = mu/(rho c_s^2) + 1/2 (Eq. 27).  In vortex mode u0 is ignored.
 * The arrays may lie in pageable host memory (copied through the workspace's
 * staging planes), or in page-locked host or device memory (read in place by
 * the init kernel).  The call synchronises the stream: on return no array
 * is read any more.
 * d_workspace: device pointer, >= lbm_workspace_bytes(), 256-byte aligned.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: LBM_ERR_ARG, LBM_ERR_WORKSPACE, LBM_ERR_CUDA. */
int lbm_init(const lbm_params* cases, int32_t ncases, void* d_workspace,
             size_t ws_bytes, const double* const* h_phi0,
             const double* const* h_u0, void* stream, lbm_handle** out);

/* Advance every case by nsteps >= 0 coupled time steps (Eqs. 20-37):
 * stream, phi = sum g (Eq. 35), psi (Eq. 37, phi clipped to [0,1]),
 * isotropic stencils (Sec. 3.2), hbar (Eq. 2), F = hbar grad phi, u and p
 * (Eqs. 28-29), MRT collision of f (Eqs. 21-25) and of g (Eqs. 31-33) with
 * d_t(phi u) by backward difference.  Asynchronous on the handle's stream:
 * runs of 4 steps or more are cut into chunks of up to 64 steps; the first
 * chunk of a given length (and source buffer) is launched directly, and
 * when that length comes again its steps are captured into a CUDA graph,
 * cached (a few per handle) and replayed from then on (lbm_prepare_steps
 * builds them ahead of time).  Shorter runs are always launched directly.
 * Errors: LBM_ERR_ARG,
 * LBM_ERR_CUDA (launch failure; device faults surface at the next
 * synchronising call). */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Build (capture and instantiate) the graphs that a following
 * lbm_step(h, nsteps) will replay, without running any step, so that the
 * first call of a new step count does not pay for the capture.  Optional.
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_prepare_steps(lbm_handle* h, int64_t nsteps);

/* Chains: the batch's cases are split into nchains contiguous groups of
 * nearly equal node counts (1 <= nchains <= 4, at most one per case; the
 * default is 2 when there are two cases or more).  The steps of each group
 * are captured as a separate branch of the step graph, so that while the
 * last CTAs of one group's step drain, the other group's CTAs keep the SMs
 * busy; the groups are independent, so the results do not change.  Within
 * a group the largest cases are scheduled first.
 * lbm_get_chains returns the number of chains in use (up to 8 with
 * whole-row chains, below).  lbm_set_chains rebuilds the work-item table
 * (synchronises).  Errors: LBM_ERR_ARG. */
int lbm_set_chains(lbm_handle* h, int32_t nchains);
int32_t lbm_get_chains(const lbm_handle* h);

/* Whole-row chains (on = 1; off by default; lbm_autotune tries both): with
 * the bulk-copy kernel in FP32 and strips of 128 columns, a case whose row
 * fits a width of 64, 96, 192 or 256 columns (the smallest that holds it,
 * 128 included, decides) runs each row as one strip of that width, in one
 * extra chain per width.  A whole-row strip copies its row once per plane and
 * needs no periodic-wrap pieces, so batches of such cases step faster (192-
 * wide cases: 0.81 of the HBM roofline instead of 0.69 with 128-column
 * strips); in a batch that mixes them with wide cases the chains of different
 * widths share the SMs less well.  The other cases form the nchains groups.
 * Results are those of any tiling (see lbm_set_tiling).  lbm_get_row_chains
 * reports whether they are in use (1) or not (0).  Rebuilds the work-item
 * table (synchronises).  Errors: LBM_ERR_ARG. */
int lbm_set_row_chains(lbm_handle* h, int32_t on);
int32_t lbm_get_row_chains(const lbm_handle* h);

/* Bound of the device waits, in SM clock cycles: the bulk-copy kernel's
 * waits for its staged rows and the persistent kernel's grid barrier.  A
 * wait that gives up raises LBM_ERR_TIMEOUT (reported by the next
 * synchronising call or lbm_status); the kernel first waits, with the
 * default bound, for the copies it issued, then returns, and the step's
 * results are not valid.  cycles < 0 restores the default, about 2 s
 * (4e9 cycles); 0 gives up at the first poll that finds the data missing
 * (used to test the timeout path).  Errors: LBM_ERR_ARG. */
int lbm_set_wait_limit(lbm_handle* h, int64_t cycles);

/* Declare the volume regions of case c: h_labels [ny][nx] with values in
 * [0, nregions) or -1 (no region); NULL means one region = whole grid.
 * 1 <= nregions <= 8.  Copies the labels into the workspace. */
int lbm_set_regions(lbm_handle* h, int32_t c, const int8_t* h_labels,
                    int32_t nregions);

/* Phase volumes V_r = sum over region r of phi (the droplet volumes of
 * Fig. 3b) for every case, reduced in FP64 in a fixed order (bitwise
 * reproducible).  h_out receives lbm_num_regions(h) doubles, case-major.
 * Synchronises; returns LBM_ERR_NONFINITE if a NaN/Inf was flagged. */
int lbm_volume(lbm_handle* h, double* h_out);

/* Same reduction, written to device memory d_out (lbm_num_regions doubles)
 * without synchronising. */
int lbm_volume_async(lbm_handle* h, double* d_out);

/* Fused volume tracking.  With d_out non-NULL, every following step also
 * reduces phi (Eq. 35, the state entering the step) over each case in FP64
 * inside the step kernel and writes the per-case totals to d_out[ncases]
 * (device memory, overwritten every step, so after lbm_step(n) it holds the
 * volumes at time t+n-1).  Under LBM_F32 the fused sum may leave out the low
 * part of g_0 (below 2^-24 g_0 per node); lbm_volume counts it.  Only for
 * batches whose cases all have one region (no labels): LBM_ERR_ARG
 * otherwise.  d_out = NULL switches tracking off. */
int lbm_track_volume(lbm_handle* h, double* d_out);

/* Fused volume tracking with a history: like lbm_track_volume, but the step
 * from time t writes the per-case volumes of the state at time t to slot
 * t mod nslots of out (slot k: out[k * ncases .. (k+1) * ncases)).  out may
 * be device memory or page-locked host memory that the device can address
 * (cudaHostAlloc, or pinned and registered memory): the step kernels' final
 * reduction then writes each step's volumes to the host by itself, so a run
 * of n <= nslots steps in one lbm_step call delivers every step's volumes
 * without a copy or a synchronisation between steps.  The caller reads them
 * after synchronising the stream.  nslots >= 1; lbm_track_volume(h, p) is
 * nslots = 1.  out = NULL switches tracking off.  Errors: LBM_ERR_ARG
 * (labelled regions, nslots < 1, out neither device nor page-locked). */
int lbm_track_volume_history(lbm_handle* h, double* out, int64_t nslots);

/* Work tiling of the step kernel: each CTA owns a strip of bx columns
 * (bx in {32, 64, 128}; whole-row chains, see lbm_set_chains, take their own
 * width) and marches down runs of `rows` rows (2..1024).
 * lbm_init picks a default from the batch size; lbm_set_tiling replaces it
 * (results agree for every tiling up to floating-point rounding: the
 * per-node operations are the same, but different kernel instantiations
 * may fuse multiply-adds differently; for a given tiling runs are
 * bitwise reproducible).
 * lbm_get_tiling also reports the number of CTAs (work items) per step. */
int lbm_get_tiling(const lbm_handle* h, int32_t* bx, int32_t* rows,
                   int32_t* n_items);
int lbm_set_tiling(lbm_handle* h, int32_t bx, int32_t rows);

/* Self-tuning: time every (kernel variant, bx, rows) candidate on this
 * batch with max(trials, 8) trial steps each (CUDA events on the handle's
 * stream) and keep the fastest.  The step kernels of variants 1 and 2 are
 * timed as a captured CUDA graph of those steps, as lbm_step replays them;
 * variant 3 as one persistent launch.  Trial launches read the current
 * state and write only the buffers the next step overwrites, so the state
 * and the step index do not change.  Outputs may be NULL.  Synchronises. */
int lbm_autotune(lbm_handle* h, int32_t trials, int32_t* best_kernel,
                 int32_t* best_bx, int32_t* best_rows, double* best_ms);

/* Step-kernel variant: 0 = automatic, 1 = register-pipelined loads (any
 * grid), 2 = bulk-copy (TMA) staged loads through shared memory (needs every
 * case to have nx >= 4 and nx a multiple of 4 in FP32, of 2 in FP64).  Both
 * run the same per-node arithmetic (equal up to rounding, see
 * lbm_set_tiling).  lbm_get_kernel returns the variant in use (1 or 2).
 * Changing the variant rebuilds the work-item table (whole-row chains run
 * the bulk-copy kernel only; synchronises). */
int lbm_set_kernel(lbm_handle* h, int32_t variant);
int32_t lbm_get_kernel(const lbm_handle* h);

/* Total number of volume regions over all cases. */
int32_t lbm_num_regions(const lbm_handle* h);

/* Macroscopic fields of case c at the current time, each [ny][nx] FP64:
 * phi (Eq. 35), u (Eq. 28, or the prescribed velocity), p (Eq. 29, 0 in
 * vortex mode).  Any pointer may be NULL.  Synchronises. */
int lbm_fields(lbm_handle* h, int32_t c, double* h_phi, double* h_ux,
               double* h_uy, double* h_p);

/* Copy the state of case c to the host: the distributions f_i(x,t), g_i(x,t)
 * after streaming (left-hand sides of Eqs. 20 and 30) as [9][ny][nx] FP64,
 * phi*u at t-1 as [2][ny][nx], and the step index t.  h_f is ignored in
 * vortex mode.  Any pointer may be NULL.  Synchronises. */
int lbm_get_state(lbm_handle* h, int32_t c, double* h_f, double* h_g,
                  double* h_j, int64_t* t);

/* Overwrite the state of case c (same layout as lbm_get_state; values are
 * rounded to the device precision) and set the step index of the batch. */
int lbm_set_state(lbm_handle* h, int32_t c, const double* h_f,
                  const double* h_g, const double* h_j, int64_t t);

/* Current step index of the batch. */
int64_t lbm_time(const lbm_handle* h);

/* Checkpoint / resume: the raw device state of the batch (populations in
 * device precision, under LBM_F32 with the low part of g_0, phi*u, step
 * index), bitwise.  lbm_save synchronises. */
size_t lbm_checkpoint_bytes(const lbm_handle* h);
int lbm_save(lbm_handle* h, void* h_buf, size_t bytes);
int lbm_load(lbm_handle* h, const void* h_buf, size_t bytes);

/* Synchronise the stream and report device-side error flags:
 * LBM_OK, LBM_ERR_NONFINITE or LBM_ERR_CUDA.  Clears the flags. */
int lbm_status(lbm_handle* h);

/* Device snapshots of the state of case c, for checkpointed recomputation:
 * [f*: 9 planes][g*: 9 planes][phi*u: 2 planes], each nx*ny elements of the
 * device precision, in the pull layout (plane i, position x holds the
 * post-collision value that streams to x + c_i; f planes are zero in vortex
 * mode).  Under LBM_F32 a 21st plane follows with the low part of the float
 * pair that stores g_0 (the g_0 plane holds its high part), so that a
 * restored state continues bit for bit.  lbm_snapshot_bytes gives the size.
 * lbm_restore writes such a buffer back as the current state; the step index
 * is set separately with lbm_set_time.  All three are asynchronous on the
 * handle's stream. */
size_t lbm_snapshot_bytes(const lbm_handle* h, int32_t c);
int lbm_snapshot(lbm_handle* h, int32_t c, void* d_buf);
int lbm_restore(lbm_handle* h, int32_t c, const void* d_buf);
int lbm_set_time(lbm_handle* h, int64_t t);

/* Record and advance (single-case handles): for j = 0..count-1, snapshot
 * the current state into d_states + j * stride_bytes (layout of
 * lbm_snapshot), then advance one step.  One call for a whole run of
 * recorded steps, for the reverse mode; asynchronous on the handle's stream.
 * Errors: LBM_ERR_ARG (batch, null buffer, stride below
 * lbm_snapshot_bytes), LBM_ERR_CUDA. */
int lbm_record_steps(lbm_handle* h, int64_t count, void* d_states, int64_t stride_bytes);

/* Reverse mode (discrete adjoint of the coupled step; single-case handles,
 * FP64 or FP32).  An adjoint state has the first 20 planes of the snapshot
 * layout above, in the handle's precision: the derivative of a scalar
 * objective with respect to each stored value.  An FP32 handle runs the
 * adjoint arithmetic in FP32, sums the parameter terms of each warp in FP32
 * and accumulates those sums in FP64; it differentiates the FP32 step at its stored states (g_0 taken as
 * the high part of its float pair, a difference of at most half an FP32 ulp
 * of g_0 in phi).
 *   lbm_adjoint_attach: device scratch of lbm_adjoint_workspace_bytes()
 *     bytes (256-byte aligned, caller-owned, outlives the handle).
 *   lbm_adjoint_seed_phi: adjoint state of an objective that depends on the
 *     current phi only, from its FP64 field derivative d_dphi [ny][nx]
 *     (phi = sum of the pulled g, Eq. 35).
 *   lbm_adjoint_step: the handle must hold the state S_t at step index t;
 *     given the adjoint of S_{t+1} (d_adj_in), writes the adjoint of S_t
 *     (d_adj_out, a different buffer) through the transposed Jacobian of one
 *     step (Eqs. 20-37 as computed by lbm_step), and accumulates on the device
 *     the derivatives with respect to (sigma, tau_g, lambda, tau_f,
 *     u_wall_top, u_wall_bottom); with h_param_grads[6] non-NULL the
 *     accumulated values are added to it and the accumulator is cleared (this
 *     synchronises), with NULL the call is asynchronous.  The tau_f entry is
 *     zero when tau_f varies with phi or in vortex mode, the wall entries
 *     without walls.  Walls are transposed with the rest (bounce-back, the
 *     moving-wall term, the mirrored ghost rows).  The state is not modified.
 *     At the clip of Eq. 37 and where the normal of Eq. 17 is cut to 0
 *     (|grad psi| below 0.1, the ridges of psi and the clipped bulk) the
 *     derivative of the branch taken is used.
 *   lbm_adjoint_step_from: as lbm_adjoint_step, for the state S_t held in
 *     d_state (a snapshot of the case, layout of lbm_snapshot) at step
 *     index t instead of the handle's own state, which is neither read nor
 *     modified.  A reverse sweep over recorded states then needs no
 *     lbm_restore before each step.  d_adj_out must differ from d_adj_in and
 *     d_state; d_state is caller-owned and read on the handle's stream.
 *   lbm_adjoint_init: adjoint of the initial-state map of lbm_init: given the
 *     adjoint of S_0, writes d_adj_phi0 [ny][nx] and accumulates the sigma and
 *     lambda derivatives (h_param_grads as for lbm_adjoint_step); d_phi0
 *     [ny][nx] and d_u0 ([2][ny][nx] or NULL) are FP64 device copies of the
 *     initial fields, and d_adj_phi0 is FP64 whatever the precision.
 *   lbm_adjoint_take_param_grads: adds the accumulated parameter derivatives
 *     to h_param_grads[6] and clears the accumulator (synchronises).
 * Synchronise when h_param_grads is non-NULL.  Errors: LBM_ERR_ARG (batch,
 * null buffers), LBM_ERR_WORKSPACE (no scratch), LBM_ERR_CUDA. */
size_t lbm_adjoint_workspace_bytes(const lbm_handle* h);
int lbm_adjoint_attach(lbm_handle* h, void* d_scratch, size_t bytes);
int lbm_adjoint_seed_phi(lbm_handle* h, const double* d_dphi, void* d_adj_state);
int lbm_adjoint_step(lbm_handle* h, const void* d_adj_in, void* d_adj_out,
                     double* h_param_grads);
int lbm_adjoint_step_from(lbm_handle* h, const void* d_state, int64_t t,
                          const void* d_adj_in, void* d_adj_out, double* h_param_grads);
int lbm_adjoint_init(lbm_handle* h, const double* d_phi0, const double* d_u0,
                     const void* d_adj_state, double* d_adj_phi0,
                     double* h_param_grads);
/* Reverse sweep over recorded states: d_adj holds the adjoint of
 * S_{t0+count} on entry and the adjoint of S_{t0} on return; the state S_t,
 * t0 <= t < t0+count, is read from d_states + (t - t0) * stride_bytes
 * (snapshot layout, as lbm_record_steps writes it).  The count adjoint
 * steps (lbm_adjoint_step_from each) are enqueued in one call, alternating
 * between d_adj and d_spare (a second adjoint state); parameter derivatives
 * accumulate on the device.  Asynchronous.  Errors: LBM_ERR_ARG,
 * LBM_ERR_WORKSPACE, LBM_ERR_CUDA. */
int lbm_adjoint_sweep(lbm_handle* h, const void* d_states, int64_t stride_bytes, int64_t t0,
                      int32_t count, void* d_adj, void* d_spare);
int lbm_adjoint_take_param_grads(lbm_handle* h, double* h_param_grads);

/* Allocation-free phase volumes, for callers that cannot allocate device
 * memory (for example code that runs while a memory pool forbids new
 * allocations, or a host framework that only lends out buffers it owns).
 * The paper has no counterpart: this is a variant of the labelled volume
 * reduction behind lbm_volume that needs no workspace.
 *   d_g: device pointer to the nine phase-field populations after streaming,
 *        g_i(x,t), plane i at d_g + i*plane_stride elements, each plane
 *        [y][x] with x fastest; element type FP64 or FP32 (precision).
 *   d_labels: device int8 [ny][nx], region of each node in [0, nregions) or
 *        -1 (none); NULL = one region, the whole grid.
 *   d_out: device FP64 [nregions], V_r = sum over region r of
 *        phi = sum_i g_i (Eq. 35), reduced in a fixed order.  The nine planes
 *        are summed as given: for an LBM_F32 state of this library, whose g_0
 *        carries a low part outside these planes, the result differs from
 *        lbm_volume by at most half an FP32 ulp of g_0 per node.
 *   stream: cudaStream_t (NULL = legacy default stream); the call enqueues
 *        two kernels and does not synchronise.
 * Limits: 1 <= nregions <= 8, plane_stride >= nx*ny, nx <= 524288 columns
 * (4096 CTAs of 128 columns); larger sizes return LBM_ERR_ARG with a message
 * in lbm_last_error().  Allocates nothing: the per-CTA partial sums live in a
 * fixed static device array of 256 KiB that every GPU which loads the library
 * holds until the process exits.  Every call looks up that array's address
 * on the current device (a host-side query that allocates nothing, so a
 * device reset that reloads the library's kernels leaves no stale address);
 * the first call on a device also loads them, so make it before any stream
 * capture.  All calls share the array and each overwrites what it
 * uses; calls whose kernels overlap on the GPU (different streams, or
 * concurrent host threads) race on it and must be serialised by the caller.
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_phase_volume_noalloc(const void* d_g, int32_t precision, int32_t nx,
                             int32_t ny, int64_t plane_stride,
                             const int8_t* d_labels, int32_t nregions,
                             double* d_out, void* stream);

/* Measurement aid: FP64 fused multiply-add throughput of the current
 * device, the bound of the FP64 step on GB300.  Launches blocks_per_sm
 * (1..8) CTAs of 256 threads per SM, each thread running 8 independent
 * chains of 4 * trips dependent FMAs, once untimed and once timed with CUDA
 * events; *out_per_s receives FMAs per second (count / event time) and
 * *out_ms (may be NULL) the timed duration.  Allocates no device memory;
 * synchronises.  The paper has no counterpart.  Errors: LBM_ERR_ARG,
 * LBM_ERR_CUDA. */
int lbm_fp64_fma_rate(int64_t trips, int32_t blocks_per_sm, double* out_per_s,
                      double* out_ms);

void lbm_destroy(lbm_handle* h);
const char* lbm_status_string(int status);
const char* lbm_last_error(void);
int32_t lbm_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_API_H */
