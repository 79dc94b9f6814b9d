/*
 * lbm3_api.h -- C ABI of the three-dimensional coupled step: the locally
 * volume-conserving model of Xiong, Wang & Liu (arXiv 2505.10899) carried to
 * three dimensions.
 *
 * The paper states the model in two dimensions (D2Q9, MRT).  This extension
 * is its single-relaxation-time limit (Sec. 3.1: with all MRT rates equal the
 * model reduces to SRT) written on textbook three-dimensional lattices:
 *   - hydrodynamics (Eqs. 20-29) on D3Q19, c_s^2 = 1/3, weights 1/3 (rest),
 *     1/18 (6 axis vectors), 1/36 (12 face diagonals), relaxation rate
 *     1/tau_f(phi) with tau_f from Eq. 27;
 *   - the modified Cahn-Hilliard LB (Eqs. 30-37) on D3Q7, c_s^2 = 1/4,
 *     weights 1/4 (rest), 1/8 (axis), rate 1/tau_g; mobility
 *     M = (tau_g - 1/2)/4 (Eq. 34 with this c_s^2);
 *   - the isotropic gradient and Laplacian of Sec. 3.2 with the D3Q19 set.
 * Lattice units, dt = dx = 1; the box is periodic in x, y and z.
 *
 * Conventions are those of lbm_api.h (status codes, caller-owned 256-byte
 * aligned device workspace, host arrays FP64 and copied during the call, one
 * CUDA stream per handle, lbm_last_error()).  Field layout [z][y][x], x
 * fastest; populations [i][z][y][x] with the velocity order
 *    0 (0,0,0)   1 (1,0,0)   2 (-1,0,0)   3 (0,1,0)    4 (0,-1,0)
 *    5 (0,0,1)   6 (0,0,-1)  7 (1,1,0)    8 (-1,-1,0)  9 (1,-1,0)
 *   10 (-1,1,0) 11 (1,0,1)  12 (-1,0,-1) 13 (1,0,-1)  14 (-1,0,1)
 *   15 (0,1,1)  16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 * (D3Q7 uses the first seven).  phi*u: [component][z][y][x].
 */
#ifndef LBM3_API_H
#define LBM3_API_H

#include <stddef.h>
#include <stdint.h>

#include "lbm_api.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3_handle lbm3_handle; /* opaque; freed by lbm3_destroy */

/* Storage precision of the populations.
 *   LBM3_F64: everything FP64.
 *   LBM3_F32: populations and phi*u FP32, arithmetic FP32.
 *   LBM3_F16: f and the six moving g populations stored as IEEE binary16,
 *     arithmetic and phi*u FP32.
 * Under FP32 arithmetic (F32, F16) the rest population g_0 is stored as an
 * unevaluated sum of two FP32 values and formed exactly from phi minus the
 * stored (rounded) movers, so that sum g = phi, hence the phase volume, is
 * kept to ~2^-48 per node and step whatever the rounding of the movers. */
enum { LBM3_F64 = LBM_F64, LBM3_F32 = LBM_F32, LBM3_F16 = 2 };

typedef struct {
  int32_t abi_version; /* LBM_ABI_VERSION */
  int32_t nx, ny, nz;  /* nodes per axis, each >= 1; nx*ny*nz <= 2^31 - 1 */
  int32_t precision;   /* LBM3_F64, LBM3_F32 or LBM3_F16 */
  int32_t reserved;    /* set to 0 */
  double W;            /* interface width (Eq. 4) */
  double sigma;        /* surface tension: beta = 12 sigma/W, kappa = 3 sigma W/2 */
  double lambda;       /* penalty constant (Eq. 6); 0 = classical C-H */
  double xi;           /* regulariser of psi (Eq. 37) */
  double tau_g;        /* phase-field relaxation time, > 1/2 */
  double rho_l, rho_g;     /* densities of the phi = 1 and phi = 0 fluids */
  double tau_f_l, tau_f_g; /* f relaxation times in each bulk (Eq. 27) */
} lbm3_params;

/* Device bytes the caller must provide (0 on bad params). */
size_t lbm3_workspace_bytes(const lbm3_params* p);

/* Create a handle and set the initial state (as lbm_init, in 3-D):
 *   phi = h_phi0 ([nz][ny][nx] FP64), u = h_u0 ([3][nz][ny][nx] FP64, or NULL
 *   for a fluid at rest), p = 0; hbar0 = Eq. 2 on phi0 with the D3Q19
 *   Laplacian; g = g_eq(phi0, hbar0, u0) (Eq. 31 on D3Q7);
 *   f = f_eq(p = 0, rho(phi0), u0) (Eq. 22 on D3Q19); phi*u at t-1 = phi0 u0.
 * rho(phi), mu(phi) linear in phi; tau_f(x) = mu/(rho c_s^2) + 1/2 (Eq. 27).
 * Errors: LBM_ERR_ARG, LBM_ERR_WORKSPACE, LBM_ERR_CUDA. */
int lbm3_init(const lbm3_params* p, void* d_workspace, size_t ws_bytes,
              const double* h_phi0, const double* h_u0, void* stream,
              lbm3_handle** out);

/* Advance nsteps >= 0 coupled steps (the 3-D form of Eqs. 20-37: stream,
 * phi = sum g, psi with clip, D3Q19 stencils of phi and psi, hbar, F, u, p,
 * SRT collisions of f and g with d_t(phi u) by backward difference).
 * Asynchronous on the handle's stream. */
int lbm3_step(lbm3_handle* h, int64_t nsteps);

/* Volume regions: h_labels [nz][ny][nx] int8 in [0, nregions) or -1; NULL =
 * one region, the whole box.  1 <= nregions <= 8. */
int lbm3_set_regions(lbm3_handle* h, const int8_t* h_labels, int32_t nregions);

/* Phase volumes V_r = sum over region r of phi (Eq. 35) in FP64, fixed
 * reduction order.  h_out: nregions doubles.  Synchronises; returns
 * LBM_ERR_NONFINITE if a NaN/Inf was flagged. */
int lbm3_volume(lbm3_handle* h, double* h_out);

/* Fused tracking: with d_out non-NULL every following step also sums phi
 * (the state entering the step) over the box in FP64 inside the step kernel
 * and writes the total to d_out[0] (device memory, overwritten every step).
 * d_out = NULL switches it off. */
int lbm3_track_volume(lbm3_handle* h, double* d_out);

/* Macroscopic fields at the current time, FP64 [nz][ny][nx]: phi (Eq. 35),
 * u ([3][nz][ny][nx], Eq. 28), p (Eq. 29).  Any pointer may be NULL.
 * Synchronises. */
int lbm3_fields(lbm3_handle* h, double* h_phi, double* h_u, double* h_p);

/* State after streaming: f [19][nz][ny][nx], g [7][nz][ny][nx], phi*u at t-1
 * [3][nz][ny][nx], FP64, and the step index.  Any pointer may be NULL.
 * lbm3_set_state rounds to the storage precision (under LBM3_F16, g_0 is
 * stored as given).  Synchronise. */
int lbm3_get_state(lbm3_handle* h, double* h_f, double* h_g, double* h_j, int64_t* t);
int lbm3_set_state(lbm3_handle* h, const double* h_f, const double* h_g,
                   const double* h_j, int64_t t);

/* Step index. */
int64_t lbm3_time(const lbm3_handle* h);

/* Tiling of the step kernel: CTA tile bx x by columns, marching zc planes.
 * Allowed (bx, by): (32, 4), (32, 8), (32, 16), (64, 4) for variants 1-3;
 * (128, 4) and (256, 2) -- whole rows, nx <= bx -- for variant 4; (32, 8)
 * and (64, 4) with nx a multiple of bx and nx >= 2 bx for variant 5; (64, 4)
 * and (64, 2), with the same conditions, for variant 6.  Setting a tile
 * that the variant in use does not run switches to the variant made for it
 * (LBM_ERR_ARG if none runs it, or if a variant was requested with
 * lbm3_set_kernel and does not run it).  8 <= zc <= nz (or zc = nz when
 * nz < 8).  Every tiling gives the same values up to floating-point
 * contraction (see lbm_set_tiling).  n_ctas: CTAs per step. */
int lbm3_set_tiling(lbm3_handle* h, int32_t bx, int32_t by, int32_t zc);
int lbm3_get_tiling(const lbm3_handle* h, int32_t* bx, int32_t* by, int32_t* zc,
                    int32_t* n_ctas);

/* Step-kernel variant.  All variants run the same per-node arithmetic.
 *   0: automatic -- the register kernel until lbm3_autotune picks the
 *      fastest (on a tile the register kernel does not run, with the
 *      default tile (32, 8));
 *   1: register-pipelined loads (any precision; tiles of variants 1-3,
 *      others switch to (32, 8));
 *   2 / 3: asynchronous 4-byte copies (cp.async) through shared memory,
 *      2 / 3 stages deep (LBM3_F32 only; tiles (32, 4), (32, 8), (64, 4));
 *   4: bulk copies (cp.async.bulk) of whole x-rows into shared memory, one
 *      or two planes ahead (LBM3_F32 and LBM3_F16; nx <= 256, a row of nx
 *      stored values and of nx FP32 values a multiple of 16 bytes; tiles
 *      (128, 4) for nx <= 128, (256, 2); selecting it on another tile takes
 *      its own tile);
 *   5: bulk copies of padded row segments of a bx-column strip (one 16-byte
 *      chunk each side for the pull's shift and the halo column; split where
 *      they cross the periodic edge), two (FP32) or three (FP16) stages
 *      deep, two CTAs per SM (LBM3_F32 and LBM3_F16; nx a multiple of bx and
 *      nx >= 2 bx; tiles (32, 8), (64, 4); selecting it on another tile takes
 *      (64, 4) where nx allows, else (32, 8));
 *   6: the strip kernel of 5 with two stages and three (64, 4) or five
 *      (64, 2) CTAs per SM at fewer registers: more warps, less look-ahead
 *      (same precisions and box conditions; selecting it on another tile
 *      takes (64, 4)).
 * Other variants on a tile they do not run: LBM_ERR_ARG.  Every wait of
 * variants 4 to 6 is bounded: on expiry the step is abandoned and
 * lbm3_status reports LBM_ERR_TIMEOUT.  lbm3_get_kernel returns the variant
 * in use (1 to 6).  Errors: LBM_ERR_ARG (variant outside [0, 6], or not
 * available for this precision or box). */
int lbm3_set_kernel(lbm3_handle* h, int32_t variant);
int32_t lbm3_get_kernel(const lbm3_handle* h);

/* Bound of the device waits of the bulk-copy variants (4 to 6), in SM clock
 * cycles: the waits for their staged planes.  A wait that gives up makes
 * lbm3_status report LBM_ERR_TIMEOUT; the CTA first waits, with the default
 * bound, for the copies it issued, then returns, and the step's results are
 * not valid.  cycles < 0 restores the default, about 2 s (4e9 cycles); 0
 * gives up at the first poll that finds the data missing (used to test the
 * timeout path).  Variants 1-3 do not wait on data.  Errors: LBM_ERR_ARG. */
int lbm3_set_wait_limit(lbm3_handle* h, int64_t cycles);

/* Time every allowed (variant, bx, by) with a few zc choices (`trials`
 * launches each, CUDA events) and keep the fastest; with a variant set by
 * lbm3_set_kernel only that variant is tried.  Trial launches write only the
 * buffers the next step overwrites; the state and the step index do not
 * change.  Outputs may be NULL.  Synchronises. */
int lbm3_autotune(lbm3_handle* h, int32_t trials, int32_t* variant, int32_t* bx,
                  int32_t* by, int32_t* zc, double* best_ms);

/* Synchronise and report device error flags (LBM_OK, LBM_ERR_NONFINITE,
 * LBM_ERR_TIMEOUT, LBM_ERR_CUDA); clears them. */
int lbm3_status(lbm3_handle* h);

void lbm3_destroy(lbm3_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* LBM3_API_H */
