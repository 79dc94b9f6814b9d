// Device-side data layout of the three-dimensional step (D3Q19 flow, D3Q7
// phase field): the single-relaxation-time limit of Eqs. 20-37 (Sec. 3.1:
// equal MRT rates reduce the model to SRT) on the textbook 3-D lattices.
//
// Populations are structure-of-arrays planes of n = nx*ny*nz nodes, [z][y][x]
// with x fastest; plane i of a buffer holds the post-collision value f*_i at
// every node, so that the pull step reads f_i(x, t+1) = f*_i(x - c_i, t).  Two
// buffers (parity 0/1) alternate between source and destination.
#pragma once
#include <cstdint>

#include "lbm_layout.h"

namespace lbmk3 {

using lbmk::kNormalMin;  // threshold of the interface normal, as in 2-D

constexpr int kQF = 19;  // D3Q19 (hydrodynamics)
constexpr int kQG = 7;   // D3Q7 (phase field)
constexpr int kMaxRegions = 8;

// Velocity order (both lattices share the first 7 vectors):
//  0 (0,0,0)  1 (1,0,0)  2 (-1,0,0)  3 (0,1,0)  4 (0,-1,0)  5 (0,0,1)  6 (0,0,-1)
//  7 (1,1,0)  8 (-1,-1,0)  9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
// 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
// Weights: D3Q19 1/3, 1/18, 1/36 (c_s^2 = 1/3); D3Q7 1/4, 1/8 (c_s^2 = 1/4).

enum { kModeStep = 0, kModeFields = 1 };
enum { kFlagNonFinite = 1, kFlagTimeout3 = 2 };  // device error flags (bits)
enum { kOutPhi = 0, kOutUx = 1, kOutUy = 2, kOutUz = 3, kOutP = 4 };

// Launch arguments.  T is the arithmetic type, S the storage type.
template <typename T, typename S>
struct Args3 {
  S* f[2];          // 19 planes per buffer
  S* g[2];          // the 6 moving phase-field populations (i = 1..6 -> plane i-1)
  T* g0[2];         // the rest population g_0, kept in the arithmetic type
  T* g0lo[2];       // FP32 arithmetic: low part of g_0 (g_0 = g0 + g0lo, a float
                    // pair), so that sum g = phi holds to ~2^-48; null in FP64
  T* J[2];          // phi*u of the previous step, 3 planes per buffer
  int64_t plane;    // elements per plane (n rounded up)
  int32_t nx, ny, nz, zc;  // grid; planes per CTA along z
  int32_t parity;          // source buffer
  int32_t var_tau;         // 1: tau_f varies with phi (Eq. 27 per node)
  T beta4, kappa, lambda;  // 4 beta (beta = 12 sigma/W), kappa = 3 sigma W/2
  T lamW, xi, tfac;        // lambda/W, xi, 4/(1+2 xi)^2
  T qmin2;                 // |12 grad(psi_k)|^2 at |grad(psi)| = kNormalMin
  T wg, hg;                // 1/tau_g, 1 - 1/(2 tau_g)
  T wf, hf;                // uniform tau_f: 1/tau_f, 1 - 1/(2 tau_f)
  T rho_g, drho, mu_g, dmu;  // rho(phi) = rho_g + phi drho, mu(phi) likewise
  int32_t* flags;          // device error flags (kFlag*)
  double* vol_part;        // kModeStep: per-CTA FP64 sum of phi, or null
  double* out;             // kModeFields: FP64 field [z][y][x]
  int32_t out_which;       // kOut*
  long long wait;          // bound of the bulk-copy kernels' waits, SM cycles (0: one poll)
};

}  // namespace lbmk3
