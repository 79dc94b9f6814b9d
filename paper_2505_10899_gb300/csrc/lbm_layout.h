// Device-side data layout shared by the host runtime (lbm_api.cu) and the
// kernels.  One "case" is one periodic nx x ny grid; a batch holds several.
//
// Populations are structure-of-arrays planes: plane i of a buffer holds the
// post-collision value f*_i at every node, [y][x] with x fastest, so that the
// pull step of Eqs. 20/30 reads f_i(x, t+1) = f*_i(x - c_i, t) from plane i.
// Two buffers (parity 0/1) alternate between source and destination.
#pragma once
#include <cstdint>

namespace lbmk {

constexpr int kQ = 9;
constexpr int kMaxRegions = 8;

template <typename T>
struct CaseDev {
  T* f[2];               // hydrodynamic populations, 9 planes per buffer
  T* g[2];               // phase-field populations, 9 planes per buffer
  T* J[2];               // phi*u of the previous step, 2 planes per buffer
  T* g0lo[2];            // FP32: low part of the rest population, g_0 = g[0] + g0lo
                         // (a float pair formed exactly, see node_update); null in FP64
  const int8_t* labels;  // volume regions, [y][x]; nullptr = one region
  int64_t plane;         // elements per plane (nx*ny rounded up)
  int32_t nx, ny;
  T rho_g, drho;         // rho(phi) = rho_g + phi*drho
  T mu_g, dmu;           // mu(phi)  = mu_g + phi*dmu
  T sD7, hD7;            // uniform tau_f: -s7/4 and (1 - s7/2)/4 (s8 = s7)
  int32_t var_tau;       // 1: tau_f varies with phi (Eq. 27 per node)
  int32_t nregions;      // volume regions of this case
  int32_t vol_base;      // first output slot of this case's volumes
  int32_t item_begin, item_end;  // work items of this case
  int32_t walls;         // 1: moving walls below row 0 and above row ny-1
  int32_t pad_;
  T u_top, u_bot;        // wall velocities along x
};

// Launch-uniform physics, converted to the working precision T.
// Moment-space rates are folded with the inverse row norms
// D = diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) of Eq. 24:
//   sD[k] = -s_k D_k,  hD[k] = (1 - s_k/2) D_k.
// Interface normal of Eq. 17: n = grad(psi)/|grad(psi)| where |grad(psi)| >=
// kNormalMin, else 0 (psi of Eq. 14 in lattice units).  psi is a signed
// distance, |grad(psi)| = 1 on the equilibrium profile; it falls below
// kNormalMin only on ridges of psi (the centre of a droplet, the axis of a
// thread, the mid-plane of a neck: points no nearer to one part of the
// interface than to another) and in the clipped bulk.  There a unit vector
// would take its direction from rounding, and a small |grad(psi)| would
// amplify any perturbation by 1/|grad(psi)|.
constexpr double kNormalMin = 0.1;

// Default bound of the device waits: ~2 s at 2 GHz.
constexpr long long kWaitCycles = 4000000000LL;

template <typename T>
struct Phys {
  T beta4;   // 4 beta, beta = 12 sigma / W
  T kappa;   // 3 sigma W / 2
  T lambda;
  T lamW;    // lambda / W
  T xi;
  T tfac;    // 4 / (1 + 2 xi)^2 : 1 - tanh^2(2 psi / W) = tfac * a * b
  T qmin2;   // |12 grad(psi_k)|^2 at |grad(psi)| = kNormalMin (psi_k: the kernel's psi)
  T fsD[kQ], fhD[kQ];
  T gsD[kQ], ghD3[kQ];  // ghD3 = ghD / 3 (the source moments carry a 1/3)
  double vU, vT;        // prescribed vortex amplitude and period
};

struct Item {
  int32_t c, x0, y0, nrows;  // case, first column, first row, rows
};

// Initial fields of one case as the init kernel reads them: device
// pointers to [ny][nx] FP64 phi0 and [2][ny][nx] u0 (u0 may be null: at
// rest), either in the workspace (staged copies) or in host memory that the
// device reads directly (page-locked memory, over the CPU-GPU link); and
// rho(phi) = rho_g + phi drho in FP64.
struct InitSrc {
  const double* phi;
  const double* u;
  double rho_g, drho;
};


enum { kModeStep = 0, kModeFields = 1 };
enum { kFlagNonFinite = 1, kFlagTimeout = 2 };

template <typename T>
struct StepArgs {
  Phys<T> ph;
  const CaseDev<T>* cases;
  const Item* items;
  const int64_t* t_base;  // device step counter
  int64_t t_off;          // this launch is step t_base + t_off
  int32_t parity;         // source buffer index
  int32_t pad_;
  int32_t* flags;         // device error flags (kFlag*)
  // bound of every wait on data or on other CTAs, in SM clock cycles (the
  // TMA kernel's waits for its staged rows, the persistent kernel's grid
  // barrier); on expiry the kernel raises kFlagTimeout and returns
  long long wait_cycles;
  // kModeStep: if non-null, each CTA writes the FP64 sum of the phi it
  // collided (the pre-collision phi of Eq. 35) to vol_part[blockIdx.x * 8]
  double* vol_part;
  // kModeFields outputs (FP64, [y][x]) for the items of one case
  double* out_phi;
  double* out_ux;
  double* out_uy;
  double* out_p;
};

}  // namespace lbmk
