// Device code of the coupled volume-conserving LB step (arXiv 2505.10899,
// Secs. 3.1-3.2), templated on the working precision T (float or double).
//
// One CTA owns a strip of BX columns and marches down `nrows` rows of it
// (a work item).  Per row it pulls the 18 populations of its nodes
// (Eqs. 20 and 30, left-hand sides), forms phi = sum g (Eq. 35) and the
// level-set variable psi (Eq. 37), keeps phi and psi of the last four rows
// in a shared-memory ring with a one-column halo on each side, and collides
// row k once rows k-1, k, k+1 are in the ring.  Loads of row k+2 are issued
// before the collision of row k so that their latency overlaps the
// arithmetic (two-row software pipeline, one __syncthreads per row).
//
// The collisions run in moment space (Eqs. 25 and 33) without matrix
// products: the moments of f, g are formed with add/sub butterflies of the
// rows of M (Eq. 24); the equilibrium and source moments M f_eq, M F, M g_eq,
// M G are their closed forms (derived from Eqs. 21-23, 31-32 with the D2Q9
// lattice sums); M^-1 = M^T D is applied as the transposed butterfly.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_layout.h"

namespace lbmk {

template <typename T>
struct Num;

template <>
struct Num<float> {
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
  // psi up to a positive constant factor: only grad(psi)/|grad(psi)| is used
  static __device__ __forceinline__ float lratio(float a, float b) {
    return __log2f(a) - __log2f(b);
  }
  static __device__ __forceinline__ float clamp01(float v) {
    return fminf(fmaxf(v, 0.0f), 1.0f);
  }
  static __device__ __forceinline__ void sincospi_(float v, float* s, float* c) {
    sincospif(v, s, c);
  }
};

template <>
struct Num<double> {
  static __device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double lratio(double a, double b) {
    return log(a / b);
  }
  static __device__ __forceinline__ double clamp01(double v) {
    return fmin(fmax(v, 0.0), 1.0);
  }
  static __device__ __forceinline__ void sincospi_(double v, double* s, double* c) {
    sincospi(v, s, c);
  }
};

// Pull the 9 populations of node (x, row) from a buffer: value i comes from
// (x - c_ix, row - c_iy).  o0/om/op are the offsets of rows row, row-1,
// row+1 (periodic), xm/xp the columns x-1, x+1 (periodic).  Eq. 19 order:
// c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
template <typename T>
__device__ __forceinline__ void pull9(const T* __restrict__ b, int64_t P,
                                      int64_t o0, int64_t om, int64_t op,
                                      int x, int xm, int xp, T v[9]) {
  v[0] = __ldg(b + o0 + x);
  v[1] = __ldg(b + P + o0 + xm);
  v[2] = __ldg(b + 2 * P + om + x);
  v[3] = __ldg(b + 3 * P + o0 + xp);
  v[4] = __ldg(b + 4 * P + op + x);
  v[5] = __ldg(b + 5 * P + om + xm);
  v[6] = __ldg(b + 6 * P + om + xp);
  v[7] = __ldg(b + 7 * P + op + xp);
  v[8] = __ldg(b + 8 * P + op + xm);
}

template <typename T>
__device__ __forceinline__ T sum9(const T v[9]) {
  return (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
}

// psi of Eq. 37 (scaled by 4/W and a constant), phi clipped to [0,1].
template <typename T>
__device__ __forceinline__ T psi_of(T phi, T xi) {
  const T pc = Num<T>::clamp01(phi);
  return Num<T>::lratio(pc + xi, (T(1) - pc) + xi);
}

// Forward moments m = M v (rows of Eq. 24) by butterflies.
template <typename T>
struct Mom {
  T m0, m1, m2, m3, m4, m5, m6, m7, m8;
};

template <typename T>
__device__ __forceinline__ Mom<T> moments(const T v[9]) {
  Mom<T> m;
  const T sa = (v[1] + v[3]) + (v[2] + v[4]);
  const T sd = (v[5] + v[7]) + (v[6] + v[8]);
  m.m0 = v[0] + sa + sd;
  m.m1 = T(2) * sd - sa - T(4) * v[0];
  m.m2 = T(4) * v[0] - T(2) * sa + sd;
  const T ax = v[1] - v[3];
  const T dx = (v[5] - v[7]) + (v[8] - v[6]);
  m.m3 = ax + dx;
  m.m4 = dx - T(2) * ax;
  const T ay = v[2] - v[4];
  const T dy = (v[5] - v[7]) + (v[6] - v[8]);
  m.m5 = ay + dy;
  m.m6 = dy - T(2) * ay;
  m.m7 = (v[1] + v[3]) - (v[2] + v[4]);
  m.m8 = (v[5] + v[7]) - (v[6] + v[8]);
  return m;
}

// v_i += (M^T d)_i for i = 0..8 (d already carries the factor D of M^-1).
template <typename T>
__device__ __forceinline__ void add_back(T v[9], T d0, T d1, T d2, T d3, T d4,
                                         T d5, T d6, T d7, T d8) {
  const T A = d0 - d1 - T(2) * d2;
  const T B = d0 + T(2) * d1 + d2;
  const T X = d3 - T(2) * d4, Y = d5 - T(2) * d6;
  const T Xd = d3 + d4, Yd = d5 + d6;
  v[0] += d0 - T(4) * d1 + T(4) * d2;
  v[1] += (A + X) + d7;
  v[3] += (A - X) + d7;
  v[2] += (A + Y) - d7;
  v[4] += (A - Y) - d7;
  v[5] += (B + Xd) + (Yd + d8);
  v[7] += (B - Xd) - (Yd - d8);
  v[6] += (B - Xd) + (Yd - d8);
  v[8] += (B + Xd) - (Yd + d8);
}

// Shared-memory ring of phi and psi: 4 rows x (BX + 2) columns.
template <typename T, int BX>
struct Ring {
  T phi[4][BX + 2];
  T psi[4][BX + 2];
};

// Prescribed single-vortex velocity (Eqs. 43-44, sign of the flow mode doc).
template <typename T>
struct VortexCol {
  T sx2, s2x;  // sin^2(pi X), sin(2 pi X) of this thread's column
};

// ---------------------------------------------------------------------------
// The fused step kernel.
//   COUPLED: f and g (true) or g only with the prescribed vortex (false).
//   MODE:    kModeStep collides and stores; kModeFields writes phi, u, p.
// ---------------------------------------------------------------------------
template <typename T, int BX, bool COUPLED, int MODE>
__global__ void __launch_bounds__(BX) step_kernel(const StepArgs<T> a) {
  __shared__ Ring<T, BX> ring;
  __shared__ double vred[BX / 32];

  const Item it = a.items[blockIdx.x];
  const CaseDev<T>* __restrict__ cdp = a.cases + it.c;
  const int nx = cdp->nx, ny = cdp->ny;
  const int64_t P = cdp->plane;
  const int x0 = it.x0, y0 = it.y0, nrows = it.nrows;
  const int tid = threadIdx.x;
  const int wact = min(BX, nx - x0);
  const bool act = tid < wact;
  const int xc = act ? x0 + tid : x0;
  const int xm = (xc == 0) ? nx - 1 : xc - 1;
  const int xp = (xc == nx - 1) ? 0 : xc + 1;

  const T* __restrict__ gs = cdp->g[a.parity];
  T* __restrict__ gd = cdp->g[a.parity ^ 1];
  const T* __restrict__ fs = COUPLED ? cdp->f[a.parity] : nullptr;
  T* __restrict__ fd = COUPLED ? cdp->f[a.parity ^ 1] : nullptr;
  T* __restrict__ Jb = cdp->J;

  // Halo columns: thread 0 serves the column left of the strip, thread BX-1
  // the column right of the last active one.
  const bool hthr = (tid == 0) || (tid == BX - 1);
  int hc = 0, hslot = 0;
  if (tid == 0) {
    hc = (x0 == 0) ? nx - 1 : x0 - 1;
    hslot = 0;
  } else if (tid == BX - 1) {
    hc = x0 + wact;
    if (hc >= nx) hc -= nx;
    hslot = wact + 1;
  }
  const int hcm = (hc == 0) ? nx - 1 : hc - 1;
  const int hcp = (hc == nx - 1) ? 0 : hc + 1;

  const Phys<T>& ph = a.ph;
  const T xi = ph.xi;
  // fused phase volume of the case (one region: the whole grid)
  const bool do_vol = (MODE == kModeStep) && (a.vol_part != nullptr);
  double vacc = 0.0;

  // case constants
  const T rho_g = cdp->rho_g, drho = cdp->drho;
  const T mu_g = cdp->mu_g, dmu = cdp->dmu;
  const T sD7c = cdp->sD7, hD7c = cdp->hD7;
  const bool var_tau = cdp->var_tau != 0;

  // time (vortex mode)
  T ct = T(0);
  VortexCol<T> vc{T(0), T(0)};
  if (!COUPLED) {
    const double t = (double)(*a.t_base + a.t_off);
    ct = (T)cospi(t / ph.vT) * (T)ph.vU;
    T s, c;
    Num<T>::sincospi_((T(xc) + T(0.5)) / T(nx), &s, &c);
    vc.sx2 = s * s;
    vc.s2x = T(2) * s * c;  // sin(2 pi X)
  }

  auto rowoff = [&](int r) -> int64_t { return (int64_t)r * nx; };
  auto wrap = [&](int r) -> int {
    r %= ny;
    return r < 0 ? r + ny : r;
  };

  // --- register sets of the pipeline: rows k (cur), k+1 (nxt), k+2 (nn) ---
  T Fc[9], Gc[9], Fn[9], Gn[9], Fq[9], Gq[9];
  T hq[9];  // halo-column g of the row being fetched

  auto fetch_full = [&](int r, T F[9], T G[9]) {
    const int rr = wrap(r);
    const int64_t o0 = rowoff(rr), om = rowoff(rr == 0 ? ny - 1 : rr - 1),
                  op = rowoff(rr == ny - 1 ? 0 : rr + 1);
    pull9(gs, P, o0, om, op, xc, xm, xp, G);
    if (COUPLED) pull9(fs, P, o0, om, op, xc, xm, xp, F);
  };
  auto fetch_g = [&](int r, T G[9]) {
    const int rr = wrap(r);
    const int64_t o0 = rowoff(rr), om = rowoff(rr == 0 ? ny - 1 : rr - 1),
                  op = rowoff(rr == ny - 1 ? 0 : rr + 1);
    pull9(gs, P, o0, om, op, xc, xm, xp, G);
  };
  auto fetch_halo = [&](int r, T H[9]) {
    const int rr = wrap(r);
    const int64_t o0 = rowoff(rr), om = rowoff(rr == 0 ? ny - 1 : rr - 1),
                  op = rowoff(rr == ny - 1 ? 0 : rr + 1);
    pull9(gs, P, o0, om, op, hc, hcm, hcp, H);
  };
  // write phi/psi of local row k (k >= -1) into the ring
  auto put_row = [&](int k, const T G[9], const T H[9]) {
    const int s = (k + 4) & 3;
    if (act) {
      const T phi = sum9(G);
      ring.phi[s][tid + 1] = phi;
      ring.psi[s][tid + 1] = psi_of(phi, xi);
    }
    if (hthr) {
      const T phi = sum9(H);
      ring.phi[s][hslot] = phi;
      ring.psi[s][hslot] = psi_of(phi, xi);
    }
  };

  // --- prologue: rows -1 (phi only), 0 and 1 -------------------------------
  {
    T Gm[9];
    fetch_g(y0 - 1, Gm);
    if (hthr) fetch_halo(y0 - 1, hq);
    put_row(-1, Gm, hq);
  }
  fetch_full(y0, Fc, Gc);
  if (hthr) fetch_halo(y0, hq);
  put_row(0, Gc, hq);
  if (nrows > 1) {
    fetch_full(y0 + 1, Fn, Gn);
  } else {
    fetch_g(y0 + 1, Gn);
  }
  if (hthr) fetch_halo(y0 + 1, hq);
  put_row(1, Gn, hq);
  __syncthreads();

  // One pipeline stage: collide local row k from (Fc, Gc) while the loads of
  // row k+2 land in (Fq, Gq).  Called three times per trip with the register
  // sets rotated, so no copies are needed between rows.
  auto stage = [&](int k, T(&Fc)[9], T(&Gc)[9], T(&Fq)[9], T(&Gq)[9]) {
    // issue loads of row k+2 (full if it is an own row, phi-only if it is
    // the halo row below the item, nothing beyond)
    const bool q_full = (k + 2 < nrows);
    const bool q_any = (k + 2 <= nrows);
    if (q_full) {
      fetch_full(y0 + k + 2, Fq, Gq);
    } else if (q_any) {
      fetch_g(y0 + k + 2, Gq);
    }
    if (q_any && hthr) fetch_halo(y0 + k + 2, hq);

    // ---------------- collide row k ----------------
    if (act) {
      const int y = wrap(y0 + k);
      const int lc = tid + 1;
      const int sm = (k + 3) & 3, s0 = k & 3, sp = (k + 1) & 3;
      const T phi = ring.phi[s0][lc];  // = sum of Gc (Eq. 35)
      if (do_vol) vacc += (double)phi;
      const T pE = ring.phi[s0][lc + 1], pW = ring.phi[s0][lc - 1];
      const T pN = ring.phi[sp][lc], pS = ring.phi[sm][lc];
      const T pNE = ring.phi[sp][lc + 1], pNW = ring.phi[sp][lc - 1];
      const T pSE = ring.phi[sm][lc + 1], pSW = ring.phi[sm][lc - 1];
      const T qE = ring.psi[s0][lc + 1], qW = ring.psi[s0][lc - 1];
      const T qN = ring.psi[sp][lc], qS = ring.psi[sm][lc];
      const T qNE = ring.psi[sp][lc + 1], qNW = ring.psi[sp][lc - 1];
      const T qSE = ring.psi[sm][lc + 1], qSW = ring.psi[sm][lc - 1];

      // isotropic stencils (Sec. 3.2): grad = (1/3) axis + (1/12) diagonal
      // differences; lap = (2/3) axis + (1/6) diagonal second differences
      const T gpx = T(1.0 / 3.0) * (pE - pW) + T(1.0 / 12.0) * ((pNE - pNW) + (pSE - pSW));
      const T gpy = T(1.0 / 3.0) * (pN - pS) + T(1.0 / 12.0) * ((pNE - pSE) + (pNW - pSW));
      const T lap = T(2.0 / 3.0) * (((pE + pW) + (pN + pS)) - T(4) * phi) +
                    T(1.0 / 6.0) * (((pNE + pNW) + (pSE + pSW)) - T(4) * phi);
      // 12 grad(psi) (direction only)
      const T qx = T(4) * (qE - qW) + ((qNE - qNW) + (qSE - qSW));
      const T qy = T(4) * (qN - qS) + ((qNE - qSE) + (qNW - qSW));

      // chemical potential, Eq. 2, and surface force F = hbar grad(phi)
      const T mu = ph.beta4 * phi * (phi - T(1)) * (phi - T(0.5)) - ph.kappa * lap;
      const T Fx = mu * gpx, Fy = mu * gpy;

      T ux, uy, p = T(0);
      Mom<T> mf;
      T rho = T(1), irho = T(1);
      if (COUPLED) {
        rho = rho_g + phi * drho;  // linear rho(phi)
        irho = Num<T>::rcp(rho);
        mf = moments(Fc);
        // Eq. 28: rho u = sum c f + F/2
        ux = (mf.m3 + T(0.5) * Fx) * irho;
        uy = (mf.m5 + T(0.5) * Fy) * irho;
        const T Rx = drho * gpx, Ry = drho * gpy;  // grad(rho)
        const T uR = ux * Rx + uy * Ry;
        const T u2 = ux * ux + uy * uy;
        // Eq. 29: p = c_s^2/(1-w0) [sum_{i!=0} f_i + u.grad(rho)/2 + rho s_0(u)],
        // s_0(u) = -w0 |u|^2/(2 c_s^2) = -(2/3)|u|^2
        p = T(0.6) * ((mf.m0 - Fc[0]) + T(0.5) * uR - T(2.0 / 3.0) * rho * u2);
        if (MODE == kModeStep) {
          // equilibrium moments M f_eq (Eqs. 22-23):
          //   (0, 6p + 3 rho u^2, -9p - 3 rho u^2, rho ux, -rho ux, rho uy,
          //    -rho uy, rho (ux^2 - uy^2), rho ux uy)
          // forcing moments M F (Eq. 21):
          //   (u.R, 0, -u.R, Fx, -Fx, Fy, -Fy, (2/3)(ux Rx - uy Ry), (ux Ry + uy Rx)/3)
          const T ru2 = rho * u2;
          const T jx = rho * ux, jy = rho * uy;
          T sD7 = sD7c, hD7 = hD7c;
          if (var_tau) {
            const T mu_v = mu_g + phi * dmu;
            const T tau = T(3) * mu_v * irho + T(0.5);  // Eq. 27
            const T s7 = Num<T>::rcp(tau);
            sD7 = T(-0.25) * s7;
            hD7 = T(0.25) - T(0.125) * s7;
          }
          const T d0 = ph.fsD[0] * mf.m0 + ph.fhD[0] * uR;
          const T d1 = ph.fsD[1] * (mf.m1 - (T(6) * p + T(3) * ru2));
          const T d2 = ph.fsD[2] * (mf.m2 + (T(9) * p + T(3) * ru2)) - ph.fhD[2] * uR;
          const T d3 = ph.fsD[3] * (mf.m3 - jx) + ph.fhD[3] * Fx;
          const T d4 = ph.fsD[4] * (mf.m4 + jx) - ph.fhD[4] * Fx;
          const T d5 = ph.fsD[5] * (mf.m5 - jy) + ph.fhD[5] * Fy;
          const T d6 = ph.fsD[6] * (mf.m6 + jy) - ph.fhD[6] * Fy;
          const T d7 = sD7 * (mf.m7 - rho * (ux * ux - uy * uy)) +
                       hD7 * (T(2.0 / 3.0) * (ux * Rx - uy * Ry));
          const T d8 = sD7 * (mf.m8 - jx * uy) + hD7 * (T(1.0 / 3.0) * (ux * Ry + uy * Rx));
          add_back(Fc, d0, d1, d2, d3, d4, d5, d6, d7, d8);
        }
      } else {
        T sy, cy;
        Num<T>::sincospi_((T(y) + T(0.5)) / T(ny), &sy, &cy);
        ux = -ct * vc.sx2 * (T(2) * sy * cy);
        uy = ct * (sy * sy) * vc.s2x;
      }

      const int64_t node = (int64_t)y * nx + xc;
      if (MODE == kModeStep) {
        // ---- phase-field collision, Eqs. 31-33 ----
        const T Jx = phi * ux, Jy = phi * uy;
        const T dJx = Jx - Jb[node], dJy = Jy - Jb[P + node];  // backward difference
        const T pc = Num<T>::clamp01(phi);
        const T ta = pc + xi, tb = (T(1) - pc) + xi;
        const T q2 = qx * qx + qy * qy;
        const T iq = (q2 > T(0)) ? Num<T>::rsq(q2) : T(0);
        // (lambda/W) [1 - tanh^2(2psi/W)] / |grad psi|, tanh via Eqs. 13-15
        const T sh = ph.lamW * ph.tfac * ta * tb * iq;
        const T Vx = T(3) * dJx + sh * qx;  // d_t(phi u)/c_s^2 + sharpening flux
        const T Vy = T(3) * dJy + sh * qy;
        const T Lam = mu + ph.lambda * phi;
        const Mom<T> mg = moments(Gc);
        // M g_eq = (phi, 2Lam - 4phi, 4phi - 3Lam, Jx, -Jx, Jy, -Jy, 0, 0);
        // M G    = (0, 0, 0, Vx/3, -Vx/3, Vy/3, -Vy/3, 0, 0)
        const T e1 = ph.gsD[1] * (mg.m1 - (T(2) * Lam - T(4) * phi));
        const T e2 = ph.gsD[2] * (mg.m2 - (T(4) * phi - T(3) * Lam));
        const T e3 = ph.gsD[3] * (mg.m3 - Jx) + ph.ghD3[3] * Vx;
        const T e4 = ph.gsD[4] * (mg.m4 + Jx) - ph.ghD3[4] * Vx;
        const T e5 = ph.gsD[5] * (mg.m5 - Jy) + ph.ghD3[5] * Vy;
        const T e6 = ph.gsD[6] * (mg.m6 + Jy) - ph.ghD3[6] * Vy;
        const T e7 = ph.gsD[7] * mg.m7;
        const T e8 = ph.gsD[8] * mg.m8;
        add_back(Gc, T(0), e1, e2, e3, e4, e5, e6, e7, e8);
        // rest population from the conserved zeroth moment: sum g* = phi
        Gc[0] = phi - (((Gc[1] + Gc[2]) + (Gc[3] + Gc[4])) + ((Gc[5] + Gc[6]) + (Gc[7] + Gc[8])));

        Jb[node] = Jx;
        Jb[P + node] = Jy;
#pragma unroll
        for (int i = 0; i < 9; ++i) gd[i * P + node] = Gc[i];
        if (COUPLED) {
#pragma unroll
          for (int i = 0; i < 9; ++i) fd[i * P + node] = Fc[i];
        }
        const T chk = phi + ux + uy + p;
        if (!isfinite(chk)) atomicOr(a.flags, kFlagNonFinite);
      } else {
        a.out_phi[node] = (double)phi;
        a.out_ux[node] = (double)ux;
        a.out_uy[node] = (double)uy;
        a.out_p[node] = (double)p;
      }
    }

    if (q_any) put_row(k + 2, Gq, hq);
    __syncthreads();
  };

  for (int k = 0; k < nrows; k += 3) {
    stage(k, Fc, Gc, Fq, Gq);
    if (k + 1 < nrows) stage(k + 1, Fn, Gn, Fc, Gc);
    if (k + 2 < nrows) stage(k + 2, Fq, Gq, Fn, Gn);
  }

  if (do_vol) {  // deterministic CTA reduction: warp shuffles, then warps in order
    for (int o = 16; o > 0; o >>= 1) vacc += __shfl_down_sync(0xffffffffu, vacc, o);
    if ((tid & 31) == 0) vred[tid >> 5] = vacc;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int w = 0; w < BX / 32; ++w) v += vred[w];
      a.vol_part[(int64_t)blockIdx.x * kMaxRegions] = v;
    }
  }
}

}  // namespace lbmk
