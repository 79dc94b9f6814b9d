// Per-node arithmetic of the coupled volume-conserving LB step (arXiv
// 2505.10899, Secs. 3.1-3.2), shared by both step kernels and templated on
// the working precision T (float or double).
//
// The collisions run in moment space (Eqs. 25 and 33) without matrix
// products: the moments of f, g are formed with add/sub butterflies of the
// rows of M (Eq. 24); the equilibrium and source moments M f_eq, M F, M g_eq,
// M G are their closed forms (from Eqs. 21-23, 31-32 and the D2Q9 lattice
// sums); M^-1 = M^T D is applied as the transposed butterfly.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_check.h"
#include "lbm_layout.h"

namespace lbmk {

template <typename T>
struct Num;

template <>
struct Num<float> {
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
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

template <typename T>
__device__ __forceinline__ T sum9(const T v[9]) {
  return (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
}

// Error-free sum s + e == a + b (TwoSum, Knuth, TAOCP vol. 2, 4.2.2).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Rest population under FP32 arithmetic.  The populations of a node must
// sum to the phi that entered it, or the phase volume drifts: a rounded FP32
// g_0 = phi - sum(movers*) leaves an error of up to half an ulp of g_0 per node
// and step, and slowly varying interface values repeat its sign step after
// step.  So g_0 is kept as a float pair (g_0 + lo) and advanced by the exact
// identity  g_0* = g_0 + lo + sum_{i>0} (g_i - g*_i),  where g_i are the pulled
// and g*_i the stored post-collision movers: the 8 differences are summed in
// plain FP32 (their rounding is 2^-24 of the collision change, not of g_0) and
// added to g_0 with an error-free TwoSum, the low part kept.
__device__ __forceinline__ void rest_pair(const float Gin[9], float lo, const float G[9],
                                          float& g0, float& glo) {
  const float d = ((Gin[1] - G[1]) + (Gin[2] - G[2])) + ((Gin[3] - G[3]) + (Gin[4] - G[4])) +
                  (((Gin[5] - G[5]) + (Gin[6] - G[6])) + ((Gin[7] - G[7]) + (Gin[8] - G[8])));
  two_sum_f(Gin[0], lo + d, g0, glo);
}

// psi of Eq. 37 (up to the factor W/4 and the log base), phi clipped to [0,1].
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

// (phi, psi) pair of one node, read with one vector load.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

// Shared-memory ring of (phi, psi): 4 rows x (BX + 2) columns; column 0 and
// BX+1 (or wact+1) hold the halo columns left and right of the strip.
template <typename T, int BX>
struct Ring {
  typename Pair<T>::type pq[4][BX + 2];
  __device__ __forceinline__ void put(int s, int c, T phi, T psi) {
    typename Pair<T>::type v;
    v.x = phi;
    v.y = psi;
    pq[s][c] = v;
  }
};

// phi at the node and its 8 neighbours, psi at the 8 neighbours.
template <typename T>
struct Stencil {
  T p, pE, pW, pN, pS, pNE, pNW, pSE, pSW;
  T qE, qW, qN, qS, qNE, qNW, qSE, qSW;
};

// Stencil of local row k, local column lc (1-based) from the ring.
template <typename T, int BX>
__device__ __forceinline__ Stencil<T> read_stencil(const Ring<T, BX>& ring, int k, int lc) {
  const int sm = (k + 3) & 3, s0 = k & 3, sp = (k + 1) & 3;
  Stencil<T> S;
  const auto c = ring.pq[s0][lc], e = ring.pq[s0][lc + 1], w = ring.pq[s0][lc - 1];
  const auto n = ring.pq[sp][lc], ne = ring.pq[sp][lc + 1], nw = ring.pq[sp][lc - 1];
  const auto so = ring.pq[sm][lc], se = ring.pq[sm][lc + 1], sw = ring.pq[sm][lc - 1];
  S.p = c.x;
  S.pE = e.x;
  S.pW = w.x;
  S.pN = n.x;
  S.pS = so.x;
  S.pNE = ne.x;
  S.pNW = nw.x;
  S.pSE = se.x;
  S.pSW = sw.x;
  S.qE = e.y;
  S.qW = w.y;
  S.qN = n.y;
  S.qS = so.y;
  S.qNE = ne.y;
  S.qNW = nw.y;
  S.qSE = se.y;
  S.qSW = sw.y;
  return S;
}

// Constants of the case a CTA works on (per thread where noted).
template <typename T>
struct CaseK {
  T rho_g, drho, mu_g, dmu, sD7, hD7;
  bool var_tau;
  int ny;
  T ct;        // vortex: U cos(pi t / T)
  T sx2, s2x;  // vortex: sin^2(pi X), sin(2 pi X) of this thread's column
};

template <typename T, bool COUPLED>
__device__ __forceinline__ CaseK<T> case_consts(const StepArgs<T>& a, const CaseDev<T>* cdp,
                                                int xc) {
  CaseK<T> K;
  K.rho_g = cdp->rho_g;
  K.drho = cdp->drho;
  K.mu_g = cdp->mu_g;
  K.dmu = cdp->dmu;
  K.sD7 = cdp->sD7;
  K.hD7 = cdp->hD7;
  K.var_tau = cdp->var_tau != 0;
  K.ny = cdp->ny;
  K.ct = T(0);
  K.sx2 = T(0);
  K.s2x = T(0);
  if (!COUPLED) {
    const double t = (double)(*a.t_base + a.t_off);
    K.ct = (T)(cospi(t / a.ph.vT) * a.ph.vU);
    T s, c;
    Num<T>::sincospi_((T(xc) + T(0.5)) / T(cdp->nx), &s, &c);
    K.sx2 = s * s;
    K.s2x = T(2) * s * c;
  }
  return K;
}

// Macroscopic values and both collisions at one node.  Fc, Gc hold the pulled
// populations on entry and the post-collision populations on exit
// (kModeStep).  jpx, jpy = phi*u of the previous step.  Returns phi, u, p.
template <typename T>
struct NodeOut {
  T ux, uy, p, Jx, Jy;
};

template <typename T, bool COUPLED, int MODE>
__device__ __forceinline__ NodeOut<T> node_update(const Phys<T>& ph, const CaseK<T>& K,
                                                  T (&Fc)[9], T (&Gc)[9], T& Glo, T jpx,
                                                  T jpy, const Stencil<T>& S, int y) {
  const T phi = S.p;
  // isotropic stencils (Sec. 3.2): grad = (1/3) axis + (1/12) diagonal
  // differences; lap = (2/3) axis + (1/6) diagonal second differences
  const T gpx = T(1.0 / 3.0) * (S.pE - S.pW) + T(1.0 / 12.0) * ((S.pNE - S.pNW) + (S.pSE - S.pSW));
  const T gpy = T(1.0 / 3.0) * (S.pN - S.pS) + T(1.0 / 12.0) * ((S.pNE - S.pSE) + (S.pNW - S.pSW));
  const T lap = T(2.0 / 3.0) * (((S.pE + S.pW) + (S.pN + S.pS)) - T(4) * phi) +
                T(1.0 / 6.0) * (((S.pNE + S.pNW) + (S.pSE + S.pSW)) - T(4) * phi);
  // 12 grad(psi): only its direction is used
  const T qx = T(4) * (S.qE - S.qW) + ((S.qNE - S.qNW) + (S.qSE - S.qSW));
  const T qy = T(4) * (S.qN - S.qS) + ((S.qNE - S.qSE) + (S.qNW - S.qSW));

  // chemical potential, Eq. 2, and surface force F = hbar grad(phi) (Eq. 18)
  const T mu = ph.beta4 * phi * (phi - T(1)) * (phi - T(0.5)) - ph.kappa * lap;
  const T Fx = mu * gpx, Fy = mu * gpy;

  NodeOut<T> o;
  o.p = T(0);
  if (COUPLED) {
    const T rho = K.rho_g + phi * K.drho;  // linear rho(phi)
    const T irho = Num<T>::rcp(rho);
    const Mom<T> mf = moments(Fc);
    // Eq. 28: rho u = sum c f + F/2
    o.ux = (mf.m3 + T(0.5) * Fx) * irho;
    o.uy = (mf.m5 + T(0.5) * Fy) * irho;
    const T ux = o.ux, uy = o.uy;
    const T Rx = K.drho * gpx, Ry = K.drho * gpy;  // grad(rho)
    const T uR = ux * Rx + uy * Ry;
    const T u2 = ux * ux + uy * uy;
    // Eq. 29: p = c_s^2/(1-w0) [sum_{i!=0} f_i + u.grad(rho)/2 + rho s_0(u)],
    // s_0(u) = -w0 |u|^2/(2 c_s^2) = -(2/3)|u|^2
    o.p = T(0.6) * ((mf.m0 - Fc[0]) + T(0.5) * uR - T(2.0 / 3.0) * rho * u2);
    if (MODE == kModeStep) {
      // equilibrium moments M f_eq (Eqs. 22-23):
      //   (0, 6p + 3 rho u^2, -9p - 3 rho u^2, rho ux, -rho ux, rho uy,
      //    -rho uy, rho (ux^2 - uy^2), rho ux uy)
      // forcing moments M F (Eq. 21):
      //   (u.R, 0, -u.R, Fx, -Fx, Fy, -Fy, (2/3)(ux Rx - uy Ry), (ux Ry + uy Rx)/3)
      const T p = o.p;
      const T ru2 = rho * u2;
      const T jx = rho * ux, jy = rho * uy;
      T sD7 = K.sD7, hD7 = K.hD7;
      if (K.var_tau) {
        const T mu_v = K.mu_g + phi * K.dmu;
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
    Num<T>::sincospi_((T(y) + T(0.5)) / T(K.ny), &sy, &cy);
    o.ux = -K.ct * K.sx2 * (T(2) * sy * cy);
    o.uy = K.ct * (sy * sy) * K.s2x;
  }

  o.Jx = phi * o.ux;
  o.Jy = phi * o.uy;
  if (MODE == kModeStep) {
    // ---- phase-field collision, Eqs. 31-33 ----
    const T Jx = o.Jx, Jy = o.Jy;
    const T dJx = Jx - jpx, dJy = Jy - jpy;  // backward difference for d_t(phi u)
    const T pc = Num<T>::clamp01(phi);
    const T ta = pc + ph.xi, tb = (T(1) - pc) + ph.xi;
    const T q2 = qx * qx + qy * qy;
    const T iq = (q2 >= ph.qmin2) ? Num<T>::rsq(q2) : T(0);  // n := 0 on ridges of psi
    // (lambda/W) [1 - tanh^2(2psi/W)] / |grad psi|, tanh via Eqs. 13-15
    const T sh = ph.lamW * ph.tfac * ta * tb * iq;
    const T Vx = T(3) * dJx + sh * qx;  // d_t(phi u)/c_s^2 + sharpening flux
    const T Vy = T(3) * dJy + sh * qy;
    const T Lam = mu + ph.lambda * phi;
    const Mom<T> mg = moments(Gc);
    T Gin[9];  // FP32: the pulled populations, for the rest population below
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int i = 0; i < 9; ++i) Gin[i] = Gc[i];
    }
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
    if constexpr (sizeof(T) == 4) {
      rest_pair(Gin, Glo, Gc, Gc[0], Glo);
    } else {
      Gc[0] = phi - (((Gc[1] + Gc[2]) + (Gc[3] + Gc[4])) + ((Gc[5] + Gc[6]) + (Gc[7] + Gc[8])));
    }
  }
  return o;
}

// Store the post-collision state of one node (pull layout: own position).
template <typename T, bool COUPLED>
__device__ __forceinline__ void store_node(T* __restrict__ fd, T* __restrict__ gd,
                                           T* __restrict__ Jd, T* __restrict__ lod, uint32_t P,
                                           uint32_t node, const T (&Fc)[9], const T (&Gc)[9],
                                           T Glo, const NodeOut<T>& o, int32_t* flags,
                                           uint32_t nn) {
#ifdef LBM_CHECK_BOUNDS
  if (!LBM_BOUND(flags, node, nn)) return;
#else
  (void)flags;
  (void)nn;
#endif
  if (sizeof(T) == 4) lod[node] = Glo;
  Jd[node] = o.Jx;
  Jd[P + node] = o.Jy;
#pragma unroll
  for (int i = 0; i < 9; ++i) gd[i * P + node] = Gc[i];
  if (COUPLED) {
#pragma unroll
    for (int i = 0; i < 9; ++i) fd[i * P + node] = Fc[i];
  }
}

}  // namespace lbmk
