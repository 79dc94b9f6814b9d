// Kernels of the three-dimensional coupled step (D3Q19 flow + D3Q7 phase
// field, SRT limit of Eqs. 20-37), templated on the arithmetic type T and the
// population storage type S (S = T, or __half with T = float).
//
// step3_kernel: one CTA owns a BX x BY column tile and marches along z over
// `zc` planes.  For each plane it
//   A. pulls the 7 phase-field populations of the next plane (z+1) at every
//      tile node and at the one-node halo ring around the tile, forms
//      phi = sum g (Eq. 35) and psi (Eq. 37, phi clipped to [0,1]), and puts
//      the (phi, psi) pair into a 4-slot shared-memory ring of planes;
//   B. updates the nodes of plane z: pulls the 19 f populations, takes the
//      isotropic D3Q19 stencils (Sec. 3.2) of phi and psi from planes z-1, z,
//      z+1 of the ring, and runs both collisions; stores f*, g*, phi*u.
// The ring has 4 slots, so one barrier per plane separates A(z+1) from B(z)
// and B(z) from A(z+3).  The pulled g of the tile nodes stay in registers
// from A (as the next plane) to B.
//
// Phase volume in FP32 arithmetic: phi is conserved node by node only if the
// stored rest population is phi minus the stored movers.  A rounded FP32 g_0
// leaves an error of up to half an ulp of g_0 per node and step whose sign the
// slowly varying interface values repeat step after step, so the volume
// drifts.  Under FP32 arithmetic g_0 is therefore kept as a float pair
// (hi + lo) and advanced by the exact identity
//   g_0* = g_0 + lo + sum_{i>0} (g_i - g*_i)
// (pulled minus stored movers), the differences summed in plain FP32 (their
// rounding is 2^-24 of the collision change, not of g_0) and added to g_0 with
// an error-free TwoSum (Knuth, TAOCP vol. 2, 4.2.2).
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm3_layout.h"

namespace lbmk3 {

// ---- lattice ----------------------------------------------------------------
// Components of the 19 velocities in the order of lbm3_layout.h.
struct Lat {
  static constexpr int cx[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  static constexpr int cy[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  static constexpr int cz[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
};

// ---- precision helpers ------------------------------------------------------
template <typename T>
struct N3;
template <>
struct N3<float> {
  using pair = float2;
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  // psi up to a positive factor (only grad(psi)/|grad(psi)| is used)
  static __device__ __forceinline__ float lratio(float a, float b) {
    return __log2f(a) - __log2f(b);
  }
  static __device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }
};
template <>
struct N3<double> {
  using pair = double2;
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
  static __device__ __forceinline__ double lratio(double a, double b) { return log(a / b); }
  static __device__ __forceinline__ double clamp01(double v) { return fmin(fmax(v, 0.0), 1.0); }
};

template <typename T, typename S>
struct Conv {
  static __device__ __forceinline__ T ld(const S* p) { return *p; }
  static __device__ __forceinline__ S st(T v) { return v; }
  static __device__ __forceinline__ T round(T v) { return v; }
};
template <>
struct Conv<float, __half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ __half st(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float round(float v) {
    return __half2float(__float2half_rn(v));
  }
};

template <typename T>
__device__ __forceinline__ T psi3(T phi, T xi) {
  const T pc = N3<T>::clamp01(phi);
  return N3<T>::lratio(pc + xi, (T(1) - pc) + xi);
}

// Offsets of the source nodes of a pull: o[1 - c] is the offset along an axis
// of the node at coordinate - c (o[0]: minus one, o[1]: same, o[2]: plus one).
struct Offs {
  uint32_t x[3], y[3], z[3];
};

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void set_xy(Offs& o, int x, int y, int nx, int ny) {
  o.x[0] = (uint32_t)wrap1(x - 1, nx);
  o.x[1] = (uint32_t)x;
  o.x[2] = (uint32_t)wrap1(x + 1, nx);
  o.y[0] = (uint32_t)wrap1(y - 1, ny) * nx;
  o.y[1] = (uint32_t)y * nx;
  o.y[2] = (uint32_t)wrap1(y + 1, ny) * nx;
}

__device__ __forceinline__ void set_z(Offs& o, int z, int nz, uint32_t nxy) {
  o.z[0] = (uint32_t)wrap1(z - 1, nz) * nxy;
  o.z[1] = (uint32_t)z * nxy;
  o.z[2] = (uint32_t)wrap1(z + 1, nz) * nxy;
}

template <int I>
__device__ __forceinline__ uint32_t src_of(const Offs& o) {
  return o.z[1 - Lat::cz[I]] + o.y[1 - Lat::cy[I]] + o.x[1 - Lat::cx[I]];
}

// Pull the 7 phase-field populations of one node: g0 (and its low part) from
// its own position, the 6 movers from plane i-1 of gm at the source node.
template <typename T, typename S>
__device__ __forceinline__ void pull_g(const T* __restrict__ g0, const T* __restrict__ g0lo,
                                       const S* __restrict__ gm, int64_t P, const Offs& o,
                                       T (&G)[7], T& Glo) {
  G[0] = g0[src_of<0>(o)];
  Glo = g0lo ? g0lo[src_of<0>(o)] : T(0);
  G[1] = Conv<T, S>::ld(gm + 0 * P + src_of<1>(o));
  G[2] = Conv<T, S>::ld(gm + 1 * P + src_of<2>(o));
  G[3] = Conv<T, S>::ld(gm + 2 * P + src_of<3>(o));
  G[4] = Conv<T, S>::ld(gm + 3 * P + src_of<4>(o));
  G[5] = Conv<T, S>::ld(gm + 4 * P + src_of<5>(o));
  G[6] = Conv<T, S>::ld(gm + 5 * P + src_of<6>(o));
}

template <typename T>
__device__ __forceinline__ T sum7(const T (&G)[7]) {
  return ((G[0] + (G[1] + G[2])) + (G[3] + G[4])) + (G[5] + G[6]);
}

// Error-free sum: s + e == a + b exactly (TwoSum, no ordering condition).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// phi of one node from its pulled populations (plus the low part of g_0).
template <typename T>
__device__ __forceinline__ T phi_of(const T (&G)[7], T glo) {
  return sum7(G) + glo;
}

template <int I, typename T, typename S>
__device__ __forceinline__ void pull_f1(const S* __restrict__ f, int64_t P, const Offs& o,
                                        T (&F)[19]) {
  F[I] = Conv<T, S>::ld(f + I * P + src_of<I>(o));
}

template <typename T, typename S>
__device__ __forceinline__ void pull_f(const S* __restrict__ f, int64_t P, const Offs& o,
                                       T (&F)[19]) {
  pull_f1<0>(f, P, o, F);   pull_f1<1>(f, P, o, F);   pull_f1<2>(f, P, o, F);
  pull_f1<3>(f, P, o, F);   pull_f1<4>(f, P, o, F);   pull_f1<5>(f, P, o, F);
  pull_f1<6>(f, P, o, F);   pull_f1<7>(f, P, o, F);   pull_f1<8>(f, P, o, F);
  pull_f1<9>(f, P, o, F);   pull_f1<10>(f, P, o, F);  pull_f1<11>(f, P, o, F);
  pull_f1<12>(f, P, o, F);  pull_f1<13>(f, P, o, F);  pull_f1<14>(f, P, o, F);
  pull_f1<15>(f, P, o, F);  pull_f1<16>(f, P, o, F);  pull_f1<17>(f, P, o, F);
  pull_f1<18>(f, P, o, F);
}

// One population pair (c, -c) of the SRT collision with forcing (Eqs. 20-23
// with all rates 1/tau_f): f*_{+-} = f + w_f (f_eq - f) + h_f F_i, where
//   f_eq = w [3p + rho (4.5 (c.u)^2 - 1.5 u^2)] +- 3 w rho c.u
//   F_i  = 3 w (c.u)(c.grad rho)              +- 3 w c.F     (Eq. 21)
template <typename T>
__device__ __forceinline__ void pair_f(T& fp, T& fm, T w, T cu, T cF, T cR, T base, T rho,
                                       T wf, T hf) {
  const T sym = w * (base + rho * (T(4.5) * cu * cu));
  const T anti = (T(3) * w) * (rho * cu);
  const T Fs = (T(3) * w) * (cu * cR);
  const T Fa = (T(3) * w) * cF;
  fp = fp + wf * ((sym + anti) - fp) + hf * (Fs + Fa);
  fm = fm + wf * ((sym - anti) - fm) + hf * (Fs - Fa);
}

// Stencil values of one node: phi at the node and its 18 D3Q19 neighbours,
// psi at the 18 neighbours.  Naming: E/W = +-x, N/S = +-y, U/D = +-z.
template <typename T>
struct St3 {
  T C, E, W, N, S, NE, NW, SE, SW, U, UE, UW, UN, US, D, DE, DW, DN, DS;
};

template <typename T, int BX, int BY>
struct Ring3 {
  typename N3<T>::pair pq[4][BY + 2][BX + 2];
};

template <typename T, int BX, int BY>
__device__ __forceinline__ void read_st(const Ring3<T, BX, BY>& r, int sm, int s0, int sp, int j,
                                        int i, St3<T>& p, St3<T>& q) {
  const auto c = r.pq[s0][j][i], e = r.pq[s0][j][i + 1], w = r.pq[s0][j][i - 1];
  const auto n = r.pq[s0][j + 1][i], s = r.pq[s0][j - 1][i];
  const auto ne = r.pq[s0][j + 1][i + 1], nw = r.pq[s0][j + 1][i - 1];
  const auto se = r.pq[s0][j - 1][i + 1], sw = r.pq[s0][j - 1][i - 1];
  const auto u = r.pq[sp][j][i], ue = r.pq[sp][j][i + 1], uw = r.pq[sp][j][i - 1];
  const auto un = r.pq[sp][j + 1][i], us = r.pq[sp][j - 1][i];
  const auto d = r.pq[sm][j][i], de = r.pq[sm][j][i + 1], dw = r.pq[sm][j][i - 1];
  const auto dn = r.pq[sm][j + 1][i], ds = r.pq[sm][j - 1][i];
  p = St3<T>{c.x, e.x, w.x, n.x, s.x, ne.x, nw.x, se.x, sw.x, u.x, ue.x, uw.x, un.x, us.x,
             d.x, de.x, dw.x, dn.x, ds.x};
  q = St3<T>{c.y, e.y, w.y, n.y, s.y, ne.y, nw.y, se.y, sw.y, u.y, ue.y, uw.y, un.y, us.y,
             d.y, de.y, dw.y, dn.y, ds.y};
}

// 6 x the D3Q19 isotropic gradient: grad = (1/6) axis + (1/12) diagonal
// differences (weights 1/18, 1/36 over c_s^2 = 1/3), times 12.
template <typename T>
__device__ __forceinline__ void grad12(const St3<T>& s, T& gx, T& gy, T& gz) {
  gx = T(2) * (s.E - s.W) + (((s.NE + s.SE) + (s.UE + s.DE)) - ((s.NW + s.SW) + (s.UW + s.DW)));
  gy = T(2) * (s.N - s.S) + (((s.NE + s.NW) + (s.UN + s.DN)) - ((s.SE + s.SW) + (s.US + s.DS)));
  gz = T(2) * (s.U - s.D) + (((s.UE + s.UW) + (s.UN + s.US)) - ((s.DE + s.DW) + (s.DN + s.DS)));
}

// Macroscopic values and both collisions at one node; F, G hold the pulled
// populations on entry and the post-collision ones on exit (kModeStep).
template <typename T>
struct Out3 {
  T ux, uy, uz, p;
};

template <typename T, typename S, int MODE>
__device__ __forceinline__ Out3<T> node3(const Args3<T, S>& a, T (&F)[19], T (&G)[7], T& Glo,
                                         const T (&jp)[3], const St3<T>& P, const St3<T>& Q) {
  const T phi = P.C;
  T gpx, gpy, gpz;
  grad12(P, gpx, gpy, gpz);
  gpx *= T(1.0 / 12.0);
  gpy *= T(1.0 / 12.0);
  gpz *= T(1.0 / 12.0);
  // lap = (1/3) sum_axis (chi_n - chi) + (1/6) sum_diag (chi_n - chi)
  const T lap = T(1.0 / 3.0) * ((((P.E + P.W) + (P.N + P.S)) + (P.U + P.D)) - T(6) * phi) +
                T(1.0 / 6.0) * (((((P.NE + P.SW) + (P.SE + P.NW)) + ((P.UE + P.UW) + (P.UN + P.US))) +
                                  ((P.DE + P.DW) + (P.DN + P.DS))) -
                                 T(12) * phi);
  T qx, qy, qz;  // 12 grad(psi): only its direction is used
  grad12(Q, qx, qy, qz);

  // chemical potential (Eq. 2) and surface force F = hbar grad(phi)
  const T mu = a.beta4 * phi * (phi - T(1)) * (phi - T(0.5)) - a.kappa * lap;
  const T Fx = mu * gpx, Fy = mu * gpy, Fz = mu * gpz;

  const T rho = a.rho_g + phi * a.drho;
  const T irho = N3<T>::rcp(rho);
  // sum c f
  const T jx = ((F[1] - F[2]) + (F[7] - F[8])) + ((F[9] - F[10]) + ((F[11] - F[12]) + (F[13] - F[14])));
  const T jy = ((F[3] - F[4]) + (F[7] - F[8])) + (((F[15] - F[16]) + (F[17] - F[18])) - (F[9] - F[10]));
  const T jz = ((F[5] - F[6]) + (F[11] - F[12])) + (((F[15] - F[16]) - (F[13] - F[14])) - (F[17] - F[18]));
  Out3<T> o;
  o.ux = (jx + T(0.5) * Fx) * irho;  // Eq. 28
  o.uy = (jy + T(0.5) * Fy) * irho;
  o.uz = (jz + T(0.5) * Fz) * irho;
  const T ux = o.ux, uy = o.uy, uz = o.uz;
  const T Rx = a.drho * gpx, Ry = a.drho * gpy, Rz = a.drho * gpz;  // grad(rho)
  const T uR = (ux * Rx + uy * Ry) + uz * Rz;
  const T u2 = (ux * ux + uy * uy) + uz * uz;
  T snz = (((F[1] + F[2]) + (F[3] + F[4])) + ((F[5] + F[6]) + (F[7] + F[8]))) +
          (((F[9] + F[10]) + (F[11] + F[12])) + ((F[13] + F[14]) + (F[15] + F[16]))) +
          (F[17] + F[18]);
  // Eq. 29 on D3Q19: c_s^2/(1-w0) = 1/2, rho s_0(u) = -rho |u|^2/2
  o.p = T(0.5) * (snz + T(0.5) * uR - T(0.5) * rho * u2);
  if (MODE != kModeStep) return o;

  T wf = a.wf, hf = a.hf;
  if (a.var_tau) {
    const T tau = T(3) * (a.mu_g + phi * a.dmu) * irho + T(0.5);  // Eq. 27
    wf = N3<T>::rcp(tau);
    hf = T(1) - T(0.5) * wf;
  }
  const T p = o.p;
  const T base = T(3) * p - T(1.5) * rho * u2;
  // rest population: f_eq,0 = (w0 - 1) p / c_s^2 + rho s_0 = -2p - rho u^2/2; F_0 = 0
  F[0] = F[0] + wf * ((T(-2) * p - T(0.5) * rho * u2) - F[0]);
  const T w1 = T(1.0 / 18.0), w2 = T(1.0 / 36.0);
  pair_f(F[1], F[2], w1, ux, Fx, Rx, base, rho, wf, hf);
  pair_f(F[3], F[4], w1, uy, Fy, Ry, base, rho, wf, hf);
  pair_f(F[5], F[6], w1, uz, Fz, Rz, base, rho, wf, hf);
  pair_f(F[7], F[8], w2, ux + uy, Fx + Fy, Rx + Ry, base, rho, wf, hf);
  pair_f(F[9], F[10], w2, ux - uy, Fx - Fy, Rx - Ry, base, rho, wf, hf);
  pair_f(F[11], F[12], w2, ux + uz, Fx + Fz, Rx + Rz, base, rho, wf, hf);
  pair_f(F[13], F[14], w2, ux - uz, Fx - Fz, Rx - Rz, base, rho, wf, hf);
  pair_f(F[15], F[16], w2, uy + uz, Fy + Fz, Ry + Rz, base, rho, wf, hf);
  pair_f(F[17], F[18], w2, uy - uz, Fy - Fz, Ry - Rz, base, rho, wf, hf);

  // ---- phase field: SRT limit of Eq. 33 on D3Q7 (c_s^2 = 1/4) ----
  const T Jx = phi * ux, Jy = phi * uy, Jz = phi * uz;
  const T pc = N3<T>::clamp01(phi);
  const T ta = pc + a.xi, tb = (T(1) - pc) + a.xi;
  const T q2 = (qx * qx + qy * qy) + qz * qz;
  const T iq = (q2 >= a.qmin2) ? N3<T>::rsq(q2) : T(0);  // n := 0 on ridges of psi
  // (lambda/W)[1 - tanh^2(2 psi/W)] / |grad psi|, with 1 - tanh^2 = 4ab/(a+b)^2
  const T sh = a.lamW * a.tfac * ta * tb * iq;
  // c_s^2 x the braced vector of Eq. 32: d_t(phi u) + (sharpening) / 4
  const T Vx = (Jx - jp[0]) + T(0.25) * sh * qx;
  const T Vy = (Jy - jp[1]) + T(0.25) * sh * qy;
  const T Vz = (Jz - jp[2]) + T(0.25) * sh * qz;
  const T L8 = T(0.125) * (mu + a.lambda * phi);  // w_i (hbar + lambda phi)
  const T wg = a.wg, hg2 = T(0.5) * a.hg;         // G_i = w_i c.V / c_s^2 = (1/2) c.V
  T Gin[7];  // FP32: the pulled populations, for the rest population below
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < 7; ++i) Gin[i] = G[i];
  }
  // g_eq,+- = L8 +- (1/2) c.J (Eq. 31)
  G[1] = G[1] + wg * ((L8 + T(0.5) * Jx) - G[1]) + hg2 * Vx;
  G[2] = G[2] + wg * ((L8 - T(0.5) * Jx) - G[2]) - hg2 * Vx;
  G[3] = G[3] + wg * ((L8 + T(0.5) * Jy) - G[3]) + hg2 * Vy;
  G[4] = G[4] + wg * ((L8 - T(0.5) * Jy) - G[4]) - hg2 * Vy;
  G[5] = G[5] + wg * ((L8 + T(0.5) * Jz) - G[5]) + hg2 * Vz;
  G[6] = G[6] + wg * ((L8 - T(0.5) * Jz) - G[6]) - hg2 * Vz;
#pragma unroll
  for (int i = 1; i < 7; ++i) G[i] = Conv<T, S>::round(G[i]);
  // rest population from the conserved zeroth moment: sum g* = phi
  if constexpr (sizeof(T) == 8) {
    G[0] = phi - (((G[1] + G[2]) + (G[3] + G[4])) + (G[5] + G[6]));
    Glo = T(0);
  } else {
    const float d = (((float)Gin[1] - (float)G[1]) + ((float)Gin[2] - (float)G[2])) +
                    ((((float)Gin[3] - (float)G[3]) + ((float)Gin[4] - (float)G[4])) +
                     (((float)Gin[5] - (float)G[5]) + ((float)Gin[6] - (float)G[6])));
    float hi, lo;
    two_sum((float)Gin[0], (float)Glo + d, hi, lo);
    G[0] = (T)hi;
    Glo = (T)lo;
  }
  return o;
}

// ---- the step kernel --------------------------------------------------------
template <typename T, typename S, int BX, int BY, int MODE>
__global__ void __launch_bounds__(BX* BY) step3_kernel(
    const Args3<T, S> a, const T* __restrict__ g0s, const T* __restrict__ g0ls,
    const S* __restrict__ gms, const S* __restrict__ fs, const T* __restrict__ js,
    T* __restrict__ g0d, T* __restrict__ g0ld, S* __restrict__ gmd, S* __restrict__ fd,
    T* __restrict__ jd) {
  constexpr int NH = 2 * (BX + 2) + 2 * BY;  // halo ring of the tile
  static_assert(NH <= BX * BY, "tile too small for its halo");
  __shared__ Ring3<T, BX, BY> ring;
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
  const int64_t P = a.plane;
  const int gx = blockIdx.x * BX + tx, gy = blockIdx.y * BY + ty;
  const bool valid = gx < nx && gy < ny;
  Offs own, hal;
  set_xy(own, gx % nx, gy % ny, nx, ny);
  // halo slot of this thread (tile coordinates -1..BX, -1..BY)
  int hx = 0, hy = 0;
  const bool has_h = tid < NH;
  if (has_h) {
    if (tid < BX + 2) {
      hx = tid - 1, hy = -1;
    } else if (tid < 2 * (BX + 2)) {
      hx = tid - (BX + 2) - 1, hy = BY;
    } else if (tid < 2 * (BX + 2) + BY) {
      hx = -1, hy = tid - 2 * (BX + 2);
    } else {
      hx = BX, hy = tid - 2 * (BX + 2) - BY;
    }
    const int ax = (int)(((int64_t)blockIdx.x * BX + hx + nx) % nx);
    const int ay = (int)(((int64_t)blockIdx.y * BY + hy + ny) % ny);
    set_xy(hal, ax, ay, nx, ny);
  }
  const int zb = blockIdx.z * a.zc;
  const int ze = min(zb + a.zc, nz);

  // phase A for plane zl into ring slot s; own pulled g returned in G, Glo
  auto phaseA = [&](int zl, int s, T (&G)[7], T& Glo) {
    const int zw = zl < 0 ? zl + nz : (zl >= nz ? zl - nz : zl);
    set_z(own, zw, nz, nxy);
    pull_g(g0s, g0ls, gms, P, own, G, Glo);
    T H[7], Hlo;
    if (has_h) {
      set_z(hal, zw, nz, nxy);
      pull_g(g0s, g0ls, gms, P, hal, H, Hlo);
    }
    const T phi = phi_of(G, Glo);
    typename N3<T>::pair v;
    v.x = phi;
    v.y = psi3(phi, a.xi);
    ring.pq[s][ty + 1][tx + 1] = v;
    if (has_h) {
      const T phh = phi_of(H, Hlo);
      v.x = phh;
      v.y = psi3(phh, a.xi);
      ring.pq[s][hy + 1][hx + 1] = v;
    }
  };

  T Gc[7], Gn[7], Gcl, Gnl;
  phaseA(zb - 1, (zb + 3) & 3, Gn, Gnl);
  phaseA(zb, zb & 3, Gc, Gcl);
  double vsum = 0.0;
  for (int z = zb; z < ze; ++z) {
    // independent loads of this plane first
    Offs oz = own;
    set_z(oz, z, nz, nxy);
    T F[19], jp[3];
    const uint32_t node = oz.z[1] + oz.y[1] + oz.x[1];
    if (valid) {
      pull_f(fs, P, oz, F);
      jp[0] = js[node];
      jp[1] = js[P + node];
      jp[2] = js[2 * P + node];
    }
    phaseA(z + 1, (z + 1) & 3, Gn, Gnl);
    __syncthreads();
    if (valid) {
      St3<T> SP, SQ;
      read_st(ring, (z + 3) & 3, z & 3, (z + 1) & 3, ty + 1, tx + 1, SP, SQ);
      const Out3<T> o = node3<T, S, MODE>(a, F, Gc, Gcl, jp, SP, SQ);
      const T phi = SP.C;
      if (!(isfinite(phi) && isfinite(o.ux + o.uy + o.uz))) atomicOr(a.flags, kFlagNonFinite);
      if (MODE == kModeStep) {
        if (a.vol_part) vsum += (double)phi;
        jd[node] = phi * o.ux;
        jd[P + node] = phi * o.uy;
        jd[2 * P + node] = phi * o.uz;
        g0d[node] = Gc[0];
        if (g0ld) g0ld[node] = Gcl;
#pragma unroll
        for (int i = 1; i < 7; ++i) gmd[(i - 1) * P + node] = Conv<T, S>::st(Gc[i]);
#pragma unroll
        for (int i = 0; i < 19; ++i) fd[i * P + node] = Conv<T, S>::st(F[i]);
      } else {
        const T v = a.out_which == kOutPhi ? phi
                    : a.out_which == kOutUx ? o.ux
                    : a.out_which == kOutUy ? o.uy
                    : a.out_which == kOutUz ? o.uz
                                            : o.p;
        a.out[node] = (double)v;
      }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) Gc[i] = Gn[i];
    Gcl = Gnl;
  }
  if (MODE == kModeStep && a.vol_part) {
    // fixed-order block reduction of the phi this CTA collided
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vsum += __shfl_down_sync(0xffffffffu, vsum, off);
    __shared__ double wsum[BX * BY / 32];
    __syncthreads();
    if ((tid & 31) == 0) wsum[tid >> 5] = vsum;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < BX * BY / 32; ++w) s += wsum[w];
      a.vol_part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
  }
}

// ---- auxiliary kernels ------------------------------------------------------
// The velocity components again, for run-time indexing.
__device__ __constant__ static const int kC3x[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1,
                                                     -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ __constant__ static const int kC3y[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1,
                                                     1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ __constant__ static const int kC3z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0,
                                                     0, 1, -1, -1, 1, 1, -1, -1, 1};

__device__ __forceinline__ void node_xyz(int64_t k, int nx, int ny, int& x, int& y, int& z) {
  x = (int)(k % nx);
  const int64_t r = k / nx;
  y = (int)(r % ny);
  z = (int)(r / ny);
}

__device__ __forceinline__ int64_t pull_pos(int i, int x, int y, int z, int nx, int ny, int nz) {
  const int xs = wrap1(x - kC3x[i], nx), ys = wrap1(y - kC3y[i], ny);
  const int zs = wrap1(z - kC3z[i], nz);
  return ((int64_t)zs * ny + ys) * nx + xs;
}

// Initial state in FP64, rounded once (as the 2-D path): hbar0 from Eq. 2 with
// the D3Q19 Laplacian, g = g_eq(phi0, hbar0, u0) (Eq. 31, D3Q7),
// f = f_eq(p = 0, rho(phi0), u0) (Eq. 22, D3Q19), phi*u at t-1 = phi0 u0.
template <typename T, typename S>
__global__ void init3_kernel(Args3<T, S> a, double beta4, double kappa, double lambda,
                             double rho_g, double drho, const double* __restrict__ phi0,
                             const double* __restrict__ u0) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t n = (int64_t)nx * ny * nz, P = a.plane;
  const int par = a.parity;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(k, nx, ny, x, y, z);
    const double p = phi0[k];
    double sa = 0.0, sd = 0.0;
    for (int i = 1; i < 19; ++i) {
      const int64_t m = pull_pos(i, x, y, z, nx, ny, nz);  // node x - c_i
      (i < 7 ? sa : sd) += phi0[m] - p;
    }
    const double lap = sa / 3.0 + sd / 6.0;
    const double mu = beta4 * p * (p - 1.0) * (p - 0.5) - kappa * lap;
    double u[3] = {0.0, 0.0, 0.0};
    if (u0) u[0] = u0[k], u[1] = u0[n + k], u[2] = u0[2 * n + k];
    const double L = mu + lambda * p;
    const double rho = rho_g + p * drho;
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
      const double cu = kC3x[i] * u[0] + kC3y[i] * u[1] + kC3z[i] * u[2];
      const double w = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
      const double fe = rho * w * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
      // f at node x after streaming sits at x - c_i in the pull layout
      const int64_t dst = pull_pos(i, x, y, z, nx, ny, nz);
      a.f[par][i * P + dst] = Conv<T, S>::st((T)fe);
      if (i > 0 && i < 7) {
        const double ge = 0.125 * L + 0.5 * cu * p;  // w_i (L + c.J / c_s^2)
        a.g[par][(i - 1) * P + dst] = Conv<T, S>::st((T)ge);
      }
    }
    a.J[par][k] = (T)(p * u[0]);
    a.J[par][P + k] = (T)(p * u[1]);
    a.J[par][2 * P + k] = (T)(p * u[2]);
  }
}

// g0 after the movers are stored: g0 = phi0 - sum of the stored movers of the
// node (so that sum g = phi0 with the stored, possibly rounded, values).
template <typename T, typename S>
__global__ void init3_rest_kernel(Args3<T, S> a, const double* __restrict__ phi0) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t n = (int64_t)nx * ny * nz, P = a.plane;
  const S* gm = a.g[a.parity];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(k, nx, ny, x, y, z);
    double s = 0.0;
    for (int i = 1; i < 7; ++i)
      s += (double)Conv<T, S>::ld(gm + (i - 1) * P + pull_pos(i, x, y, z, nx, ny, nz));
    const double g0 = phi0[k] - s;
    const T hi = (T)g0;
    a.g0[a.parity][k] = hi;
    if (a.g0lo[a.parity]) a.g0lo[a.parity][k] = (T)(g0 - (double)hi);
  }
}

// Import/export of one population plane between the FP64 host layout (value
// at the node it is delivered to, after streaming) and the pull layout.
// kind: 0 = f plane i, 1 = g plane i (0: rest plane g0), 2 = phi*u component i.
template <typename T, typename S>
__global__ void plane3_kernel(Args3<T, S> a, int kind, int i, double* __restrict__ buf,
                              int to_device) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t n = (int64_t)nx * ny * nz, P = a.plane;
  const int par = a.parity;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(k, nx, ny, x, y, z);
    if (kind == 2) {
      T* p = a.J[par] + i * P + k;
      if (to_device) *p = (T)buf[k];
      else buf[k] = (double)*p;
      continue;
    }
    if (kind == 1 && i == 0) {  // g_0 = hi + lo
      T* lo = a.g0lo[par];
      if (to_device) {
        const T hi = (T)buf[k];
        a.g0[par][k] = hi;
        if (lo) lo[k] = (T)(buf[k] - (double)hi);
      } else {
        buf[k] = (double)a.g0[par][k] + (lo ? (double)lo[k] : 0.0);
      }
      continue;
    }
    const int64_t m = pull_pos(i, x, y, z, nx, ny, nz);
    S* p = kind == 0 ? a.f[par] + i * P + m : a.g[par] + (i - 1) * P + m;
    if (to_device) *p = Conv<T, S>::st((T)buf[k]);
    else buf[k] = (double)Conv<T, S>::ld(p);
  }
}

// Phase volumes per region (Eq. 35 summed in FP64): block b sums a contiguous
// chunk of nodes; part[b * 8 + r] receives region r.  Fixed order throughout.
template <typename T, typename S>
__global__ void __launch_bounds__(256) volume3_kernel(Args3<T, S> a,
                                                      const int8_t* __restrict__ labels,
                                                      int nregions, double* part) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t n = (int64_t)nx * ny * nz, P = a.plane;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = blockIdx.x * chunk, k1 = min(n, k0 + chunk);
  const S* gm = a.g[a.parity];
  double acc[kMaxRegions];
#pragma unroll
  for (int r = 0; r < kMaxRegions; ++r) acc[r] = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    int x, y, z;
    node_xyz(k, nx, ny, x, y, z);
    double phi = (double)a.g0[a.parity][k];
    if (a.g0lo[a.parity]) phi += (double)a.g0lo[a.parity][k];
    for (int i = 1; i < 7; ++i)
      phi += (double)Conv<T, S>::ld(gm + (i - 1) * P + pull_pos(i, x, y, z, nx, ny, nz));
    const int r = labels ? labels[k] : 0;
#pragma unroll
    for (int q = 0; q < kMaxRegions; ++q)
      if (q == r) acc[q] += phi;
  }
  __shared__ double red[kMaxRegions][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < nregions; ++q) {
    double v = acc[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nregions) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    part[blockIdx.x * kMaxRegions + threadIdx.x] = s;
  }
}

// Sum of nparts partial sums per region, fixed order, one warp per region.
static __global__ void volume3_final(const double* __restrict__ part, int nparts, int stride,
                                     int nregions, double* __restrict__ out) {
  const int r = blockIdx.x;
  if (r >= nregions) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += 32) s += part[(size_t)b * stride + r];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) out[r] = s;
}

}  // namespace lbmk3
