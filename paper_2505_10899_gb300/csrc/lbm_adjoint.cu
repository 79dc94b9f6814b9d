// Reverse mode of the coupled step: vector-Jacobian products of one time step
// and of the initial-state map, hand-written for the per-node arithmetic of
// lbm_node.cuh (FP64, single-case handles).
//
// State S_t = the three source buffers of the pull layout: post-collision
// populations f*, g* (9 planes each, value i of node x at position x) and
// phi*u (2 planes).  One step maps S_t to S_{t+1}; lbm_adjoint_step maps an
// adjoint lambda_{t+1} (same layout, FP64, 20 planes of nx*ny) to lambda_t and
// accumulates the parameter gradients.  The sweep runs in three kernels:
//   ad_phase:  phi = sum of pulled g (Eq. 35) and psi (Eq. 37) of S_t;
//   ad_node:   at every node, recompute the collision, then apply its
//              transposed Jacobian to the output adjoints: the adjoints of the
//              node's pulled inputs go to their source positions (the
//              transpose of the pull), the adjoints of the 9 phi and 8 psi
//              stencil values go to scratch;
//   ad_gather: every node sums the stencil adjoints that refer to its phi and
//              psi, and adds the total to the adjoints of its 9 pulled g.
// The clip of Eq. 37 and the normalisation of grad(psi) use the derivative
// of the branch taken (0 outside (0,1), and 0 where |grad psi| falls below the
// cut of the normal, 0.1).
// Walls (bounce-back rows, moving-wall term, mirrored ghost rows) are
// transposed as well: the bounce-back keeps the pull a bijection between
// buffer positions and (node, direction), and the mirrored ghost rows add
// the uses of a wall row's phi and psi by the wall row itself.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "lbm_handle.h"
#include "lbm_node.cuh"

namespace lbmk {
int set_last_error(int code, const char* msg);
}  // namespace lbmk

using lbmk::CaseDev;
using lbmk::Mom;
using lbmk::Phys;

namespace {

constexpr int kAdThreads = 256;
constexpr int kAdBlocks = 152 * 8;
// raw partials: beta4, kappa, lambda, tau_g (via s3,s5), tau_f (via s7,s8),
// u_wall_top, u_wall_bottom
constexpr int kNParam = 7;

// D2Q9 (Eq. 19): components, weights and opposite directions as
// compile-time functions of i (constants once the loops over i unroll; a
// __constant__ table would cost a load per use).
__host__ __device__ constexpr int kAX(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int kAY(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr double kAW(int i) {
  return i == 0 ? 4.0 / 9 : (i < 5 ? 1.0 / 9 : 1.0 / 36);
}
__host__ __device__ constexpr int kAOPP(int i) {
  return i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : (i - 5 + 2) % 4 + 5);
}
static_assert(kAOPP(1) == 3 && kAOPP(2) == 4 && kAOPP(3) == 1 && kAOPP(4) == 2 &&
                  kAOPP(5) == 7 && kAOPP(6) == 8 && kAOPP(7) == 5 && kAOPP(8) == 6,
              "opposite directions");
static_assert(kAX(5) == 1 && kAY(5) == 1 && kAX(6) == -1 && kAY(6) == 1 && kAX(7) == -1 &&
                  kAY(7) == -1 && kAX(8) == 1 && kAY(8) == -1,
              "diagonal directions");

int fail(int code, const std::string& m) { return lbmk::set_last_error(code, m.c_str()); }

// In-plane offsets are 32-bit: a case has at most 2.3e8 nodes.
__device__ __forceinline__ int shift(int x, int y, int dx, int dy, int nx, int ny) {
  x += dx;
  y += dy;
  x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
  return y * nx + x;
}

// Buffer position of the value population i delivers to node (x, y): the
// pull source, or with walls the node's own opposite population for a
// population that would come from beyond a wall (halfway bounce-back).
__device__ __forceinline__ int ad_src(int i, int x, int y, int nx, int ny, int walls,
                                          int* pl) {
  const int ys = y - kAY(i);
  if (walls && (ys < 0 || ys >= ny)) {
    *pl = kAOPP(i);
    return y * nx + x;
  }
  *pl = i;
  return shift(x, y, -kAX(i), -kAY(i), nx, ny);
}

// Stencil neighbour (x + dx, y + dy): periodic, or with walls the mirrored
// ghost row beyond a wall row.
__device__ __forceinline__ int ad_nb(int x, int y, int dx, int dy, int nx, int ny,
                                         int walls) {
  if (!walls) return shift(x, y, dx, dy, nx, ny);
  x += dx;
  x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  y += dy;
  y = y < 0 ? 0 : (y >= ny ? ny - 1 : y);
  return y * nx + x;
}

// Adjoint of phi (lP, [9][n]) and psi (lQ, [8][n]) stencil uses gathered at
// node (x, y): the nodes s whose stencil entry j reads this node.  Without
// walls s = (x, y) - c_j; with walls also the wall row's own uses of its
// mirrored ghost row.
template <typename R>
__device__ __forceinline__ void gather_uses(const R* __restrict__ lP, const R* __restrict__ lQ,
                                            int x, int y, int nx, int ny, int walls, R& sp,
                                            R& sq) {
  const int64_t n = (int64_t)nx * ny;
  #pragma unroll
  for (int j = 1; j < 9; ++j) {
    const int ys = y - kAY(j);
    if (!walls || (ys >= 0 && ys < ny)) {
      const int s = shift(x, y, -kAX(j), -kAY(j), nx, ny);
      sp += lP[j * n + s];
      if (lQ) sq += lQ[(j - 1) * n + s];
    }
    // a wall row reads its own row through the ghost row beyond the wall
    if (walls && ((y == 0 && kAY(j) == -1) || (y == ny - 1 && kAY(j) == 1))) {
      int xs = x - kAX(j);
      xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
      const int s = y * nx + xs;
      sp += lP[j * n + s];
      if (lQ) sq += lQ[(j - 1) * n + s];
    }
  }
}

template <typename R>
struct AdArgs {
  const R* fA;  // f* source buffer (9 planes, stride P), null in vortex mode
  const R* gA;  // g* source buffer
  const R* JA;  // phi*u source buffer (2 planes)
  int64_t P;    // plane stride of the state buffers
  int nx, ny;
  const R* phi;  // [n] scratch
  const R* psi;  // [n] scratch
  const R* ain;  // [20][n] adjoint of S_{t+1}
  R* aout;       // [20][n] adjoint of S_t
  R* lP;         // [9][n] scratch: adjoint of phi(x + c_j) used at node x
  R* lQ;         // [8][n] scratch: adjoint of psi(x + c_j), j = 1..8
  double* part;  // [gridDim][kNParam]
  Phys<R> ph;
  R rho_g, drho, mu_g, dmu, sD7, hD7, s7;
  int var_tau, coupled;
  R ct;    // vortex: U cos(pi t / T)
  R invW;  // 1/W: d(lambda/W)/d(lambda)
  int walls;
  R u_top, u_bot;
};

// d psi / d phi inside the clip for the forward's psi: ln(a/b) in FP64,
// log2(a/b) in FP32 (the FP32 kernels take psi up to the factor 1/ln 2,
// which the normal of Eq. 17 does not see).
template <typename R>
__device__ __forceinline__ R dpsi_dphi(R p, R xi) {
  const R d = R(1) / (p + xi) + R(1) / ((R(1) - p) + xi);
  return sizeof(R) == 4 ? R(1.4426950408889634) * d : d;
}

// phi (Eq. 35, pulled sum in the forward order) and psi (Eq. 37).
template <typename R>
__global__ void ad_phase(const R* __restrict__ gA, int64_t P, int nx, int ny, int walls, R xi,
                         R* __restrict__ phi, R* __restrict__ psi) {
  const int64_t n = (int64_t)nx * ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)n; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    R G[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      int pl;
      const int pos = ad_src(i, x, y, nx, ny, walls, &pl);
      G[i] = gA[pl * P + pos];
    }
    const R p = lbmk::sum9(G);
    phi[k] = p;
    psi[k] = lbmk::psi_of(p, xi);
  }
}

// Deterministic CTA reduction of the parameter partials (FP64), added to the
// CTA's own slots: a CTA covers the same nodes in every launch (grid-stride
// order over a fixed grid), so the slots accumulate over the adjoint steps in
// a fixed order without atomics, and one final sum over the CTAs (at
// take_grads) gives the same bits on every run.
template <typename A>
__device__ __forceinline__ void ad_block_partials(double (&red)[kAdThreads / 32][kNParam],
                                                  const A (&gacc)[kNParam],
                                                  double* __restrict__ part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < kNParam; ++q) {
    A v = gacc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < kNParam) {
    double v = 0.0;
    for (int w = 0; w < kAdThreads / 32; ++w) v += red[w][threadIdx.x];
    part[(int64_t)blockIdx.x * kNParam + threadIdx.x] += v;
  }
}

// The per-node reverse sweep.  R is the arithmetic and storage type of the
// states and adjoints (the handle's precision); the parameter partials are
// summed per thread and per warp in R and accumulated in FP64 above that.
template <typename R>
__global__ void __launch_bounds__(kAdThreads, sizeof(R) == 4 ? 3 : 1) ad_node(const AdArgs<R> a) {
  __shared__ double red[kAdThreads / 32][kNParam];
  using N = lbmk::Num<R>;
  const int nx = a.nx, ny = a.ny;
  const int64_t n = (int64_t)nx * ny, P = a.P;
  const Phys<R>& ph = a.ph;
  // Parameter terms: each thread sums its nodes' terms and each warp its
  // threads' sums in R; the warp sums enter the FP64 block and CTA partials.
  // Under FP32 a 32-term FP32 partial adds rounding of the order of the
  // terms' own FP32 arithmetic, and keeps the work off GB300's narrow FP64
  // pipe (FP64 conversions and a double shuffle tree per node took two
  // thirds of its cycles in this kernel).
  R gacc[kNParam] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)n; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    int src[9];
    int spl[9];
    R F[9], G[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      src[i] = ad_src(i, x, y, nx, ny, a.walls, &spl[i]);
      G[i] = a.gA[spl[i] * P + src[i]];
      F[i] = a.coupled ? a.fA[spl[i] * P + src[i]] : R(0);
    }
    const R jpx = a.JA[k], jpy = a.JA[P + k];
    R Pv[9], Qv[9];
    #pragma unroll
    for (int j = 0; j < 9; ++j) {
      const int s = ad_nb(x, y, kAX(j), kAY(j), nx, ny, a.walls);
      Pv[j] = a.phi[s];
      Qv[j] = a.psi[s];
    }
    // moving-wall term of the bounced f (rho of this node)
    const bool wbot = a.walls && y == 0, wtop = a.walls && y == ny - 1;
    if (a.coupled && (wbot || wtop)) {
      const R rw = a.rho_g + Pv[0] * a.drho;
      if (wbot) {  // as the forward step forms it
        const R d = rw * a.u_bot * R(1.0 / 6.0);
        F[5] += d;
        F[6] -= d;
      }
      if (wtop) {
        const R d = rw * a.u_top * R(1.0 / 6.0);
        F[7] -= d;
        F[8] += d;
      }
    }
    // ---------------- forward recompute (as node_update) ----------------
    const R phi = Pv[0];
    const R gpx = R(1.0 / 3.0) * (Pv[1] - Pv[3]) + R(1.0 / 12.0) * ((Pv[5] - Pv[6]) + (Pv[8] - Pv[7]));
    const R gpy = R(1.0 / 3.0) * (Pv[2] - Pv[4]) + R(1.0 / 12.0) * ((Pv[5] - Pv[8]) + (Pv[6] - Pv[7]));
    const R lap = R(2.0 / 3.0) * (((Pv[1] + Pv[3]) + (Pv[2] + Pv[4])) - R(4) * phi) +
                  R(1.0 / 6.0) * (((Pv[5] + Pv[6]) + (Pv[8] + Pv[7])) - R(4) * phi);
    const R qx = R(4) * (Qv[1] - Qv[3]) + ((Qv[5] - Qv[6]) + (Qv[8] - Qv[7]));
    const R qy = R(4) * (Qv[2] - Qv[4]) + ((Qv[5] - Qv[8]) + (Qv[6] - Qv[7]));
    const R poly = phi * (phi - R(1)) * (phi - R(0.5));
    const R mu = ph.beta4 * poly - ph.kappa * lap;
    const R Fx = mu * gpx, Fy = mu * gpy;
    R ux, uy;
    R rho = R(1), irho = R(1), Rx = R(0), Ry = R(0), u2 = R(0), mu_v = R(0), s7 = a.s7;
    R sD7 = a.sD7, hD7 = a.hD7;
    Mom<R> mf{};
    if (a.coupled) {
      rho = a.rho_g + phi * a.drho;
      irho = N::rcp(rho);  // the reciprocal the forward step takes
      mf = lbmk::moments(F);
      ux = (mf.m3 + R(0.5) * Fx) * irho;
      uy = (mf.m5 + R(0.5) * Fy) * irho;
      Rx = a.drho * gpx;
      Ry = a.drho * gpy;
      u2 = ux * ux + uy * uy;
      if (a.var_tau) {
        mu_v = a.mu_g + phi * a.dmu;
        const R tau = R(3) * mu_v * irho + R(0.5);
        s7 = N::rcp(tau);
        sD7 = R(-0.25) * s7;
        hD7 = R(0.25) - R(0.125) * s7;
      }
    } else {
      R sx, cx, sy, cy;
      N::sincospi_((R(x) + R(0.5)) / R(nx), &sx, &cx);
      N::sincospi_((R(y) + R(0.5)) / R(ny), &sy, &cy);
      ux = -a.ct * (sx * sx) * (R(2) * sy * cy);
      uy = a.ct * (sy * sy) * (R(2) * sx * cx);
    }
    const R Jx = phi * ux, Jy = phi * uy;
    const R dJx = Jx - jpx, dJy = Jy - jpy;
    const R pc = N::clamp01(phi);
    const R ta = pc + ph.xi, tb = (R(1) - pc) + ph.xi;
    const R q2 = qx * qx + qy * qy;
    const R iq = (q2 >= ph.qmin2) ? N::rsq(q2) : R(0);
    const R sh = ph.lamW * ph.tfac * ta * tb * iq;
    const R Vx = R(3) * dJx + sh * qx, Vy = R(3) * dJy + sh * qy;
    const Mom<R> mg = lbmk::moments(G);

    // ---------------- reverse ----------------
    R aF[9], aG[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      aF[i] = a.ain[i * n + k];
      aG[i] = a.ain[(9 + i) * n + k];
    }
    const R aJx = a.ain[18 * n + k], aJy = a.ain[19 * n + k];

    R lphi = R(0), lmu = R(0), lgpx = R(0), lgpy = R(0), llap = R(0), lqx = R(0), lqy = R(0);
    R lux = R(0), luy = R(0);
    // g*_0 = phi - sum_{i>=1} g*'_i; g*' = G + M^T e (e0 = 0)
    lphi += aG[0];
    R aGp[9];
    aGp[0] = R(0);
    #pragma unroll
    for (int i = 1; i < 9; ++i) aGp[i] = aG[i] - aG[0];
    R lG[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) lG[i] = aGp[i];
    const Mom<R> le = lbmk::moments(aGp);  // lambda_e = M lambda_g*'
    R lmg[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R lLam = R(0), lJx = R(0), lJy = R(0), lVx = R(0), lVy = R(0);
    // e1, e2
    lmg[1] += ph.gsD[1] * le.m1;
    lLam += R(-2) * ph.gsD[1] * le.m1;
    lphi += R(4) * ph.gsD[1] * le.m1;
    lmg[2] += ph.gsD[2] * le.m2;
    lphi += R(-4) * ph.gsD[2] * le.m2;
    lLam += R(3) * ph.gsD[2] * le.m2;
    // e3..e6
    lmg[3] += ph.gsD[3] * le.m3;
    lJx += -ph.gsD[3] * le.m3;
    lVx += ph.ghD3[3] * le.m3;
    lmg[4] += ph.gsD[4] * le.m4;
    lJx += ph.gsD[4] * le.m4;
    lVx += -ph.ghD3[4] * le.m4;
    lmg[5] += ph.gsD[5] * le.m5;
    lJy += -ph.gsD[5] * le.m5;
    lVy += ph.ghD3[5] * le.m5;
    lmg[6] += ph.gsD[6] * le.m6;
    lJy += ph.gsD[6] * le.m6;
    lVy += -ph.ghD3[6] * le.m6;
    lmg[7] += ph.gsD[7] * le.m7;
    lmg[8] += ph.gsD[8] * le.m8;
    {  // tau_g: s3 = s5 = 1/tau_g; gsD = -s/6, ghD3 = (1 - s/2)/18
      const R lgs = (mg.m3 - Jx) * le.m3 + (mg.m5 - Jy) * le.m5;
      const R lgh = Vx * le.m3 + Vy * le.m5;
      const R ls = -lgs * R(1.0 / 6.0) - lgh * R(1.0 / 36.0);
      const R sg = R(-6) * ph.gsD[3];  // = 1/tau_g
      gacc[3] += -sg * sg * ls;
    }
    // mg = M G
    lbmk::add_back(lG, lmg[0], lmg[1], lmg[2], lmg[3], lmg[4], lmg[5], lmg[6], lmg[7], lmg[8]);
    // Lam = mu + lambda phi
    lmu += lLam;
    lphi += ph.lambda * lLam;
    gacc[2] += phi * lLam;
    // V = 3 dJ + sh q
    const R ldJx = R(3) * lVx, ldJy = R(3) * lVy;
    const R lsh = qx * lVx + qy * lVy;
    lqx += sh * lVx;
    lqy += sh * lVy;
    // sh = lamW tfac ta tb iq
    const R c0 = ph.lamW * ph.tfac;
    const R lta = c0 * tb * iq * lsh, ltb = c0 * ta * iq * lsh, liq = c0 * ta * tb * lsh;
    gacc[2] += ph.tfac * ta * tb * iq * lsh * a.invW;  // lamW = lambda / W
    if (q2 >= ph.qmin2) {  // below the threshold n = 0: no derivative
      const R lq2 = R(-0.5) * iq * iq * iq * liq;
      lqx += R(2) * qx * lq2;
      lqy += R(2) * qy * lq2;
    }
    if (phi > R(0) && phi < R(1)) lphi += lta - ltb;
    // dJ = J - J_prev; J also stored
    lJx += ldJx + aJx;
    lJy += ldJy + aJy;
    const R ljpx = -ldJx, ljpy = -ldJy;
    // J = phi u
    lphi += ux * lJx + uy * lJy;
    lux += phi * lJx;
    luy += phi * lJy;

    R lF[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) lF[i] = R(0);
    if (a.coupled) {
      #pragma unroll
      for (int i = 0; i < 9; ++i) lF[i] = aF[i];
      const Mom<R> ld = lbmk::moments(aF);  // lambda_d = M lambda_f*
      R lm[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
      R lp = R(0), lru2 = R(0), luR = R(0), ljx = R(0), ljy = R(0), lFx = R(0), lFy = R(0);
      R lrho = R(0), lRx = R(0), lRy = R(0), lsD7 = R(0), lhD7 = R(0), lirho = R(0), lu2 = R(0);
      const R jx = rho * ux;
      // d0..d6
      lm[0] += ph.fsD[0] * ld.m0;
      luR += ph.fhD[0] * ld.m0;
      lm[1] += ph.fsD[1] * ld.m1;
      lp += R(-6) * ph.fsD[1] * ld.m1;
      lru2 += R(-3) * ph.fsD[1] * ld.m1;
      lm[2] += ph.fsD[2] * ld.m2;
      lp += R(9) * ph.fsD[2] * ld.m2;
      lru2 += R(3) * ph.fsD[2] * ld.m2;
      luR += -ph.fhD[2] * ld.m2;
      lm[3] += ph.fsD[3] * ld.m3;
      ljx += -ph.fsD[3] * ld.m3;
      lFx += ph.fhD[3] * ld.m3;
      lm[4] += ph.fsD[4] * ld.m4;
      ljx += ph.fsD[4] * ld.m4;
      lFx += -ph.fhD[4] * ld.m4;
      lm[5] += ph.fsD[5] * ld.m5;
      ljy += -ph.fsD[5] * ld.m5;
      lFy += ph.fhD[5] * ld.m5;
      lm[6] += ph.fsD[6] * ld.m6;
      ljy += ph.fsD[6] * ld.m6;
      lFy += -ph.fhD[6] * ld.m6;
      // d7 = sD7 (m7 - rho(ux^2 - uy^2)) + hD7 (2/3)(ux Rx - uy Ry)
      lm[7] += sD7 * ld.m7;
      lrho += -sD7 * (ux * ux - uy * uy) * ld.m7;
      lux += R(-2) * sD7 * rho * ux * ld.m7 + hD7 * R(2.0 / 3.0) * Rx * ld.m7;
      luy += R(2) * sD7 * rho * uy * ld.m7 - hD7 * R(2.0 / 3.0) * Ry * ld.m7;
      lRx += hD7 * R(2.0 / 3.0) * ux * ld.m7;
      lRy += -hD7 * R(2.0 / 3.0) * uy * ld.m7;
      lsD7 += (mf.m7 - rho * (ux * ux - uy * uy)) * ld.m7;
      lhD7 += R(2.0 / 3.0) * (ux * Rx - uy * Ry) * ld.m7;
      // d8 = sD7 (m8 - jx uy) + hD7 (1/3)(ux Ry + uy Rx)
      lm[8] += sD7 * ld.m8;
      ljx += -sD7 * uy * ld.m8;
      luy += -sD7 * jx * ld.m8 + hD7 * R(1.0 / 3.0) * Rx * ld.m8;
      lux += hD7 * R(1.0 / 3.0) * Ry * ld.m8;
      lRy += hD7 * R(1.0 / 3.0) * ux * ld.m8;
      lRx += hD7 * R(1.0 / 3.0) * uy * ld.m8;
      lsD7 += (mf.m8 - jx * uy) * ld.m8;
      lhD7 += R(1.0 / 3.0) * (ux * Ry + uy * Rx) * ld.m8;
      // s7 (= s8): sD7 = -s7/4, hD7 = 1/4 - s7/8
      const R ls7 = R(-0.25) * lsD7 - R(0.125) * lhD7;
      if (a.var_tau) {
        const R ltau = -s7 * s7 * ls7;  // s7 = 1/tau
        const R lmuv = R(3) * irho * ltau;
        lirho += R(3) * mu_v * ltau;
        lphi += a.dmu * lmuv;
      } else {
        gacc[4] += -s7 * s7 * ls7;  // s7 = 1/tau_f
      }
      // jx = rho ux, jy = rho uy
      lrho += ux * ljx + uy * ljy;
      lux += rho * ljx;
      luy += rho * ljy;
      // ru2 = rho u2
      lrho += u2 * lru2;
      lu2 += rho * lru2;
      // p = 0.6((m0 - F0) + uR/2 - (2/3) rho u2)
      lm[0] += R(0.6) * lp;
      lF[0] += R(-0.6) * lp;
      luR += R(0.3) * lp;
      lrho += R(-0.4) * u2 * lp;
      lu2 += R(-0.4) * rho * lp;
      // u2, uR
      lux += R(2) * ux * lu2 + Rx * luR;
      luy += R(2) * uy * lu2 + Ry * luR;
      lRx += ux * luR;
      lRy += uy * luR;
      // R = drho grad phi
      lgpx += a.drho * lRx;
      lgpy += a.drho * lRy;
      // u = (m + F/2) irho
      lm[3] += irho * lux;
      lFx += R(0.5) * irho * lux;
      lirho += (mf.m3 + R(0.5) * Fx) * lux;
      lm[5] += irho * luy;
      lFy += R(0.5) * irho * luy;
      lirho += (mf.m5 + R(0.5) * Fy) * luy;
      // m = M F
      lbmk::add_back(lF, lm[0], lm[1], lm[2], lm[3], lm[4], lm[5], lm[6], lm[7], lm[8]);
      // moving-wall term: F_i += rho c_ix u_w / 6, rho = rho_g + phi drho
      if (wbot) {
        const R l = (lF[5] - lF[6]) * R(1.0 / 6.0);
        lrho += a.u_bot * l;
        gacc[6] += rho * l;
      }
      if (wtop) {
        const R l = (lF[8] - lF[7]) * R(1.0 / 6.0);
        lrho += a.u_top * l;
        gacc[5] += rho * l;
      }
      // irho = 1/rho, rho = rho_g + phi drho
      lrho += -irho * irho * lirho;
      lphi += a.drho * lrho;
      // F = mu grad phi
      lmu += gpx * lFx + gpy * lFy;
      lgpx += mu * lFx;
      lgpy += mu * lFy;
    }
    // mu = beta4 poly - kappa lap
    lphi += ph.beta4 * (R(3) * phi * phi - R(3) * phi + R(0.5)) * lmu;
    llap += -ph.kappa * lmu;
    gacc[0] += poly * lmu;
    gacc[1] += -lap * lmu;

    // stencil adjoints (transpose of the difference forms above)
    const R gx3 = lgpx * R(1.0 / 3.0), gy3 = lgpy * R(1.0 / 3.0);
    const R gx12 = lgpx * R(1.0 / 12.0), gy12 = lgpy * R(1.0 / 12.0);
    const R la = R(2.0 / 3.0) * llap, ld6 = llap * R(1.0 / 6.0);
    a.lP[0 * n + k] = R(-10.0 / 3.0) * llap + lphi;
    a.lP[1 * n + k] = gx3 + la;
    a.lP[3 * n + k] = -gx3 + la;
    a.lP[2 * n + k] = gy3 + la;
    a.lP[4 * n + k] = -gy3 + la;
    a.lP[5 * n + k] = gx12 + gy12 + ld6;
    a.lP[6 * n + k] = -gx12 + gy12 + ld6;
    a.lP[7 * n + k] = -gx12 - gy12 + ld6;
    a.lP[8 * n + k] = gx12 - gy12 + ld6;
    a.lQ[0 * n + k] = R(4) * lqx;   // Q1
    a.lQ[2 * n + k] = R(-4) * lqx;  // Q3
    a.lQ[1 * n + k] = R(4) * lqy;   // Q2
    a.lQ[3 * n + k] = R(-4) * lqy;  // Q4
    a.lQ[4 * n + k] = lqx + lqy;    // Q5
    a.lQ[5 * n + k] = -lqx + lqy;   // Q6
    a.lQ[6 * n + k] = -lqx - lqy;   // Q7
    a.lQ[7 * n + k] = lqx - lqy;    // Q8

    // transpose of the pull: adjoint of the source positions (a bijection,
    // walls included)
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      a.aout[spl[i] * n + src[i]] = lF[i];
      a.aout[(9 + spl[i]) * n + src[i]] = lG[i];
    }
    a.aout[18 * n + k] = ljpx;
    a.aout[19 * n + k] = ljpy;
  }
  ad_block_partials(red, gacc, a.part);
}

// Sum the stencil adjoints referring to each node's phi and psi and add them
// to the adjoints of the node's 9 pulled g (phi = sum g).  With gB non-null
// the same launch also forms phi and psi of the state held in gB (plane
// stride PB): the state of the next adjoint step of a reverse sweep, whose
// ad_node reads them.  Each node reads its own phi before it overwrites it,
// and no other node reads it in this launch, so the two share the planes.
template <typename R>
__global__ void __launch_bounds__(kAdThreads, 4) ad_gather(R* __restrict__ phi, R* __restrict__ psi, const R* __restrict__ lP,
                          const R* __restrict__ lQ, int nx, int ny, int walls, R xi,
                          R* __restrict__ aout, const R* __restrict__ gB, int64_t PB) {
  const int64_t n = (int64_t)nx * ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)n; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    // The adjoints of the node's 9 pulled g sit at 9 distinct positions (the
    // pull is a bijection): read them all before any write, so that the
    // reads need not wait for the writes of the same array.  Offsets are
    // below 18 n < 2^32 (a case has at most 2.3e8 nodes).
    uint32_t at[9];
    R cur[9], G[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      int pl;
      const int pos = ad_src(i, x, y, nx, ny, walls, &pl);
      at[i] = (uint32_t)(9 + pl) * (uint32_t)n + (uint32_t)pos;
      cur[i] = aout[at[i]];
      if (gB) G[i] = gB[pl * PB + pos];
    }
    R sp = lP[k], sq = R(0);
    gather_uses(lP, lQ, x, y, nx, ny, walls, sp, sq);
    const R p = phi[k];
    const R dpsi = (p > R(0) && p < R(1)) ? dpsi_dphi(p, xi) : R(0);
    const R tot = sp + dpsi * sq;
    #pragma unroll
    for (int i = 0; i < 9; ++i) aout[at[i]] = cur[i] + tot;
    if (gB) {  // phi (Eq. 35) and psi (Eq. 37) of the next state, as ad_phase
      const R q = lbmk::sum9(G);
      phi[k] = q;
      psi[k] = lbmk::psi_of(q, xi);
    }
  }
}

// Adjoint of the initial state map (local part): phi0 -> hbar0, g_eq, f_eq,
// phi0 u0.  Writes the local phi0 adjoint and the adjoint of lap(phi0).
// The initial fields are FP64 (as lbm_init takes them) and so is this
// once-per-gradient arithmetic; the adjoint state is of type R.
template <typename R>
struct AdInitArgs {
  const double* phi0;
  const double* u0;  // [2][n] or null
  const R* ain;      // adjoint of S_0 [20][n]
  double* lphi;      // [n]
  double* llap;      // [n]
  double* part;
  int nx, ny;
  Phys<double> ph;
  double rho_g, drho;
  int coupled, vortex;
  double vU;
  int walls;
  double u_top, u_bot;
};

template <typename R>
__global__ void __launch_bounds__(kAdThreads) ad_init_local(const AdInitArgs<R> a) {
  __shared__ double red[kAdThreads / 32][kNParam];
  const int nx = a.nx, ny = a.ny;
  const int64_t n = (int64_t)nx * ny;
  const Phys<double>& ph = a.ph;
  double gacc[kNParam] = {0, 0, 0, 0, 0, 0, 0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)n; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    const double p = a.phi0[k];
    double s_ax = 0.0, s_dg = 0.0;
    #pragma unroll
    for (int j = 1; j < 9; ++j) {
      const double v = a.phi0[ad_nb(x, y, kAX(j), kAY(j), nx, ny, a.walls)];
      if (j < 5) s_ax += v; else s_dg += v;
    }
    const double lap = (2.0 / 3.0) * (s_ax - 4.0 * p) + (1.0 / 6.0) * (s_dg - 4.0 * p);
    const double poly = p * (p - 1.0) * (p - 0.5);
    double ux = 0.0, uy = 0.0;
    if (a.vortex) {
      double sx, cx, sy, cy;
      sincospi((x + 0.5) / nx, &sx, &cx);
      sincospi((y + 0.5) / ny, &sy, &cy);
      ux = -a.vU * sx * sx * (2.0 * sy * cy);
      uy = a.vU * sy * sy * (2.0 * sx * cx);
    } else if (a.u0) {
      ux = a.u0[k];
      uy = a.u0[n + k];
    }
    double lLam = 0.0, lphi = 0.0, lJx = a.ain[18 * n + k], lJy = a.ain[19 * n + k], lrho = 0.0;
    const double u2 = ux * ux + uy * uy;
    const double rho = a.rho_g + p * a.drho;
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      int pl;
      const int s = ad_src(i, x, y, nx, ny, a.walls, &pl);
      const double lg = a.ain[(9 + pl) * n + s];
      if (i == 0) {
        lphi += lg;
        lLam += (kAW(0) - 1.0) * lg;
      } else {
        lLam += kAW(i) * lg;
        lJx += 3.0 * kAW(i) * kAX(i) * lg;
        lJy += 3.0 * kAW(i) * kAY(i) * lg;
      }
      if (a.coupled) {
        const double cu = kAX(i) * ux + kAY(i) * uy;
        const double lf = a.ain[pl * n + s];
        lrho += kAW(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2) * lf;
        // the stored f of a population entering from a wall is f_eq minus the
        // moving-wall term rho c_ix u_w / 6 (added back when it is pulled)
        if (a.walls && ((y == 0 && kAY(i) == 1) || (y == ny - 1 && kAY(i) == -1))) {
          const bool bot = y == 0 && kAY(i) == 1;
          const double uw = bot ? a.u_bot : a.u_top;
          lrho += -kAX(i) * uw / 6.0 * lf;
          gacc[bot ? 6 : 5] += -rho * kAX(i) / 6.0 * lf;
        }
      }
    }
    lphi += ux * lJx + uy * lJy + a.drho * lrho;
    const double lmu = lLam;
    lphi += ph.lambda * lLam;
    gacc[2] += p * lLam;
    lphi += ph.beta4 * (3.0 * p * p - 3.0 * p + 0.5) * lmu;
    gacc[0] += poly * lmu;
    gacc[1] += -lap * lmu;
    a.lphi[k] = lphi;
    a.llap[k] = -ph.kappa * lmu;
  }
  ad_block_partials(red, gacc, a.part);
}

// lambda_phi0(y) = local - (10/3) llap(y) + sum over the nodes s whose
// Laplacian entry j reads y of w_lap_j * llap(s) (walls: mirrored ghost rows)
__global__ void ad_init_gather(const double* __restrict__ lphi, const double* __restrict__ llap,
                               int nx, int ny, int walls, double* __restrict__ out) {
  const int64_t n = (int64_t)nx * ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)n; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    double v = lphi[k] - (10.0 / 3.0) * llap[k];
    #pragma unroll
    for (int j = 1; j < 9; ++j) {
      const double w = j < 5 ? 2.0 / 3.0 : 1.0 / 6.0;
      const int ys = y - kAY(j);
      if (!walls || (ys >= 0 && ys < ny)) v += w * llap[shift(x, y, -kAX(j), -kAY(j), nx, ny)];
      if (walls && ((y == 0 && kAY(j) == -1) || (y == ny - 1 && kAY(j) == 1))) {
        int xs = x - kAX(j);
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        v += w * llap[y * nx + xs];
      }
    }
    out[k] = v;
  }
}

// The adjoint of phi = sum of pulled g, seeded from an FP64 field adjoint:
// every node scatters dphi to the positions of its 9 pulled g (the f and
// phi*u planes are cleared beforehand).
template <typename R>
__global__ void ad_seed_phi(const double* __restrict__ dphi, int nx, int ny, int walls,
                            R* __restrict__ aout) {
  const int64_t n = (int64_t)nx * ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)n; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      int pl;
      const int pos = ad_src(i, x, y, nx, ny, walls, &pl);
      aout[(9 + pl) * n + pos] = (R)dphi[k];
    }
  }
}

// Adds the accumulated per-block parameter partials (in block order) to the
// device accumulator `acc`, which lbm_adjoint_take_param_grads reads and
// clears, and clears the partials.  Deterministic sum (launch: one block of
// 32 * kNParam threads): warp q sums parameter q, lane l the blocks l, l + 32,
// ... in order, then a fixed shuffle tree.
__global__ void ad_sum_partials(double* __restrict__ part, int nb, double* __restrict__ acc) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= kNParam) return;
  double v = 0.0;
  for (int b = lane; b < nb; b += 32) {
    v += part[(int64_t)b * kNParam + q];
    part[(int64_t)b * kNParam + q] = 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) acc[q] += v;
}

// Scratch layout inside the caller's adjoint workspace: 19 planes of n
// values in the handle's precision (phi, psi, 9 phi-stencil and 8
// psi-stencil adjoints), then the FP64 per-block partials and accumulators.
// The initial-state adjoint reuses the stencil planes as two FP64 planes.
struct AdScratch {
  void *phi, *psi, *lP, *lQ;
  double *part, *sums;
  double *init_lphi, *init_llap;
};

size_t elem_bytes(const lbm_handle* h) { return h->precision == LBM_F64 ? 8 : 4; }

size_t planes_bytes(int64_t n, size_t es) { return (19 * (size_t)n * es + 255) / 256 * 256; }

AdScratch carve(lbm_handle* h) {
  const int64_t n = (int64_t)h->params[0].nx * h->params[0].ny;
  const size_t es = elem_bytes(h);
  char* b = h->adj_ws;
  AdScratch s;
  s.phi = b;
  s.psi = b + n * es;
  s.lP = b + 2 * n * es;
  s.lQ = b + 11 * n * es;
  s.part = (double*)(b + planes_bytes(n, es));
  s.sums = s.part + kAdBlocks * kNParam;
  s.init_lphi = (double*)s.lP;  // 9 planes of es bytes hold 2 FP64 planes
  s.init_llap = s.init_lphi + n;
  return s;
}

size_t scratch_bytes(int64_t n, size_t es) {
  return planes_bytes(n, es) + (size_t)(kAdBlocks * kNParam + 8) * sizeof(double);
}

int check_handle(lbm_handle* h, bool need_ws) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (h->ncases != 1) return fail(LBM_ERR_ARG, "reverse mode needs a single-case handle");
  if (need_ws && !h->adj_ws) return fail(LBM_ERR_WORKSPACE, "call lbm_adjoint_attach first");
  return LBM_OK;
}

// Combine the raw partial sums into
// d/d(sigma, tau_g, lambda, tau_f, u_wall_top, u_wall_bottom).
void to_param_grads(const lbm_params& p, const double raw[kNParam], double* out) {
  out[0] += raw[0] * (48.0 / p.W) + raw[1] * (1.5 * p.W);  // beta4 = 48 sigma/W, kappa = 1.5 sigma W
  out[1] += raw[3];
  out[2] += raw[2];
  out[3] += raw[4];
  out[4] += raw[5];
  out[5] += raw[6];
}

// Reads and clears the device accumulator, adding d/d(sigma, tau_g, lambda,
// tau_f) to out (synchronises).
int take_grads(lbm_handle* h, double* out) {
  AdScratch s = carve(h);
  double raw[kNParam];
  ad_sum_partials<<<1, 32 * kNParam, 0, h->stream>>>(s.part, kAdBlocks, s.sums);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(raw, s.sums, sizeof raw, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.sums, 0, sizeof raw, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  to_param_grads(h->params[0], raw, out);
  return LBM_OK;
}

template <typename R>
const CaseDev<R>& case0(const lbm_handle* h) {
  if constexpr (sizeof(R) == 4) return h->cf[0]; else return h->cd[0];
}

template <typename R>
const Phys<R>& phys(const lbm_handle* h) {
  if constexpr (sizeof(R) == 4) return h->pf; else return h->pd;
}

}  // namespace

extern "C" {

size_t lbm_adjoint_workspace_bytes(const lbm_handle* h) {
  if (!h || h->ncases != 1) return 0;
  return scratch_bytes((int64_t)h->params[0].nx * h->params[0].ny, elem_bytes(h));
}

int lbm_adjoint_attach(lbm_handle* h, void* d_scratch, size_t bytes) {
  int rc = check_handle(h, false);
  if (rc) return rc;
  if (!d_scratch) return fail(LBM_ERR_WORKSPACE, "adjoint scratch is null");
  if ((uintptr_t)d_scratch % 256) return fail(LBM_ERR_WORKSPACE, "adjoint scratch not 256-byte aligned");
  if (bytes < lbm_adjoint_workspace_bytes(h)) return fail(LBM_ERR_WORKSPACE, "adjoint scratch too small");
  h->adj_ws = (char*)d_scratch;
  h->adj_ws_bytes = bytes;
  cudaError_t e = cudaMemsetAsync(carve(h).part, 0, (kAdBlocks + 1) * kNParam * sizeof(double),
                                  h->stream);  // partials and accumulator
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_adjoint_take_param_grads(lbm_handle* h, double* h_param_grads) {
  int rc = check_handle(h, true);
  if (rc) return rc;
  if (!h_param_grads) return fail(LBM_ERR_ARG, "h_param_grads is null");
  return take_grads(h, h_param_grads);
}

int lbm_adjoint_seed_phi(lbm_handle* h, const double* d_dphi, void* d_adj_state) {
  int rc = check_handle(h, false);
  if (rc) return rc;
  if (!d_dphi || !d_adj_state) return fail(LBM_ERR_ARG, "null pointer");
  const lbm_params& p = h->params[0];
  cudaError_t e = cudaMemsetAsync(d_adj_state, 0, 20 * elem_bytes(h) * p.nx * (size_t)p.ny,
                                  h->stream);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (h->precision == LBM_F32)
    ad_seed_phi<float><<<kAdBlocks, kAdThreads, 0, h->stream>>>(d_dphi, p.nx, p.ny, p.walls,
                                                                (float*)d_adj_state);
  else
    ad_seed_phi<double><<<kAdBlocks, kAdThreads, 0, h->stream>>>(d_dphi, p.nx, p.ny, p.walls,
                                                                 (double*)d_adj_state);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"

namespace {

// One adjoint step from the state S_t held in (fA, gA, JA) with plane stride
// P at step index t (the handle's own buffers, or a snapshot).
// phase_ready: phi and psi of S_t are already in the scratch planes (the
// previous step of a sweep formed them); gB/PB: g planes of the state of the
// next step of a sweep, whose phi and psi the gather launch forms, or null.
template <typename R>
int adjoint_step_impl(lbm_handle* h, const R* fA, const R* gA, const R* JA, int64_t P, int64_t t,
                      const void* d_adj_in, void* d_adj_out, double* h_param_grads,
                      bool phase_ready = false, const R* gB = nullptr, int64_t PB = 0) {
  const lbm_params& p = h->params[0];
  const CaseDev<R>& cd = case0<R>(h);
  const bool coupled = h->flow == LBM_FLOW_COUPLED;
  AdScratch s = carve(h);
  if (!phase_ready)
    ad_phase<R><<<kAdBlocks, kAdThreads, 0, h->stream>>>(gA, P, p.nx, p.ny, p.walls, (R)p.xi,
                                                         (R*)s.phi, (R*)s.psi);
  AdArgs<R> a{};
  a.fA = coupled ? fA : nullptr;
  a.gA = gA;
  a.JA = JA;
  a.P = P;
  a.nx = p.nx;
  a.ny = p.ny;
  a.phi = (const R*)s.phi;
  a.psi = (const R*)s.psi;
  a.ain = (const R*)d_adj_in;
  a.aout = (R*)d_adj_out;
  a.lP = (R*)s.lP;
  a.lQ = (R*)s.lQ;
  a.part = s.part;
  a.ph = phys<R>(h);
  a.rho_g = cd.rho_g;
  a.drho = cd.drho;
  a.mu_g = cd.mu_g;
  a.dmu = cd.dmu;
  a.sD7 = cd.sD7;
  a.hD7 = cd.hD7;
  a.s7 = (R)(1.0 / p.tau_f_l);
  a.var_tau = cd.var_tau;
  a.coupled = coupled ? 1 : 0;
  a.ct = (R)(coupled ? 0.0 : cospi((double)t / p.vortex_T) * p.vortex_U);
  a.invW = (R)(1.0 / p.W);
  a.walls = p.walls;
  a.u_top = (R)(p.walls ? p.u_wall_top : 0.0);
  a.u_bot = (R)(p.walls ? p.u_wall_bottom : 0.0);
  if (!coupled) {  // the f planes and the tau_f entry stay zero
    cudaError_t e = cudaMemsetAsync(d_adj_out, 0, 9 * sizeof(R) * p.nx * (size_t)p.ny, h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  }
  ad_node<R><<<kAdBlocks, kAdThreads, 0, h->stream>>>(a);
  ad_gather<R><<<kAdBlocks, kAdThreads, 0, h->stream>>>((R*)s.phi, (R*)s.psi, (const R*)s.lP,
                                                        (const R*)s.lQ, p.nx, p.ny, p.walls,
                                                        (R)p.xi, (R*)d_adj_out, gB, PB);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (h_param_grads) return take_grads(h, h_param_grads);
  return LBM_OK;
}

template <typename R>
int adjoint_init_impl(lbm_handle* h, const double* d_phi0, const double* d_u0,
                      const void* d_adj_state, double* d_adj_phi0, double* h_param_grads) {
  const lbm_params& p = h->params[0];
  AdScratch s = carve(h);
  AdInitArgs<R> a{};
  a.phi0 = d_phi0;
  a.u0 = d_u0;
  a.ain = (const R*)d_adj_state;
  a.lphi = s.init_lphi;
  a.llap = s.init_llap;
  a.part = s.part;
  a.nx = p.nx;
  a.ny = p.ny;
  a.ph = h->pd;
  const bool coupled = h->flow == LBM_FLOW_COUPLED;
  a.rho_g = coupled ? p.rho_g : 1.0;
  a.drho = coupled ? p.rho_l - p.rho_g : 0.0;
  a.coupled = coupled;
  a.vortex = h->flow == LBM_FLOW_VORTEX;
  a.vU = p.vortex_U;
  a.walls = p.walls;
  a.u_top = p.walls ? p.u_wall_top : 0.0;
  a.u_bot = p.walls ? p.u_wall_bottom : 0.0;
  ad_init_local<R><<<kAdBlocks, kAdThreads, 0, h->stream>>>(a);
  ad_init_gather<<<kAdBlocks, kAdThreads, 0, h->stream>>>(s.init_lphi, s.init_llap, p.nx, p.ny,
                                                          p.walls, d_adj_phi0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (h_param_grads) return take_grads(h, h_param_grads);
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_adjoint_step(lbm_handle* h, const void* d_adj_in, void* d_adj_out, double* h_param_grads) {
  int rc = check_handle(h, true);
  if (rc) return rc;
  if (!d_adj_in || !d_adj_out) return fail(LBM_ERR_ARG, "null adjoint buffer");
  if (d_adj_in == d_adj_out) return fail(LBM_ERR_ARG, "d_adj_in and d_adj_out must differ");
  if (h->precision == LBM_F32) {
    const CaseDev<float>& cd = h->cf[0];
    return adjoint_step_impl<float>(h, cd.f[h->parity], cd.g[h->parity], cd.J[h->parity],
                                    cd.plane, h->t, d_adj_in, d_adj_out, h_param_grads);
  }
  const CaseDev<double>& cd = h->cd[0];
  return adjoint_step_impl<double>(h, cd.f[h->parity], cd.g[h->parity], cd.J[h->parity], cd.plane,
                                   h->t, d_adj_in, d_adj_out, h_param_grads);
}

int lbm_adjoint_step_from(lbm_handle* h, const void* d_state, int64_t t, const void* d_adj_in,
                          void* d_adj_out, double* h_param_grads) {
  int rc = check_handle(h, true);
  if (rc) return rc;
  if (!d_state || !d_adj_in || !d_adj_out) return fail(LBM_ERR_ARG, "null buffer");
  if (t < 0) return fail(LBM_ERR_ARG, "t < 0");
  if (d_adj_in == d_adj_out || d_state == d_adj_out)
    return fail(LBM_ERR_ARG, "d_adj_out must differ from d_adj_in and d_state");
  const int64_t n = (int64_t)h->params[0].nx * h->params[0].ny;
  if (h->precision == LBM_F32) {
    const float* st = (const float*)d_state;
    return adjoint_step_impl<float>(h, st, st + 9 * n, st + 18 * n, n, t, d_adj_in, d_adj_out,
                                    h_param_grads);
  }
  const double* st = (const double*)d_state;
  return adjoint_step_impl<double>(h, st, st + 9 * n, st + 18 * n, n, t, d_adj_in, d_adj_out,
                                   h_param_grads);
}

int lbm_adjoint_sweep(lbm_handle* h, const void* d_states, int64_t stride_bytes, int64_t t0,
                      int32_t count, void* d_adj, void* d_spare) {
  int rc = check_handle(h, true);
  if (rc) return rc;
  if (!d_states || !d_adj || !d_spare || d_adj == d_spare)
    return fail(LBM_ERR_ARG, "null or aliased buffers");
  if (t0 < 0 || count < 0) return fail(LBM_ERR_ARG, "t0 and count must be >= 0");
  const int64_t n = (int64_t)h->params[0].nx * h->params[0].ny;
  const size_t es = elem_bytes(h);
  if (count > 1 && stride_bytes < (int64_t)(20 * n * es))
    return fail(LBM_ERR_ARG, "stride_bytes smaller than a state");
  void* cur = d_adj;
  void* nxt = d_spare;
  // each gather launch also forms phi and psi of the state of the next step
  for (int32_t j = count - 1; j >= 0; --j) {
    const char* st = (const char*)d_states + (int64_t)j * stride_bytes;
    const char* stB = j > 0 ? st - stride_bytes : nullptr;
    const bool ready = j != count - 1;
    if (h->precision == LBM_F32) {
      const float* sf = (const float*)st;
      const float* gB = stB ? (const float*)stB + 9 * n : nullptr;
      rc = adjoint_step_impl<float>(h, sf, sf + 9 * n, sf + 18 * n, n, t0 + j, cur, nxt, nullptr,
                                    ready, gB, n);
    } else {
      const double* sd = (const double*)st;
      const double* gB = stB ? (const double*)stB + 9 * n : nullptr;
      rc = adjoint_step_impl<double>(h, sd, sd + 9 * n, sd + 18 * n, n, t0 + j, cur, nxt,
                                     nullptr, ready, gB, n);
    }
    if (rc) return rc;
    void* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  if (cur != d_adj) {  // an odd count ends in the spare buffer
    cudaError_t e = cudaMemcpyAsync(d_adj, cur, 20 * n * es, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  }
  return LBM_OK;
}

int lbm_adjoint_init(lbm_handle* h, const double* d_phi0, const double* d_u0,
                     const void* d_adj_state, double* d_adj_phi0, double* h_param_grads) {
  int rc = check_handle(h, true);
  if (rc) return rc;
  if (!d_phi0 || !d_adj_state || !d_adj_phi0) return fail(LBM_ERR_ARG, "null pointer");
  if (h->precision == LBM_F32)
    return adjoint_init_impl<float>(h, d_phi0, d_u0, d_adj_state, d_adj_phi0, h_param_grads);
  return adjoint_init_impl<double>(h, d_phi0, d_u0, d_adj_state, d_adj_phi0, h_param_grads);
}

}  // extern "C"
