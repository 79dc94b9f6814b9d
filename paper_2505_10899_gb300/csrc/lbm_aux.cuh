// Auxiliary kernels: initial state, state import/export, phase volumes,
// step clock.  None of them is on the per-step path except the clock.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_layout.h"
#include "lbm_node.cuh"

namespace lbmk {

__device__ __constant__ static const int kCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ static const int kCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

__device__ __constant__ static const int kOPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

// Position in a pull buffer that holds the value population i must deliver
// to node (x, y): (x - c_ix, y - c_iy), periodic.
__device__ __forceinline__ int64_t pull_src(int i, int x, int y, int nx, int ny) {
  int xs = x - kCX[i], ys = y - kCY[i];
  xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
  ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
  return (int64_t)ys * nx + xs;
}

// The same with walls: a population that would come from beyond a wall is
// the node's own population in the opposite direction (halfway bounce-back).
// Returns the position; *plane receives the plane it sits in.
__device__ __forceinline__ int64_t pull_loc(int i, int x, int y, int nx, int ny, int walls,
                                            int* plane) {
  const int ys = y - kCY[i];
  if (walls && (ys < 0 || ys >= ny)) {
    *plane = kOPP[i];
    return (int64_t)y * nx + x;
  }
  *plane = i;
  return pull_src(i, x, y, nx, ny);
}

// Moving-wall term carried by population i at node (x, y) after streaming:
// 2 w_i rho (c_i . u_w) / c_s^2 for a population entering from a wall.
template <typename T>
__device__ __forceinline__ double wall_term(const CaseDev<T>& cd, int i, int y, double rho) {
  if (!cd.walls) return 0.0;
  const double w = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  if (y == 0 && kCY[i] == 1) return 6.0 * w * rho * kCX[i] * (double)cd.u_bot;
  if (y == cd.ny - 1 && kCY[i] == -1) return 6.0 * w * rho * kCX[i] * (double)cd.u_top;
  return 0.0;
}

// phi at node (x, y) of buffer `par` (Eq. 35, the pulled g), in FP64.
template <typename T>
__device__ __forceinline__ double phi_at(const CaseDev<T>& cd, int par, int x, int y) {
  double phi = 0.0;
  for (int i = 0; i < 9; ++i) {
    int pl;
    const int64_t pos = pull_loc(i, x, y, cd.nx, cd.ny, cd.walls, &pl);
    phi += (double)cd.g[par][pl * cd.plane + pos];
  }
  if (cd.g0lo[par]) phi += (double)cd.g0lo[par][(int64_t)y * cd.nx + x];
  return phi;
}

// The moving-wall term of wall_term in the arithmetic type R of the init.
template <typename T, typename R>
__device__ __forceinline__ R wall_term_r(const CaseDev<T>& cd, int i, int y, R rho) {
  if (!cd.walls) return R(0);
  const R w = (i == 0) ? R(4.0 / 9.0) : (i < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
  if (y == 0 && kCY[i] == 1) return R(6) * w * rho * R(kCX[i]) * (R)cd.u_bot;
  if (y == cd.ny - 1 && kCY[i] == -1) return R(6) * w * rho * R(kCX[i]) * (R)cd.u_top;
  return R(0);
}

// Initial state of one node (Sec. 4 set-ups): hbar0 = 4 beta phi0 (phi0-1)
// (phi0-1/2) - kappa lap(phi0) (Eq. 2), g = g_eq(phi0, hbar0, u0) (Eq. 31),
// f = f_eq(p=0, rho(phi0), u0) (Eq. 22), phi*u at t-1 = phi0 u0.  p64: phi0
// of the node in FP64, p: the same in R; nb: phi0 at the eight neighbours E,
// W, N, S, NE, NW, SE, SW in R (with walls, the ghost rows mirror the wall
// rows).
// R is the arithmetic type: FP64 for FP64 state (computed in FP64, rounded
// once); FP32 for FP32 state.  The FP64 pipe of this GPU runs at 1/64 of the
// FP32 rate, so the FP32 init keeps off it: the rest population, the
// remainder g_0 = phi0 - (sum of the stored movers) that makes the stored
// populations sum to phi0, is formed in float-pair arithmetic -- the movers
// summed by error-free TwoSums into a pair, phi0 split into a pair (one FP64
// subtraction), their difference by another TwoSum -- and stored as the float
// pair (hi + lo) of the FP32 step.  The pair sums to phi0 within about 2^-42
// of phi0 (the FP32 rounding of the summed TwoSum errors), far below the
// FP32 state's own rounding.
template <typename T, typename R>
__device__ __forceinline__ void init_node(const CaseDev<T>& cd, int x, int y, double p64, R p,
                                          const R nb[8], R ux, R uy, R beta4, R kappa,
                                          R lambda, R rho_g, R drho, int parity) {
  const int nx = cd.nx, ny = cd.ny;
  const int64_t k = (int64_t)y * nx + x;
  const R lap = R(2.0 / 3.0) * (((nb[0] + nb[1]) + (nb[2] + nb[3])) - R(4) * p) +
                R(1.0 / 6.0) * (((nb[4] + nb[5]) + (nb[6] + nb[7])) - R(4) * p);
  const R mu = beta4 * p * (p - R(1)) * (p - R(0.5)) - kappa * lap;
  const R lam = mu + lambda * p;
  const R Jx = p * ux, Jy = p * uy;
  const R rho = rho_g + p * drho;
  const R u2 = ux * ux + uy * uy;
  T* gb = cd.g[parity];
  T* fb = cd.f[parity];
  float ms = 0.f, me = 0.f;  // FP32: sum of the stored movers as a float pair
  int64_t dst0 = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const R w = (i == 0) ? R(4.0 / 9.0) : (i < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
    const R cu = R(kCX[i]) * ux + R(kCY[i]) * uy;
    const R cJ = R(kCX[i]) * Jx + R(kCY[i]) * Jy;
    int pl;
    const int64_t pos = pull_loc(i, x, y, nx, ny, cd.walls, &pl);  // sets pl
    const int64_t dst = pos + (int64_t)pl * cd.plane;
    if (i == 0) {
      dst0 = dst;
      if (sizeof(R) == 8) gb[dst] = (T)(p + (w - R(1)) * lam);
    } else {
      const T gi = (T)(w * lam + R(3) * w * cJ);
      gb[dst] = gi;
      if (sizeof(R) == 4) {
        float t, e;
        two_sum_f(ms, (float)gi, t, e);
        ms = t;
        me = __fadd_rn(me, e);
      }
    }
    // f arriving from a wall carries the moving-wall term on top of the
    // stored value: store f_eq minus that term
    if (fb)
      fb[dst] = (T)(rho * w * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * u2) -
                    wall_term_r<T, R>(cd, i, y, rho));
  }
  if (sizeof(R) == 4) {  // FP32: g_0 = phi0 - movers as a float pair (high + low part)
    const float ph = (float)p;                       // p = phi0 rounded to FP32
    const float pl = (float)(p64 - (double)ph);      // exact remainder, rounded
    float d, e;
    two_sum_f(ph, -ms, d, e);                        // ph - ms = d + e exactly
    const float rest = __fadd_rn(e, __fsub_rn(pl, me));
    float hi, lo;
    two_sum_f(d, rest, hi, lo);
    gb[dst0] = (T)hi;
    if (cd.g0lo[parity]) cd.g0lo[parity][k] = (T)lo;
  }
  cd.J[parity][k] = (T)Jx;
  cd.J[parity][cd.plane + k] = (T)Jy;
}

// Initial state of every case of a batch in one launch: one CTA per work
// item (case, strip of BX columns from x0, run of nrows rows from y0), as
// the step kernel tiles the batch.  The rows of phi0 the item needs (its own
// and one halo row above and below, each with one halo column on either
// side) pass through a ring of eight shared-memory rows, loaded two rows
// ahead of the row being initialised, so every value of phi0 is read once
// per item, coalesced along x; u0 of a node is read two rows ahead into
// registers.  The fields may sit in host memory read over the CPU-GPU link,
// whose latency the two rows in flight hide.
template <typename T, int BX>
__global__ void __launch_bounds__(BX) init_items(const CaseDev<T>* __restrict__ cases,
                                                 const Item* __restrict__ items,
                                                 const InitSrc* __restrict__ src, double beta4,
                                                 double kappa, double lambda, int vortex,
                                                 double vU, int parity) {
  __shared__ double ring[8][BX + 2];
  // FP32 state: phi0 also rounded to FP32 once per loaded value, for the
  // arithmetic (the FP64 ring serves the rest population of the own node)
  constexpr bool kF32 = sizeof(T) == 4;
  __shared__ T rring[kF32 ? 8 : 1][BX + 2];
  const Item it = items[blockIdx.x];
  const CaseDev<T> cd = cases[it.c];
  const InitSrc sc = src[it.c];
  const int nx = cd.nx, ny = cd.ny, tid = threadIdx.x;
  const int wact = min(BX, nx - it.x0);
  const bool act = tid < wact;
  const int x = it.x0 + (act ? tid : 0);
  const int yend = it.y0 + it.nrows;
  // halo columns: x0 - 1 (thread 0) and x0 + wact (thread BX - 1), periodic
  const int xl = it.x0 == 0 ? nx - 1 : it.x0 - 1;
  const int xr = it.x0 + wact == nx ? 0 : it.x0 + wact;
  auto row_of = [&](int r) -> int {  // with walls the ghost row mirrors the wall row
    if (r < 0) return cd.walls ? 0 : ny - 1;
    if (r >= ny) return cd.walls ? ny - 1 : 0;
    return r;
  };
  // phi0 of row r at this thread's ring slots (own column; thread 0 also the
  // left halo column, thread BX - 1 the right one), fetched into registers
  // and stored into the ring two rows later, so that the loads of the
  // following rows stay in flight while a row is initialised (a load
  // stored straight into shared memory would stall the thread on it)
  struct RowV {
    double c = 0.0, h = 0.0;
  };
  auto fetch = [&](int r) -> RowV {
    RowV v;
    if (r > yend) return v;  // past the halo row below the item
    const int64_t base = (int64_t)row_of(r) * nx;
    if (act) v.c = sc.phi[base + x];
    if (tid == 0) v.h = sc.phi[base + xl];
    if (tid == BX - 1) v.h = sc.phi[base + xr];
    return v;
  };
  auto stash = [&](int r, const RowV& v) {
    if (r > yend) return;
    double* dst = ring[r & 7];
    T* rdst = rring[kF32 ? (r & 7) : 0];
    auto put = [&](int slot, double val) {
      dst[slot] = val;
      if constexpr (kF32) rdst[slot] = (T)val;
    };
    if (act) put(tid + 1, v.c);
    if (tid == 0) put(0, v.h);
    if (tid == BX - 1) put(wact + 1, v.h);
  };
  // u0 of the own node of row r (rows of this item only)
  const bool has_u = !vortex && sc.u != nullptr;
  auto load_u = [&](int r, double& ux, double& uy) {
    if (has_u && act && r < yend) {
      const int64_t k = (int64_t)r * nx + x;
      ux = sc.u[k];
      uy = sc.u[(int64_t)nx * ny + k];
    }
  };
  using R = T;  // arithmetic type of the init, see init_node
  const R beta4r = (R)beta4, kappar = (R)kappa, lambdar = (R)lambda, vUr = (R)vU;
  const R rhogr = (R)sc.rho_g, drhor = (R)sc.drho;
  double ux0 = 0.0, uy0 = 0.0, ux1 = 0.0, uy1 = 0.0;
  stash(it.y0 - 1, fetch(it.y0 - 1));
  stash(it.y0, fetch(it.y0));
  stash(it.y0 + 1, fetch(it.y0 + 1));
  RowV pA = fetch(it.y0 + 2), pB = fetch(it.y0 + 3);  // rows in flight
  load_u(it.y0, ux0, uy0);
  load_u(it.y0 + 1, ux1, uy1);
  for (int y = it.y0; y < yend; ++y) {
    // phi0 of row y + 4 and u0 of row y + 2 start; row y + 2 (fetched two
    // rows ago) goes into the ring (slot (y+2) & 7, last read for row y - 5)
    const RowV pC = fetch(y + 4);
    double ux2 = 0.0, uy2 = 0.0;
    load_u(y + 2, ux2, uy2);
    stash(y + 2, pA);
    pA = pB;
    pB = pC;
    __syncthreads();  // rows up to y + 1 are in the ring
    if (act) {
      const int c = tid + 1;
      // arithmetic in R: FP32 values from the rounded ring, FP64 from the FP64 one
      const R* rS = kF32 ? (const R*)rring[kF32 ? ((y - 1) & 7) : 0] : (const R*)ring[(y - 1) & 7];
      const R* rC = kF32 ? (const R*)rring[kF32 ? (y & 7) : 0] : (const R*)ring[y & 7];
      const R* rN = kF32 ? (const R*)rring[kF32 ? ((y + 1) & 7) : 0] : (const R*)ring[(y + 1) & 7];
      const R nb[8] = {rC[c + 1], rC[c - 1], rN[c], rS[c],
                       rN[c + 1], rN[c - 1], rS[c + 1], rS[c - 1]};
      R ux = (R)ux0, uy = (R)uy0;
      if (vortex) {
        R sx, cx, sy, cy;
        Num<R>::sincospi_((R(x) + R(0.5)) / R(nx), &sx, &cx);
        Num<R>::sincospi_((R(y) + R(0.5)) / R(ny), &sy, &cy);
        ux = -vUr * sx * sx * (R(2) * sy * cy);
        uy = vUr * sy * sy * (R(2) * sx * cx);
      }
      init_node<T, R>(cd, x, y, ring[y & 7][c], rC[c], nb, ux, uy, beta4r, kappar, lambdar,
                      rhogr, drhor, parity);
    }
    ux0 = ux1, uy0 = uy1, ux1 = ux2, uy1 = uy2;
  }
}

// Device snapshot of one case's state (the layout of lbm_snapshot): plane
// blockIdx.y of [f: 9][g: 9][phi*u: 2][low part of g_0: 1, FP32 only], each
// n values, from the buffers with plane stride P (f null: zero planes).  One
// launch for the whole snapshot instead of a copy per buffer.
template <typename T>
__global__ void snapshot_kernel(const T* __restrict__ f, const T* __restrict__ g,
                                const T* __restrict__ J, const T* __restrict__ lo, int64_t P,
                                int64_t n, T* __restrict__ out) {
  const int pl = blockIdx.y;
  const T* src = pl < 9 ? (f ? f + pl * P : nullptr)
                        : (pl < 18 ? g + (pl - 9) * P : (pl < 20 ? J + (pl - 18) * P : lo));
  T* dst = out + (int64_t)pl * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src ? src[k] : T(0);
}

// Import one population plane (FP64 host layout, value at the node it
// belongs to after streaming) into a pull buffer, or export it.
// buf: the 9-plane buffer (plane stride P); with walls the value of plane i
// at a wall row may sit in the opposite plane (bounce-back).
template <typename T>
__global__ void plane_import(T* __restrict__ buf, int64_t P, const double* __restrict__ src,
                             int i, int nx, int ny, int walls) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % nx), y = (int)(k / nx);
    int pl;
    const int64_t pos = pull_loc(i, x, y, nx, ny, walls, &pl);
    buf[pl * P + pos] = (T)src[k];
  }
}

template <typename T>
__global__ void plane_export(double* __restrict__ dst, const T* __restrict__ buf, int64_t P,
                             int i, int nx, int ny, int walls) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % nx), y = (int)(k / nx);
    int pl;
    const int64_t pos = pull_loc(i, x, y, nx, ny, walls, &pl);
    dst[k] = (double)buf[pl * P + pos];
  }
}

// f plane i of an exported / imported state at the wall rows: add (sign +1)
// or remove (sign -1) the moving-wall term, with rho from the phi of the g
// buffer of parity `par` (which must already hold the state).
template <typename T>
__global__ void wall_f_fix(double* __restrict__ v, CaseDev<T> cd, int par, int i,
                           double rho_g, double drho, double sign) {
  const int nx = cd.nx, ny = cd.ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * nx; k += gridDim.x * blockDim.x) {
    const int x = k % nx, y = k < nx ? 0 : ny - 1;
    if (k >= nx && ny == 1) continue;  // one row: already handled as row 0
    const double rho = rho_g + phi_at(cd, par, x, y) * drho;
    v[(int64_t)y * nx + x] += sign * wall_term(cd, i, y, rho);
  }
}

// The low part of g_0 (FP32 float pair, own node, unshifted): added to an
// exported FP64 plane, or split off an imported FP64 plane whose high part
// the import rounded.
template <typename T>
__global__ void add_lo_f64(double* __restrict__ v, const T* __restrict__ lo, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    v[k] += (double)lo[k];
}
template <typename T>
__global__ void lo_from_f64(T* __restrict__ lo, const T* __restrict__ hi,
                            const double* __restrict__ v, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    lo[k] = (T)(v[k] - (double)hi[k]);
}

// Plain (unshifted) plane copies with precision change, for phi*u.
template <typename T>
__global__ void copy_to_T(T* __restrict__ dst, const double* __restrict__ src, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = (T)src[k];
}
template <typename T>
__global__ void copy_to_f64(double* __restrict__ dst, const T* __restrict__ src, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = (double)src[k];
}

// Phase volumes, pass 1: every CTA reduces phi = sum_i g_i (pulled, Eq. 35)
// over its work item into per-region FP64 partials, in a fixed order.
template <typename T, int BX>
__global__ void __launch_bounds__(BX) volume_partial(const CaseDev<T>* __restrict__ cases,
                                                     const Item* __restrict__ items,
                                                     int parity, double* __restrict__ part) {
  __shared__ double red[BX / 32][kMaxRegions];
  const Item it = items[blockIdx.x];
  const CaseDev<T>& cd = cases[it.c];
  const int nx = cd.nx, ny = cd.ny, nr = cd.nregions;
  const int64_t P = cd.plane;
  const int x = it.x0 + threadIdx.x;
  const bool act = x < nx;
  const T* __restrict__ gs = cd.g[parity];
  double acc[kMaxRegions];
#pragma unroll
  for (int r = 0; r < kMaxRegions; ++r) acc[r] = 0.0;
  if (act) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    for (int k = 0; k < it.nrows; ++k) {
      const int y = it.y0 + k;
      const int64_t o0 = (int64_t)y * nx;
      double phi;
      if (cd.walls) {
        phi = phi_at(cd, parity, x, y);
      } else {
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int64_t om = (int64_t)ym * nx, op = (int64_t)yp * nx;
        phi = (double)gs[o0 + x];
        if (cd.g0lo[parity]) phi += (double)cd.g0lo[parity][o0 + x];
        phi += (double)gs[P + o0 + xm];
        phi += (double)gs[2 * P + om + x];
        phi += (double)gs[3 * P + o0 + xp];
        phi += (double)gs[4 * P + op + x];
        phi += (double)gs[5 * P + om + xm];
        phi += (double)gs[6 * P + om + xp];
        phi += (double)gs[7 * P + op + xp];
        phi += (double)gs[8 * P + op + xm];
      }
      const int lab = cd.labels ? (int)cd.labels[o0 + x] : 0;
#pragma unroll
      for (int r = 0; r < kMaxRegions; ++r)
        if (lab == r) acc[r] += phi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kMaxRegions; ++r) {
    double v = acc[r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][r] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxRegions) {
    double v = 0.0;
    for (int w = 0; w < BX / 32; ++w) v += red[w][threadIdx.x];
    if (threadIdx.x < nr) part[(int64_t)blockIdx.x * kMaxRegions + threadIdx.x] = v;
  }
}

// Phase volumes, pass 2: one warp per case.  For each region, lane l sums
// the partials of items l, l+32, ... in order, then the lanes are combined
// by a fixed shuffle tree: the result does not depend on timing.
template <typename T>
// With a history (slots > 1), the volumes of the state at step t + toff (t
// the device step clock) go to slot (t + toff) mod slots, `stride` doubles
// per slot.
__global__ void volume_final(const CaseDev<T>* __restrict__ cases,
                             const int* __restrict__ case_ids, int ncases,
                             const double* __restrict__ part, double* __restrict__ out,
                             const int64_t* __restrict__ t, int64_t toff, int64_t slots,
                             int64_t stride) {
  const int w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= ncases) return;
  const int c = case_ids ? case_ids[w] : w;
  if (slots > 1) out += ((*t + toff) % slots) * stride;
  const CaseDev<T>& cd = cases[c];
  for (int r = 0; r < cd.nregions; ++r) {
    double v = 0.0;
    for (int b = cd.item_begin + lane; b < cd.item_end; b += 32)
      v += part[(int64_t)b * kMaxRegions + r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[cd.vol_base + r] = v;
  }
}

// Step clock: t += n after a group of steps (read by the vortex flow).
static __global__ void clock_kernel(int64_t* t, int64_t n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t += n;
}
static __global__ void set_clock_kernel(int64_t* t, int64_t value) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t = value;
}

}  // namespace lbmk
