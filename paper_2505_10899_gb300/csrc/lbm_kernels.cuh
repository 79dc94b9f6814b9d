// Register-pipelined step kernel: works for every grid size (the general
// path; grids whose width is a multiple of 16 bytes run the TMA-staged kernel
// of lbm_kernels_tma.cuh instead).
//
// One CTA owns a strip of BX columns and marches down `nrows` rows of it
// (a work item).  Per row it pulls the 18 populations of its nodes
// (Eqs. 20 and 30, left-hand sides), forms phi = sum g (Eq. 35) and the
// level-set variable psi (Eq. 37), keeps phi and psi of the last four rows
// in a shared-memory ring with a one-column halo on each side, and collides
// row k once rows k-1, k, k+1 are in the ring.  Loads of row k+2 are issued
// before the collision of row k so that their latency overlaps the
// arithmetic (two-row software pipeline, one __syncthreads per row).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_layout.h"
#include "lbm_check.h"
#include "lbm_node.cuh"

namespace lbmk {

// Pull the 9 populations of node (x, row) from a buffer: value i comes from
// (x - c_ix, row - c_iy).  o0/om/op are the offsets of rows row, row-1,
// row+1 (periodic), xm/xp the columns x-1, x+1 (periodic).  Eq. 19 order:
// c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
// Global load: read-only path, or L2-coherent (bypassing L1) when the data
// may have been written by other CTAs of the same launch (persistent kernel).
template <bool COHERENT, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if (COHERENT) return __ldcg(p);
  return __ldg(p);
}

template <bool COHERENT = false, typename T>
__device__ __forceinline__ void pull9(const T* __restrict__ b, uint32_t P,
                                      uint32_t o0, uint32_t om, uint32_t op,
                                      uint32_t x, uint32_t xm, uint32_t xp, T v[9],
                                      int32_t* flags = nullptr) {
  // 32-bit element offsets: a buffer of 9 planes holds < 2^31 elements
#ifdef LBM_CHECK_BOUNDS
  const uint32_t off[9] = {o0 + x,           P + o0 + xm,      2u * P + om + x,
                           3u * P + o0 + xp, 4u * P + op + x,  5u * P + om + xm,
                           6u * P + om + xp, 7u * P + op + xp, 8u * P + op + xm};
#pragma unroll
  for (int i = 0; i < 9; ++i)
    v[i] = LBM_BOUND(flags, off[i], 9ull * P) ? ld<COHERENT>(b + off[i]) : T(0);
#else
  (void)flags;
  v[0] = ld<COHERENT>(b + (o0 + x));
  v[1] = ld<COHERENT>(b + (P + o0 + xm));
  v[2] = ld<COHERENT>(b + (2u * P + om + x));
  v[3] = ld<COHERENT>(b + (3u * P + o0 + xp));
  v[4] = ld<COHERENT>(b + (4u * P + op + x));
  v[5] = ld<COHERENT>(b + (5u * P + om + xm));
  v[6] = ld<COHERENT>(b + (6u * P + om + xp));
  v[7] = ld<COHERENT>(b + (7u * P + op + xp));
  v[8] = ld<COHERENT>(b + (8u * P + op + xm));
#endif
}

// The same pull at a row next to a wall (bot: row 0, top: row ny-1):
// halfway bounce-back -- a population that would come from beyond the wall is
// the node's own post-collision population in the opposite direction (the
// moving-wall term of f is added by the caller, once phi is known).
template <bool COHERENT = false, typename T>
__device__ __forceinline__ void pull9w(const T* __restrict__ b, uint32_t P, uint32_t o0,
                                       uint32_t om, uint32_t op, uint32_t x, uint32_t xm,
                                       uint32_t xp, bool bot, bool top, T v[9],
                                       int32_t* flags = nullptr) {
#ifdef LBM_CHECK_BOUNDS
  const uint32_t off[9] = {o0 + x,
                           P + o0 + xm,
                           bot ? 4u * P + o0 + x : 2u * P + om + x,
                           3u * P + o0 + xp,
                           top ? 2u * P + o0 + x : 4u * P + op + x,
                           bot ? 7u * P + o0 + x : 5u * P + om + xm,
                           bot ? 8u * P + o0 + x : 6u * P + om + xp,
                           top ? 5u * P + o0 + x : 7u * P + op + xp,
                           top ? 6u * P + o0 + x : 8u * P + op + xm};
#pragma unroll
  for (int i = 0; i < 9; ++i)
    v[i] = LBM_BOUND(flags, off[i], 9ull * P) ? ld<COHERENT>(b + off[i]) : T(0);
#else
  (void)flags;
  v[0] = ld<COHERENT>(b + (o0 + x));
  v[1] = ld<COHERENT>(b + (P + o0 + xm));
  v[3] = ld<COHERENT>(b + (3u * P + o0 + xp));
  v[2] = ld<COHERENT>(b + (bot ? 4u * P + o0 + x : 2u * P + om + x));
  v[5] = ld<COHERENT>(b + (bot ? 7u * P + o0 + x : 5u * P + om + xm));
  v[6] = ld<COHERENT>(b + (bot ? 8u * P + o0 + x : 6u * P + om + xp));
  v[4] = ld<COHERENT>(b + (top ? 2u * P + o0 + x : 4u * P + op + x));
  v[7] = ld<COHERENT>(b + (top ? 5u * P + o0 + x : 7u * P + op + xp));
  v[8] = ld<COHERENT>(b + (top ? 6u * P + o0 + x : 8u * P + op + xm));
#endif
}

// Moving-wall term of the bounced f (walls along x at u_bot below row 0 and
// u_top above row ny-1): f_i += 2 w_i rho (c_i . u_w)/c_s^2 = rho c_ix u_w / 6
// for the diagonal populations entering from the wall (w_i = 1/36).
template <typename T>
__device__ __forceinline__ void wall_momentum(T F[9], T rho, bool bot, bool top, T u_bot,
                                              T u_top) {
  if (bot) {
    const T d = rho * u_bot * T(1.0 / 6.0);
    F[5] += d;  // c = (1, 1)
    F[6] -= d;  // c = (-1, 1)
  }
  if (top) {
    const T d = rho * u_top * T(1.0 / 6.0);
    F[7] -= d;  // c = (-1, -1)
    F[8] += d;  // c = (1, -1)
  }
}

// CTA reduction of the fused phase volume: warp shuffles, then warps in order.
template <int BX>
__device__ __forceinline__ void write_volume_partial(double vacc, double* vred, double* out) {
  for (int o = 16; o > 0; o >>= 1) vacc += __shfl_down_sync(0xffffffffu, vacc, o);
  if ((threadIdx.x & 31) == 0) vred[threadIdx.x >> 5] = vacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < BX / 32; ++w) v += vred[w];
    *out = v;
  }
}

// ---------------------------------------------------------------------------
//   COUPLED: f and g (true) or g only with the prescribed vortex (false).
//   MODE:    kModeStep collides and stores; kModeFields writes phi, u, p.
// ---------------------------------------------------------------------------
template <typename T, int BX, bool COUPLED, int MODE, bool COHERENT>
__device__ __forceinline__ void step_item(const StepArgs<T>& a, int item, Ring<T, BX>& ring,
                                          double* vred) {
  const Item it = a.items[item];
  const CaseDev<T>* __restrict__ cdp = a.cases + it.c;
  const int nx = cdp->nx, ny = cdp->ny;
  const uint32_t P = (uint32_t)cdp->plane;
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
  const T* __restrict__ Js = cdp->J[a.parity];
  T* __restrict__ Jd = cdp->J[a.parity ^ 1];
  // FP32: low part of g_0 at the own node (null in FP64)
  const T* __restrict__ los = cdp->g0lo[a.parity];
  T* __restrict__ lod = cdp->g0lo[a.parity ^ 1];
  constexpr bool LO = sizeof(T) == 4;

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

  const T xi = a.ph.xi;
  const bool do_vol = (MODE == kModeStep) && (a.vol_part != nullptr);
  double vacc = 0.0;
  const CaseK<T> K = case_consts<T, COUPLED>(a, cdp, xc);

  auto rowoff = [&](int r) -> uint32_t { return (uint32_t)r * (uint32_t)nx; };
  const uint32_t nn = (uint32_t)nx * (uint32_t)ny;  // nodes of the case (checked build)
  // row index for r in [-1, ny]: periodic, or with walls the mirrored ghost
  // row (rows -1 and ny only feed phi and psi to the stencils)
  const bool walls = cdp->walls != 0;
  auto wrap = [&](int r) -> int {
    if (walls) return r < 0 ? 0 : (r >= ny ? ny - 1 : r);
    return r < 0 ? r + ny : (r >= ny ? r - ny : r);
  };
  auto at_bot = [&](int rr) -> bool { return walls && rr == 0; };
  auto at_top = [&](int rr) -> bool { return walls && rr == ny - 1; };

  // register sets of the pipeline: rows k (current), k+1 (next), k+2 (fetch)
  struct Regs {
    T F[9], G[9], J[2], lo;
  };
  Regs Rc, Rn, Rq;
  T hq[9];  // halo-column g of the row being fetched

  auto fetch_full = [&](int r, Regs& R) {
    const int rr = wrap(r);
    const uint32_t o0 = rowoff(rr), om = rowoff(rr == 0 ? ny - 1 : rr - 1),
                   op = rowoff(rr == ny - 1 ? 0 : rr + 1);
    const bool bt = at_bot(rr), tp = at_top(rr);
    if (bt || tp) {  // a wall row (uniform over the CTA)
      pull9w<COHERENT>(gs, P, o0, om, op, xc, xm, xp, bt, tp, R.G, a.flags);
      if (COUPLED) pull9w<COHERENT>(fs, P, o0, om, op, xc, xm, xp, bt, tp, R.F, a.flags);
    } else {
      pull9<COHERENT>(gs, P, o0, om, op, xc, xm, xp, R.G, a.flags);
      if (COUPLED) pull9<COHERENT>(fs, P, o0, om, op, xc, xm, xp, R.F, a.flags);
    }
#ifdef LBM_CHECK_BOUNDS
    const bool own_ok = LBM_BOUND(a.flags, o0 + xc, nn);
#else
    constexpr bool own_ok = true;
#endif
    R.lo = (LO && own_ok) ? ld<COHERENT>(los + (o0 + xc)) : T(0);
    if (MODE == kModeStep) {  // phi*u of the previous step at the own node
      R.J[0] = own_ok ? ld<COHERENT>(Js + (o0 + xc)) : T(0);
      R.J[1] = own_ok ? ld<COHERENT>(Js + (P + o0 + xc)) : T(0);
    }
  };
  auto fetch_g = [&](int r, Regs& R) {
    const int rr = wrap(r);
    const uint32_t o0 = rowoff(rr), om = rowoff(rr == 0 ? ny - 1 : rr - 1),
                   op = rowoff(rr == ny - 1 ? 0 : rr + 1);
    if (at_bot(rr) || at_top(rr))
      pull9w<COHERENT>(gs, P, o0, om, op, xc, xm, xp, at_bot(rr), at_top(rr), R.G, a.flags);
    else
      pull9<COHERENT>(gs, P, o0, om, op, xc, xm, xp, R.G, a.flags);
  };
  auto fetch_halo = [&](int r, T H[9]) {
    const int rr = wrap(r);
    const uint32_t o0 = rowoff(rr), om = rowoff(rr == 0 ? ny - 1 : rr - 1),
                   op = rowoff(rr == ny - 1 ? 0 : rr + 1);
    if (at_bot(rr) || at_top(rr))
      pull9w<COHERENT>(gs, P, o0, om, op, hc, hcm, hcp, at_bot(rr), at_top(rr), H, a.flags);
    else
      pull9<COHERENT>(gs, P, o0, om, op, hc, hcm, hcp, H, a.flags);
  };
  // write phi/psi of local row k (k >= -1) into the ring.  phi is the plain
  // sum of the nine pulled values (FP32: the low part of g_0 enters only the
  // rest-population update, as in the bulk-copy kernel)
  auto put_row = [&](int k, const T G[9], const T H[9]) {
    const int s = (k + 4) & 3;
    if (act) {
      const T phi = sum9(G);
      ring.put(s, tid + 1, phi, psi_of(phi, xi));
    }
    if (hthr) {
      const T phi = sum9(H);
      ring.put(s, hslot, phi, psi_of(phi, xi));
    }
  };

  // --- prologue: rows -1 (phi only), 0 and 1 -------------------------------
  fetch_g(y0 - 1, Rq);
  if (hthr) fetch_halo(y0 - 1, hq);
  put_row(-1, Rq.G, hq);
  fetch_full(y0, Rc);
  if (hthr) fetch_halo(y0, hq);
  put_row(0, Rc.G, hq);
  if (nrows > 1) {
    fetch_full(y0 + 1, Rn);
  } else {
    fetch_g(y0 + 1, Rn);
  }
  if (hthr) fetch_halo(y0 + 1, hq);
  put_row(1, Rn.G, hq);
  __syncthreads();

  // One pipeline stage: collide local row k from C while the loads of row
  // k+2 land in Q.  Called three times per trip with the register sets
  // rotated, so no copies are needed between rows.
  auto stage = [&](int k, Regs& C, Regs& Q) {
    // loads of row k+2: full if it is an own row, phi-only if it is the halo
    // row below the item, nothing beyond
    const bool q_full = (k + 2 < nrows);
    const bool q_any = (k + 2 <= nrows);
    if (q_full) {
      fetch_full(y0 + k + 2, Q);
    } else if (q_any) {
      fetch_g(y0 + k + 2, Q);
    }
    if (q_any && hthr) fetch_halo(y0 + k + 2, hq);

    if (act) {
      const int y = wrap(y0 + k);
      const Stencil<T> S = read_stencil(ring, k, tid + 1);
      if (do_vol) vacc += (double)S.p;
      if (COUPLED && walls && (y == 0 || y == ny - 1))
        wall_momentum(C.F, K.rho_g + S.p * K.drho, y == 0, y == ny - 1, cdp->u_bot,
                      cdp->u_top);
      const NodeOut<T> o =
          node_update<T, COUPLED, MODE>(a.ph, K, C.F, C.G, C.lo, C.J[0], C.J[1], S, y);
      const uint32_t node = rowoff(y) + (uint32_t)xc;
      if (MODE == kModeStep) {
        store_node<T, COUPLED>(fd, gd, Jd, lod, P, node, C.F, C.G, C.lo, o, a.flags, nn);
        if (!isfinite(S.p + o.ux + o.uy + o.p)) atomicOr(a.flags, kFlagNonFinite);
      } else if (LBM_BOUND(a.flags, node, nn)) {
        a.out_phi[node] = (double)S.p;
        a.out_ux[node] = (double)o.ux;
        a.out_uy[node] = (double)o.uy;
        a.out_p[node] = (double)o.p;
      }
    }
    if (q_any) put_row(k + 2, Q.G, hq);
    __syncthreads();
  };

  for (int k = 0; k < nrows; k += 3) {
    stage(k, Rc, Rq);
    if (k + 1 < nrows) stage(k + 1, Rn, Rc);
    if (k + 2 < nrows) stage(k + 2, Rq, Rn);
  }

  if (do_vol) write_volume_partial<BX>(vacc, vred, a.vol_part + (int64_t)item * kMaxRegions);
  __syncthreads();  // the ring is reused by the next item of a persistent CTA
}

template <typename T, int BX, bool COUPLED, int MODE>
__global__ void __launch_bounds__(BX) step_kernel(const StepArgs<T> a) {
  __shared__ Ring<T, BX> ring;
  __shared__ double vred[BX / 32];
  step_item<T, BX, COUPLED, MODE, false>(a, blockIdx.x, ring, vred);
}

// ---------------------------------------------------------------------------
// Persistent variant for small grids: one cooperative launch advances nsteps
// steps.  Every CTA takes the items blockIdx.x, blockIdx.x + gridDim.x, ...
// of each step, then all CTAs meet at a grid barrier before the next step
// reads what the previous one wrote (loads are L2-coherent, see ld()).  With
// flip = 0 the source buffer stays the same for every step (autotuning
// trials: the state is not changed).
// The barrier is a counter and a generation word in the workspace header;
// its wait is bounded and raises kFlagTimeout when it expires.
// ---------------------------------------------------------------------------
struct GridBar {
  unsigned int* count;
  unsigned int* gen;
};

__device__ __forceinline__ bool grid_barrier(const GridBar& b, int32_t* flags,
                                             long long wait_cycles) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = *(volatile unsigned int*)b.gen;
    __threadfence();  // this CTA's stores are visible before it arrives
    const unsigned int arrived = atomicAdd(b.count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*(volatile unsigned int*)b.gen == g) {
        if (clock64() - t0 > wait_cycles) {
          atomicOr(flags, kFlagTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T, int BX, bool COUPLED>
__global__ void __launch_bounds__(BX) step_kernel_persistent(const StepArgs<T> a, int n_items,
                                                             int nsteps, int flip, GridBar bar) {
  __shared__ Ring<T, BX> ring;
  __shared__ double vred[BX / 32];
  for (int s = 0; s < nsteps; ++s) {
    StepArgs<T> as = a;
    if (flip) {
      as.parity = a.parity ^ (s & 1);
      as.t_off = a.t_off + s;
    }
    for (int item = blockIdx.x; item < n_items; item += gridDim.x)
      step_item<T, BX, COUPLED, kModeStep, true>(as, item, ring, vred);
    if (s + 1 < nsteps && !grid_barrier(bar, a.flags, a.wait_cycles)) return;
  }
}

}  // namespace lbmk
