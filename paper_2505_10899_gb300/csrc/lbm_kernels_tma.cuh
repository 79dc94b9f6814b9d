// TMA-staged step kernel (grids whose width nx is a multiple of 16 bytes of
// the working type and at least 4).
//
// Work decomposition is that of step_kernel (a CTA owns a strip of BX
// columns and marches down `nrows` rows), but the populations reach shared
// memory through the bulk-copy engine instead of registers: for every row
// the CTA needs, lanes of warp 0 issue one cp.async.bulk per population plane
// for the pulled source row (r - c_iy) over columns [x0-4, x0+wact+4) (the
// periodic wrap in x splits a segment into at most three 16-byte aligned
// pieces) and two for phi*u of the previous step.  Completion is tracked by
// one mbarrier per stage with its transaction byte count.  S stages form a
// ring; rows are fetched S-1 ahead of the collision, so the consumer threads
// never wait on DRAM latency.  The halo columns of the phi/psi ring come from
// the same staged segments, without extra global loads.
//
// Every wait of the consumers is bounded (StepArgs::wait_cycles); on expiry
// the CTA raises kFlagTimeout, waits for its own copies still in flight
// (bounded by kWaitCycles, whatever wait_cycles is, so that no CTA leaves
// while a copy into its shared memory is pending) and returns.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_layout.h"
#include "lbm_node.cuh"
#include "lbm_tma.cuh"

namespace lbmk {


// D2Q9 velocity components (Eq. 19) as compile-time functions of i.
__host__ __device__ constexpr int cx_of(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

template <typename T, int BX, bool COUPLED, int MODE, int S>
struct TmaShape {
  static constexpr int SEG = BX + 8;                 // staged columns per plane
  static constexpr int NPL = COUPLED ? 18 : 9;        // population planes
  static constexpr int NJ = (MODE == kModeStep) ? 2 : 0;  // phi*u planes
  static constexpr int STAGE = NPL * SEG + NJ * BX;   // elements per stage
  static constexpr size_t STAGE_BYTES = (size_t)STAGE * sizeof(T);
  static constexpr size_t BAR_OFF = S * STAGE_BYTES;
  static constexpr size_t RING_OFF = (BAR_OFF + S * 8 + 127) / 128 * 128;
  static constexpr size_t VRED_OFF = RING_OFF + sizeof(Ring<T, BX>);
  static constexpr size_t SMEM_BYTES = VRED_OFF + (BX / 32) * sizeof(double);
  static_assert(STAGE_BYTES % 16 == 0, "stage must keep 16-byte alignment");
  static_assert((SEG * sizeof(T)) % 16 == 0, "plane segment must keep 16-byte alignment");
};

// The kernel body, for strips that hold a whole row (FROW: x0 = 0 and
// nx <= BX) or not; the kernel picks one per CTA, so that the strips of wide
// rows keep compile-time staged positions.
template <typename T, int BX, bool COUPLED, int MODE, int S, bool FROW>
__device__ __forceinline__ void tma_body(const StepArgs<T>& a) {
  using SH = TmaShape<T, BX, COUPLED, MODE, S>;
  constexpr int SEG = SH::SEG, NPL = SH::NPL, NJ = SH::NJ, STAGE = SH::STAGE;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const stages = reinterpret_cast<T*>(smem);
  uint64_t* const bars = reinterpret_cast<uint64_t*>(smem + SH::BAR_OFF);
  Ring<T, BX>& ring = *reinterpret_cast<Ring<T, BX>*>(smem + SH::RING_OFF);
  double* const vred = reinterpret_cast<double*>(smem + SH::VRED_OFF);

  const Item it = a.items[blockIdx.x];
  const CaseDev<T>* __restrict__ cdp = a.cases + it.c;
  const int nx = cdp->nx, ny = cdp->ny;
  const uint32_t P = (uint32_t)cdp->plane;
  const int x0 = it.x0, y0 = it.y0, nrows = it.nrows;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wact = min(BX, nx - x0);
  const bool act = tid < wact;
  const int xc = act ? x0 + tid : x0;

  const T* __restrict__ gs = cdp->g[a.parity];
  T* __restrict__ gd = cdp->g[a.parity ^ 1];
  const T* __restrict__ fs = COUPLED ? cdp->f[a.parity] : nullptr;
  T* __restrict__ fd = COUPLED ? cdp->f[a.parity ^ 1] : nullptr;
  const T* __restrict__ Js = cdp->J[a.parity];
  T* __restrict__ Jd = cdp->J[a.parity ^ 1];
  // FP32: low part of g_0, read at the own node only (not staged: the ring's
  // phi is the plain sum of the nine staged values; the exact rest
  // population in node_update uses it)
  const T* __restrict__ los = cdp->g0lo[a.parity];
  T* __restrict__ lod = cdp->g0lo[a.parity ^ 1];

  // halo columns of the phi/psi ring: local column -1 (thread 0) and wact
  // (thread BX-1), both inside the staged segments
  const bool hthr = (tid == 0) || (tid == BX - 1);
  const int hcol = (tid == 0) ? -1 : wact;
  const int hslot = (tid == 0) ? 0 : wact + 1;
  // A strip that holds the whole row (x0 = 0, nx <= BX) stages the row once,
  // columns 0..nx-1 at positions 4..nx+3, and reads the periodic neighbours
  // of its edge columns from the other end of the same copy; other strips
  // stage global column x0 - 4 + j at position j.  Staged position of local
  // column c + d, d = -1, 0, +1 (the pull sources of c_x = +1, 0, -1):
  constexpr bool frow = FROW;
  auto spos = [&](int c, int d) -> int {
    int j = c + d;
    if (frow) j = j < 0 ? j + nx : (j >= nx ? j - nx : j);
    return j + 4;
  };
  const int om = spos(tid, -1), o0 = spos(tid, 0), op = spos(tid, 1);
  const int hm = spos(hcol, -1), h0 = spos(hcol, 0), hp = spos(hcol, 1);

  const T xi = a.ph.xi;
  const bool do_vol = (MODE == kModeStep) && (a.vol_part != nullptr);
  double vacc = 0.0;
  const CaseK<T> K = case_consts<T, COUPLED>(a, cdp, xc);

  auto wrap = [&](int r) -> int { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };
  auto slot_of = [](int k) -> int { return (k + 1) % S; };
  auto parity_of = [](int k) -> uint32_t { return (uint32_t)(((k + 1) / S) & 1); };
  auto stage_of = [&](int k) -> T* { return stages + slot_of(k) * STAGE; };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Issue the bulk copies of local row k (k in [-1, nrows]); warp 0 only.
  // Rows -1 and nrows (the halo rows of the item) need the g planes only.
  auto issue = [&](int k) {
    const bool full = (k >= 0 && k < nrows);
    const int np = full ? NPL : 9;
    const int nj = full ? NJ : 0;
    T* st = stage_of(k);
    uint64_t* bar = &bars[slot_of(k)];
    // Staged column j holds global column (x0 - 4 + j) mod nx, j < wact + 8.
    // Where the strip touches the periodic edge of the row, the four columns
    // beyond it come from the other end of the row in a separate 16-byte
    // copy, made only for the planes that read them: on the left (x0 = 0)
    // the g planes with c_x >= 0 (the halo column -1 pulls from -1 - c_x)
    // and the f planes with c_x = +1 (column 0 pulls from -1); on the right
    // the mirror image.  That is 6 g and 3 f planes a side instead of 18.
    // Lane l copies plane l (g planes 0-8, then f planes 9-17); bit l of
    // kNeedL / kNeedR says whether it needs the left / right wrap columns.
    constexpr uint32_t kNeedL = 0x137u | (0x122u << 9);  // g: c_x >= 0; f: c_x = +1
    constexpr uint32_t kNeedR = 0x0DDu | (0x0C8u << 9);  // g: c_x <= 0; f: c_x = -1
    const bool lw = (x0 == 0), rw = (x0 + wact >= nx);
    uint32_t elems = (uint32_t)(np * (wact + 8) + nj * wact);
    if (frow) {  // one copy of the whole row per plane
      elems = (uint32_t)(np * nx + nj * wact);
    } else if (lw || rw) {  // the wrap columns that no plane reads are not copied
      const int nwrap = (full && COUPLED) ? 9 : 6;  // 6 g planes, + 3 f planes on full rows
      elems -= (uint32_t)((lw ? 4 * (np - nwrap) : 0) + (rw ? 4 * (np - nwrap) : 0));
    }
    if (lane == 0) mbar_arrive_expect_tx(bar, elems * (uint32_t)sizeof(T));
    __syncwarp();
    const int r = wrap(y0 + k);
    const uint32_t nn = (uint32_t)nx * (uint32_t)ny;
    // one bulk copy of n elements from position `first` of a plane (checked
    // build: the source range must lie in the plane's nodes and the target
    // in this stage; otherwise the copy is redirected, see lbm_check.h)
    auto copy = [&](T* dst, const T* plane, const T* buf, int64_t first, uint32_t n) {
      const bool ok = LBM_BOUND(a.flags, first, nn) && LBM_BOUND(a.flags, first + n - 1, nn) &&
                      LBM_BOUND(a.flags, (dst - st) + n - 1, STAGE);
      bulk_g2s(ok ? dst : st, ok ? plane + first : buf, n * sizeof(T), bar);
    };
    if (lane < np) {
      const int i = lane < 9 ? lane : lane - 9;
      const T* buf = lane < 9 ? gs : fs;
      const T* plane = buf + (size_t)i * P;
      const int64_t row = (int64_t)wrap(r - cy_of(i)) * nx;  // pull: source row r - c_iy
      T* dst = st + lane * SEG;
      int j = 0, g0, len;
      if (frow) {
        copy(dst + 4, plane, buf, row, (uint32_t)nx);
      } else {
        if (lw) {
          if ((kNeedL >> lane) & 1u) copy(dst, plane, buf, row + (nx - 4), 4);
          j = 4;
          g0 = 0;
          len = wact;
        } else {
          g0 = x0 - 4;
          len = wact + 4;
        }
        if (!rw) {
          copy(dst + j, plane, buf, row + g0, (uint32_t)(len + 4));
        } else {
          copy(dst + j, plane, buf, row + g0, (uint32_t)len);
          if ((kNeedR >> lane) & 1u) copy(dst + j + len, plane, buf, row, 4);
        }
      }
    } else if (lane >= NPL && lane < NPL + nj) {
      const int q = lane - NPL;
      copy(st + NPL * SEG + q * BX, Js + (size_t)q * P, Js, (int64_t)r * nx + x0, (uint32_t)wact);
    }
  };

  // g of a local column from a staged row, given the staged positions of
  // its left, own and right neighbour columns
  auto staged_g = [&](const T* st, int pm, int p0, int pp, T G[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
      G[i] = st[i * SEG + (cx_of(i) == 1 ? pm : (cx_of(i) == -1 ? pp : p0))];
  };

  // phi and psi of local row k into the ring (row k must have landed)
  auto put_row = [&](int k) {
    const T* st = stage_of(k);
    const int s = (k + 4) & 3;
    T G[9];
    if (act) {
      staged_g(st, om, o0, op, G);
      const T phi = sum9(G);
      ring.put(s, tid + 1, phi, psi_of(phi, xi));
    }
    if (hthr) {
      staged_g(st, hm, h0, hp, G);
      const T phi = sum9(G);
      ring.put(s, hslot, phi, psi_of(phi, xi));
    }
  };

  // ---- prologue: rows -1 .. S-2 in flight; phi of rows -1 and 0 ----------
  if (warp == 0) {
    const int last = min(S - 2, nrows);
    for (int k = -1; k <= last; ++k) issue(k);
  }
  // rows up to `landed` have been seen complete by this thread
  int landed = -2;
  const long long lim = a.wait_cycles;
  bool bad = !mbar_wait_bounded(&bars[slot_of(-1)], parity_of(-1), lim);
  if (!bad) {
    landed = -1;
    put_row(-1);
  }
  bad = bad || !mbar_wait_bounded(&bars[slot_of(0)], parity_of(0), lim);
  if (!bad) {
    landed = 0;
    put_row(0);
  }

  int issued_last = min(S - 2, nrows);  // highest row issued so far
  // FP32: low part of g_0 of the own node, loaded one row ahead
  auto lo_of = [&](int k) -> T {
    if (sizeof(T) != 4 || !act || k >= nrows) return T(0);
    const uint32_t at = (uint32_t)wrap(y0 + k) * (uint32_t)nx + (uint32_t)xc;
    return LBM_BOUND(a.flags, at, (uint32_t)nx * (uint32_t)ny) ? __ldg(los + at) : T(0);
  };
  T lo_next = lo_of(0);
  for (int k = 0; k < nrows; ++k) {
    T glo = lo_next;
    lo_next = lo_of(k + 1);
    // row k+1 (own row or the halo row below the item) into the ring
    bad = bad || !mbar_wait_bounded(&bars[slot_of(k + 1)], parity_of(k + 1), lim);
    if (!bad) {
      landed = k + 1;
      put_row(k + 1);
    }
    if (__syncthreads_or(bad)) {
      // a wait gave up: report, wait for every row issued but not yet seen
      // complete (its copies write into this CTA's shared memory), leave
      if (tid == 0) atomicOr(a.flags, kFlagTimeout);
      for (int m = landed + 1; m <= issued_last; ++m)
        mbar_wait_bounded(&bars[slot_of(m)], parity_of(m), kWaitCycles);
      return;
    }
    // the stage of row k-1 is free: refill it with row k-1+S
    const int nxt = k - 1 + S;
    if (nxt <= nrows) {
      if (warp == 0) {
        fence_proxy_async_smem();
        issue(nxt);
      }
      issued_last = nxt;
    }
    if (act) {
      const T* st = stage_of(k);
      T F[9], G[9];
      staged_g(st, om, o0, op, G);
      if (COUPLED) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
          F[i] = st[(9 + i) * SEG + (cx_of(i) == 1 ? om : (cx_of(i) == -1 ? op : o0))];
      }
      T jpx = T(0), jpy = T(0);
      if (MODE == kModeStep) {
        jpx = st[NPL * SEG + tid];
        jpy = st[NPL * SEG + BX + tid];
      }
      const int y = wrap(y0 + k);
      const uint32_t node = (uint32_t)y * (uint32_t)nx + (uint32_t)xc;
      const Stencil<T> Sn = read_stencil(ring, k, tid + 1);
      // fused volume: the plain phi (the low part of g_0, below 2^-24 g_0 per
      // node, is left out here; lbm_volume counts it)
      if (do_vol) vacc += (double)Sn.p;
      const NodeOut<T> o = node_update<T, COUPLED, MODE>(a.ph, K, F, G, glo, jpx, jpy, Sn, y);
      if (MODE == kModeStep) {
        store_node<T, COUPLED>(fd, gd, Jd, lod, P, node, F, G, glo, o, a.flags,
                               (uint32_t)nx * (uint32_t)ny);
        if (!isfinite(Sn.p + o.ux + o.uy + o.p)) atomicOr(a.flags, kFlagNonFinite);
      } else if (LBM_BOUND(a.flags, node, (uint32_t)nx * (uint32_t)ny)) {
        a.out_phi[node] = (double)Sn.p;
        a.out_ux[node] = (double)o.ux;
        a.out_uy[node] = (double)o.uy;
        a.out_p[node] = (double)o.p;
      }
    }
  }

  if (do_vol) {
    for (int o = 16; o > 0; o >>= 1) vacc += __shfl_down_sync(0xffffffffu, vacc, o);
    if (lane == 0) vred[warp] = vacc;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int w = 0; w < BX / 32; ++w) v += vred[w];
      a.vol_part[(int64_t)blockIdx.x * kMaxRegions] = v;
    }
  }
}

// CTAs per SM the FP32 kernel is register-capped for (its shared memory
// allows about as many): about 80 registers a thread in every width.
template <typename T, int BX>
constexpr int tma_min_blocks() {
  return sizeof(T) != 4 ? 1
         : BX == 128    ? 6
         : BX == 96     ? 6
         : BX == 192    ? 4
         : BX == 256    ? 3
                        : 1;
}

template <typename T, int BX, bool COUPLED, int MODE, int S>
__global__ void __launch_bounds__(BX, (tma_min_blocks<T, BX>()))
    step_kernel_tma(const StepArgs<T> a) {
  const Item it = a.items[blockIdx.x];
  if (it.x0 == 0 && a.cases[it.c].nx <= BX)
    tma_body<T, BX, COUPLED, MODE, S, true>(a);
  else
    tma_body<T, BX, COUPLED, MODE, S, false>(a);
}

}  // namespace lbmk
