// Strip-tiled bulk-copy variant of the three-dimensional step kernel (FP32
// arithmetic, FP32 or FP16 population storage) for boxes whose nx is a
// multiple of the strip width BX and at least 2 BX.  Same per-node
// arithmetic as step3_kernel (node3, the same stencils and phase-A sums); the
// difference is how the pulled values reach the threads.
//
// A CTA owns a BX x BY column tile (x0 .. x0+BX-1, y0 .. y0+BY-1) and marches
// along z over `zc` planes, like step3_kernel, so several CTAs share an SM.
// Every value it reads for plane z arrives in shared memory by 1-D bulk
// copies (cp.async.bulk) of row segments, one segment per thread of the CTA,
// NST-1 planes ahead, completed on one mbarrier per stage:
//   - f_i: row (y - c_iy, z - c_iz) of plane i for each of the BY rows, over
//     columns x0 .. x0+BX-1 shifted by -c_ix;
//   - phi*u: rows (y, z), columns x0 .. x0+BX-1;
//   - the 7 g (and the low part of g_0) pulled to the BY + 2 rows y0-1 ..
//     y0+BY of plane z+1 over the BX + 2 columns x0-1 .. x0+BX, for phase A
//     (phi = sum g, Eq. 35; psi, Eq. 37) into a 4-plane ring of (phi, psi)
//     from which the D3Q19 stencils of Sec. 3.2 are read.
// A staged row starts one 16-byte chunk (ES stored values, or ET values of
// the arithmetic type for the g_0 rows) left of x0 and ends one chunk right
// of x0+BX-1, so that the pull's one-column shift and the halo
// columns are index offsets inside it; a segment copies only the chunks its
// population reads (no left chunk for c_x = -1 rows of f, and so on).  Where a
// segment crosses the periodic edge x = 0 or x = nx it is split there (nx is
// a multiple of the chunk, so every piece stays 16-byte aligned).  The pulled
// g of a thread's own node stay in registers from phase A (plane z+1) to the
// update of plane z+1.
//
// Every wait is bounded (wait_cycles); on expiry the CTA raises
// kFlagTimeout3, waits (bounded by lbmk::kWaitCycles) for its own copies in
// flight and returns.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm3_bulk.cuh"
#include "lbm3_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbmk3 {

template <typename T, typename S, int BX, int BY, int NST>
struct StripShape {
  static constexpr int ES = 16 / (int)sizeof(S);  // elements of one 16-byte chunk, storage type
  static constexpr int ET = 16 / (int)sizeof(T);  // the same for the arithmetic type
  static constexpr int WS = BX + 2 * ES;          // staged S row: x0-ES .. x0+BX+ES-1
  static constexpr int WT = BX + 2 * ET;          // staged g_0 row: x0-ET .. x0+BX+ET-1
  static constexpr int NR = BY + 2;               // phase-A rows (with the halo rows)
  static constexpr int RW = BX + 2;               // ring columns (with the halo columns)
  static constexpr size_t F_OFF = 0;                                         // [19][BY][WS] S
  static constexpr size_t GM_OFF = F_OFF + (size_t)19 * BY * WS * sizeof(S);  // [6][NR][WS] S
  static constexpr size_t J_OFF = GM_OFF + (size_t)6 * NR * WS * sizeof(S);   // [3][BY][BX] T
  static constexpr size_t G0_OFF = J_OFF + (size_t)3 * BY * BX * sizeof(T);   // [2][NR][WT] T
  static constexpr size_t STAGE_BYTES = G0_OFF + (size_t)2 * NR * WT * sizeof(T);
  static constexpr size_t BAR_OFF = NST * STAGE_BYTES;
  static constexpr size_t RING_OFF = (BAR_OFF + NST * 8 + 127) / 128 * 128;
  static constexpr size_t RING_BYTES = (size_t)4 * NR * RW * sizeof(typename N3<T>::pair);
  static constexpr size_t SMEM_BYTES = RING_OFF + RING_BYTES;
  static constexpr int NQ = 22 * BY + 8 * NR;  // row segments per stage
  // bytes one stage receives: five f rows per tile row carry a left chunk and
  // five a right chunk; of the six g movers one has no left chunk and one no
  // right chunk; g_0 and its low part carry both
  static constexpr uint32_t TX_BYTES =
      (uint32_t)(((19 * BX + 10 * ES) * BY + (6 * BX + 10 * ES) * NR) * sizeof(S) +
                 (3 * BX * BY + 2 * (BX + 2 * ET) * NR) * sizeof(T));
  static constexpr int NH = 2 * RW + 2 * BY;  // halo ring of the tile
  static_assert(BX % ES == 0 && BX % ET == 0, "strip width must be whole 16-byte chunks");
  static_assert(ES >= 2 && ET >= 2, "a chunk must cover the pull shift and the halo column");
  static_assert(STAGE_BYTES % 16 == 0 && GM_OFF % 16 == 0 && J_OFF % 16 == 0 &&
                    G0_OFF % 16 == 0 && (WS * sizeof(S)) % 16 == 0 && (WT * sizeof(T)) % 16 == 0,
                "stage regions and rows must keep 16-byte alignment");
};

template <typename T, typename S, int BX, int BY, int NST>
constexpr size_t strip_smem_bytes() {
  return StripShape<T, S, BX, BY, NST>::SMEM_BYTES;
}

template <typename T, typename S, int BX, int BY, int NST, int MINB>
__global__ void __launch_bounds__(BX* BY, MINB)
    step3_strip_kernel(const Args3<T, S> a, long long wait_cycles) {
  using SH = StripShape<T, S, BX, BY, NST>;
  using Pair = typename N3<T>::pair;
  constexpr int NR = SH::NR, RW = SH::RW, ES = SH::ES, ET = SH::ET, WS = SH::WS, WT = SH::WT;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* const bars = reinterpret_cast<uint64_t*>(smem + SH::BAR_OFF);
  Pair(*const ring)[NR][RW] = reinterpret_cast<Pair(*)[NR][RW]>(smem + SH::RING_OFF);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX, warp = tid >> 5, lane = tid & 31;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t P = a.plane;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int zb = blockIdx.z * a.zc;
  const int ze = min(zb + a.zc, nz);
  const int nplanes = ze - zb;
  const bool act = y0 + ty < ny;  // nx is a multiple of BX: every column is in the box
  // periodic wrap of row and plane indices (any number of periods: boxes may
  // be thinner than the rows and planes a CTA touches)
  auto wrapy = [&](int v) { return ((v % ny) + ny) % ny; };
  auto wrapz = [&](int v) { return ((v % nz) + nz) % nz; };

  const int par = a.parity, dst = par ^ 1;
  const S* __restrict__ fs = a.f[par];
  const S* __restrict__ gms = a.g[par];
  const T* __restrict__ g0s = a.g0[par];
  const T* __restrict__ g0ls = a.g0lo[par];
  const T* __restrict__ js = a.J[par];
  S* __restrict__ fd = a.f[dst];
  S* __restrict__ gmd = a.g[dst];
  T* __restrict__ g0d = a.g0[dst];
  T* __restrict__ g0ld = a.g0lo[dst];
  T* __restrict__ jd = a.J[dst];

  auto stage = [&](int k) { return smem + (size_t)(k % NST) * SH::STAGE_BYTES; };
  auto sF = [&](unsigned char* st, int i, int r) {
    return reinterpret_cast<S*>(st + SH::F_OFF) + ((size_t)i * BY + r) * WS;
  };
  auto sGM = [&](unsigned char* st, int m, int r) {  // mover m = 1..6, phase-A row r
    return reinterpret_cast<S*>(st + SH::GM_OFF) + ((size_t)(m - 1) * NR + r) * WS;
  };
  auto sJ = [&](unsigned char* st, int c, int r) {
    return reinterpret_cast<T*>(st + SH::J_OFF) + ((size_t)c * BY + r) * BX;
  };
  auto sG0 = [&](unsigned char* st, int h, int r) {  // h = 0: g_0, 1: its low part
    return reinterpret_cast<T*>(st + SH::G0_OFF) + ((size_t)h * NR + r) * WT;
  };
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) lbmk::mbar_init(&bars[s], 1);
    lbmk::fence_mbar_init();
  }

  // Row segments of a stage (local plane k, plane z = zb + k): f and phi*u of
  // the BY rows of plane z, the g of the NR phase-A rows of plane z + 1.
  // Thread q < NQ copies segment q of every stage.  Its segment is described
  // once per CTA (only the plane changes from stage to stage): piece A's
  // global address without the plane offset, its byte offset inside a stage,
  // its size, the plane it reads (0..3: z-1 .. z+2) and the element size;
  // and, where the segment crosses x = 0 or x = nx (nx >= 2 BX: at most one
  // of the two), piece B's address relative to A, stage offset and size.
  constexpr int NT = BX * BY;
  static_assert(SH::NQ <= NT, "one row segment per thread at most");
  __shared__ uint4 qdesc[2][NT];
  if (tid < SH::NQ) {
    const int q = tid;
    const unsigned char* base;
    int rsel, dz, xa, len, esz;
    size_t dst;
    if (q < 19 * BY) {  // f_i of tile row r: row y0 + r - c_iy, plane z - c_iz
      const int i = q / BY, r = q % BY, cx = bcx(i);
      const int lp = cx == 1 ? ES : 0, rp = cx == -1 ? ES : 0;
      base = reinterpret_cast<const unsigned char*>(fs + (int64_t)i * P);
      rsel = r - bcy(i), dz = 1 - bcz(i), xa = x0 - lp, len = BX + lp + rp, esz = sizeof(S);
      dst = SH::F_OFF + (((size_t)i * BY + r) * WS + (ES - lp)) * sizeof(S);
    } else if (q < 19 * BY + 6 * NR) {  // mover m of phase-A row r: row y0-1+r-c_my, plane z+1-c_mz
      const int u = q - 19 * BY, m = u / NR + 1, r = u % NR, cx = bcx(m);
      const int lp = cx == -1 ? 0 : ES, rp = cx == 1 ? 0 : ES;
      base = reinterpret_cast<const unsigned char*>(gms + (int64_t)(m - 1) * P);
      rsel = r - 1 - bcy(m), dz = 2 - bcz(m), xa = x0 - lp, len = BX + lp + rp, esz = sizeof(S);
      dst = SH::GM_OFF + (((size_t)(m - 1) * NR + r) * WS + (ES - lp)) * sizeof(S);
    } else if (q < 22 * BY + 6 * NR) {  // phi*u: row y0 + r, plane z
      const int u = q - 19 * BY - 6 * NR, c = u / BY, r = u % BY;
      base = reinterpret_cast<const unsigned char*>(js + (int64_t)c * P);
      rsel = r, dz = 1, xa = x0, len = BX, esz = sizeof(T);
      dst = SH::J_OFF + ((size_t)c * BY + r) * BX * sizeof(T);
    } else {  // g_0 (h = 0) and its low part: row y0 - 1 + r, plane z + 1
      const int u = q - 22 * BY - 6 * NR, h = u / NR, r = u % NR;
      base = reinterpret_cast<const unsigned char*>(h == 0 ? g0s : g0ls);
      rsel = r - 1, dz = 2, xa = x0 - ET, len = BX + 2 * ET, esz = sizeof(T);
      dst = SH::G0_OFF + ((size_t)h * NR + r) * WT * sizeof(T);
    }
    const unsigned char* row = base + (size_t)wrapy(y0 + rsel) * (size_t)nx * esz;
    int xA = xa, nA = len, xB = 0, nB = 0;
    size_t dB = 0;
    if (xa < 0) {  // the left chunk comes from the end of the row
      xB = nx + xa, nB = -xa, dB = dst;
      dst += (size_t)nB * esz;
      xA = 0, nA = len - nB;
    } else if (xa + len > nx) {  // the right chunk comes from the start of the row
      nA = nx - xa, nB = len - nA, xB = 0;
      dB = dst + (size_t)nA * esz;
    }
    const uint64_t srcA = reinterpret_cast<uint64_t>(row + (size_t)xA * esz);
    qdesc[0][q] = make_uint4((uint32_t)srcA, (uint32_t)(srcA >> 32), (uint32_t)dst,
                             (uint32_t)(nA * esz) | ((uint32_t)dz << 24) |
                                 ((esz == 4 ? 2u : 1u) << 28));
    qdesc[1][q] = make_uint4((uint32_t)((xB - xA) * esz), (uint32_t)dB, (uint32_t)(nB * esz), 0u);
  }
  __syncthreads();

  // Issue the copies of the next stage; thread 0 first arms the stage's
  // barrier with the stage's byte count (bytes that land before it only take
  // the transaction count below zero for a moment; the phase cannot complete
  // before the one arrival).  Stages are issued in order, k = 0, 1, ...:
  // zq is the wrapped index of plane z - 1 of the next stage.
  const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
  int zq = wrapz(zb - 1);
  auto issue = [&](int k) {
    unsigned char* st = stage(k);
    uint64_t* bar = &bars[k % NST];
    const int z1 = zq + 1 == nz ? 0 : zq + 1;
    const int z2 = z1 + 1 == nz ? 0 : z1 + 1;
    const int z3 = z2 + 1 == nz ? 0 : z2 + 1;
    if (tid == 0) lbmk::mbar_arrive_expect_tx(bar, SH::TX_BYTES);
    if (tid < SH::NQ) {
      const uint4 d0 = qdesc[0][tid];
      const uint32_t dz = (d0.w >> 24) & 3u;
      const int zp = dz == 0 ? zq : (dz == 1 ? z1 : (dz == 2 ? z2 : z3));
      const unsigned char* src =
          reinterpret_cast<const unsigned char*>(((uint64_t)d0.y << 32) | d0.x) +
          ((size_t)((uint32_t)zp * nxy) << (d0.w >> 28));
      lbmk::bulk_g2s(st + d0.z, src, d0.w & 0xFFFFFFu, bar);
      const uint4 d1 = qdesc[1][tid];
      if (d1.z) lbmk::bulk_g2s(st + d1.y, src + (int32_t)d1.x, d1.z, bar);
    }
    zq = z1;
  };

  // pulled g at tile column xl (-1 .. BX) of phase-A row r from a staged plane
  auto staged_g = [&](unsigned char* st, int r, int xl, T (&G)[7], T& glo) {
    G[0] = sG0(st, 0, r)[xl + ET];
    glo = sG0(st, 1, r)[xl + ET];
#pragma unroll
    for (int m = 1; m < 7; ++m) G[m] = Conv<T, S>::ld(sGM(st, m, r) + (xl - bcx(m) + ES));
  };
  auto put = [&](int slot, int r, int xl, const T (&G)[7], T glo) {
    const T phi = phi_of(G, glo);
    Pair v;
    v.x = phi;
    v.y = psi3(phi, a.xi);
    ring[slot][r][xl + 1] = v;
  };

  // Halo position h of the tile (tile coordinates -1..BX, -1..BY): the rows
  // above and below, then the columns left and right.  Thread tid takes
  // positions tid, tid + NT, ... (one at most where NH <= NT).
  auto halo_xy = [&](int h, int& hx, int& hy) {
    if (h < RW) {
      hx = h - 1, hy = -1;
    } else if (h < 2 * RW) {
      hx = h - RW - 1, hy = BY;
    } else if (h < 2 * RW + BY) {
      hx = -1, hy = h - 2 * RW;
    } else {
      hx = BX, hy = h - 2 * RW - BY;
    }
  };

  for (int k = 0; k < NST - 1 && k < nplanes; ++k) issue(k);
  int issued_last = min(NST - 1, nplanes) - 1;
  int landed = -1;

  // ---- prologue: phase A of planes zb-1 and zb from global memory ----------
  T Gc[7], Gn[7], Gcl = T(0), Gnl = T(0);
  {
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    Offs own;
    set_xy(own, x0 + tx, wrapy(y0 + ty), nx, ny);
    for (int q = 0; q < 2; ++q) {
      const int zl = wrapz(zb - 1 + q);
      set_z(own, zl, nz, nxy);
      T G[7], gl;
      pull_g(g0s, g0ls, gms, P, own, G, gl);
      put((zb - 1 + q) & 3, ty + 1, tx, G, gl);
#pragma unroll
      for (int i = 0; i < 7; ++i) (q == 0 ? Gn : Gc)[i] = G[i];
      (q == 0 ? Gnl : Gcl) = gl;
      for (int h = tid; h < SH::NH; h += NT) {
        int hx, hy;
        halo_xy(h, hx, hy);
        Offs hal;
        set_xy(hal, (x0 + hx + nx) % nx, wrapy(y0 + hy), nx, ny);
        set_z(hal, zl, nz, nxy);
        pull_g(g0s, g0ls, gms, P, hal, G, gl);
        put((zb - 1 + q) & 3, hy + 1, hx, G, gl);
      }
    }
  }

  const long long lim = wait_cycles;
  double vsum = 0.0;
  for (int k = 0; k < nplanes; ++k) {
    const int z = zb + k;
    unsigned char* st = stage(k);
    const bool bad = !lbmk::mbar_wait_bounded(&bars[k % NST], (uint32_t)((k / NST) & 1), lim);
    if (!bad) {
      landed = k;
      // phase A of plane z + 1 from the staged g rows
      staged_g(st, ty + 1, tx, Gn, Gnl);
      put((z + 1) & 3, ty + 1, tx, Gn, Gnl);
      for (int h = tid; h < SH::NH; h += NT) {
        int hx, hy;
        halo_xy(h, hx, hy);
        T H[7], hl;
        staged_g(st, hy + 1, hx, H, hl);
        put((z + 1) & 3, hy + 1, hx, H, hl);
      }
    }
    if (__syncthreads_or(bad)) {
      // a wait gave up: report, wait for every stage issued but not yet seen
      // complete (its copies write into this CTA's shared memory), leave
      if (tid == 0) atomicOr(a.flags, kFlagTimeout3);
      for (int m = landed + 1; m <= issued_last; ++m)
        lbmk::mbar_wait_bounded(&bars[m % NST], (uint32_t)((m / NST) & 1), lbmk::kWaitCycles);
      return;
    }
    // the stage of plane k-1 is free: refill it with plane k-1+NST
    const int nxt = k + NST - 1;
    if (nxt < nplanes) {
      lbmk::fence_proxy_async_smem();
      issue(nxt);
      issued_last = nxt;
    }
    if (act) {
      T F[19], jp[3];
#pragma unroll
      for (int i = 0; i < 19; ++i) F[i] = Conv<T, S>::ld(sF(st, i, ty) + (tx - bcx(i) + ES));
#pragma unroll
      for (int c = 0; c < 3; ++c) jp[c] = sJ(st, c, ty)[tx];
      // stencils of plane z from the ring: planes z-1, z, z+1, rows ty..ty+2
      const int sm = (z + 3) & 3, s0 = z & 3, sp = (z + 1) & 3, j = ty + 1, i = tx + 1;
      const Pair c = ring[s0][j][i], e = ring[s0][j][i + 1], w = ring[s0][j][i - 1];
      const Pair n = ring[s0][j + 1][i], s = ring[s0][j - 1][i];
      const Pair ne = ring[s0][j + 1][i + 1], nw = ring[s0][j + 1][i - 1];
      const Pair se = ring[s0][j - 1][i + 1], sw = ring[s0][j - 1][i - 1];
      const Pair u = ring[sp][j][i], ue = ring[sp][j][i + 1], uw = ring[sp][j][i - 1];
      const Pair un = ring[sp][j + 1][i], us = ring[sp][j - 1][i];
      const Pair d = ring[sm][j][i], de = ring[sm][j][i + 1], dw = ring[sm][j][i - 1];
      const Pair dn = ring[sm][j + 1][i], ds = ring[sm][j - 1][i];
      const St3<T> SP{c.x, e.x, w.x, n.x, s.x, ne.x, nw.x, se.x, sw.x, u.x, ue.x, uw.x,
                      un.x, us.x, d.x, de.x, dw.x, dn.x, ds.x};
      const St3<T> SQ{c.y, e.y, w.y, n.y, s.y, ne.y, nw.y, se.y, sw.y, u.y, ue.y, uw.y,
                      un.y, us.y, d.y, de.y, dw.y, dn.y, ds.y};
      const Out3<T> o = node3<T, S, kModeStep>(a, F, Gc, Gcl, jp, SP, SQ);
      const T phi = SP.C;
      if (!(isfinite(phi) && isfinite(o.ux + o.uy + o.uz))) atomicOr(a.flags, kFlagNonFinite);
      if (a.vol_part) vsum += (double)phi;
      const uint32_t node = ((uint32_t)z * (uint32_t)ny + (uint32_t)(y0 + ty)) * (uint32_t)nx +
                            (uint32_t)(x0 + tx);
      jd[node] = phi * o.ux;
      jd[P + node] = phi * o.uy;
      jd[2 * P + node] = phi * o.uz;
      g0d[node] = Gc[0];
      g0ld[node] = Gcl;
#pragma unroll
      for (int m = 1; m < 7; ++m) gmd[(m - 1) * P + node] = Conv<T, S>::st(Gc[m]);
#pragma unroll
      for (int q = 0; q < 19; ++q) fd[q * P + node] = Conv<T, S>::st(F[q]);
    }
#pragma unroll
    for (int m = 0; m < 7; ++m) Gc[m] = Gn[m];
    Gcl = Gnl;
  }
  if (a.vol_part) {
    // fixed-order block reduction of the phi this CTA collided
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vsum += __shfl_down_sync(0xffffffffu, vsum, off);
    __shared__ double wsum[BX * BY / 32];
    if (lane == 0) wsum[warp] = vsum;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < BX * BY / 32; ++w) t += wsum[w];
      a.vol_part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
  }
}

}  // namespace lbmk3
