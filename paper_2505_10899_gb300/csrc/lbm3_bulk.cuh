// Bulk-copy variant of the three-dimensional step kernel (FP32 arithmetic,
// FP32 or FP16 population storage) for boxes whose rows fit one CTA: nx <=
// BX, a row of nx values a multiple of 16 bytes.  Same per-node arithmetic as
// step3_kernel (node3, the same stencils and phase-A sums); the difference is
// how the pulled values reach the threads.
//
// A CTA owns BY whole x-rows (y0 .. y0+BY-1) and marches along z over `zc`
// planes.  Every value it reads for plane z arrives in shared memory by 1-D
// bulk copies (cp.async.bulk) of whole rows, issued by the lanes of warp 0
// NST-1 planes ahead and completed on one mbarrier per stage:
//   - f_i: row (y - c_iy, z - c_iz) of plane i, for each of the BY rows
//     (the pull in x is an index shift inside the staged row, periodic);
//   - phi*u: rows (y, z);
//   - the 7 g (and the low part of g_0) pulled to the BY + 2 rows y0-1 ..
//     y0+BY of plane z+1, for phase A: phi = sum g (Eq. 35) and psi (Eq. 37)
//     into a 4-plane ring of (phi, psi), from which the D3Q19 stencils of
//     Sec. 3.2 are read.
// A row copy is one contiguous transfer of nx values: about 0.15 copies per
// node instead of one 2- or 4-byte load per population per node, and no
// global-load latency inside the collision.  The pulled g of a thread's own
// row stay in registers from phase A (plane z+1) to the update (plane z+1).
//
// Every wait is bounded (wait_cycles); on expiry the CTA raises
// kFlagTimeout3, waits (bounded by lbmk::kWaitCycles) for its own copies in
// flight and returns.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm3_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbmk3 {

// Components of the 19 velocities (the order of lbm3_layout.h) as
// compile-time functions, usable with run-time indices without a memory
// access.
__host__ __device__ constexpr int bcx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                : 0;
}
__host__ __device__ constexpr int bcy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)   ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                               : 0;
}
__host__ __device__ constexpr int bcz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)   ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                 : 0;
}
constexpr bool bulk_lattice_matches(int i = 0) {
  return i == 19 || (bcx(i) == Lat::cx[i] && bcy(i) == Lat::cy[i] && bcz(i) == Lat::cz[i] &&
                     bulk_lattice_matches(i + 1));
}
static_assert(bulk_lattice_matches(), "velocity functions must match the lattice table");

template <typename T, typename S, int BX, int BY, int NST>
struct BulkShape {
  static constexpr int NR = BY + 2;  // phase-A rows (with the halo rows)
  // element offsets inside one stage (S region first, then T region)
  static constexpr size_t F_OFF = 0;                                   // [19][BY][BX] S
  static constexpr size_t GM_OFF = F_OFF + (size_t)19 * BY * BX * sizeof(S);  // [6][NR][BX] S
  static constexpr size_t J_OFF = GM_OFF + (size_t)6 * NR * BX * sizeof(S);   // [3][BY][BX] T
  static constexpr size_t G0_OFF = J_OFF + (size_t)3 * BY * BX * sizeof(T);   // [2][NR][BX] T
  static constexpr size_t STAGE_BYTES = G0_OFF + (size_t)2 * NR * BX * sizeof(T);
  static constexpr size_t BAR_OFF = NST * STAGE_BYTES;
  static constexpr size_t RING_OFF = (BAR_OFF + NST * 8 + 127) / 128 * 128;
  static constexpr size_t RING_BYTES = (size_t)4 * NR * BX * sizeof(typename N3<T>::pair);
  static constexpr size_t SMEM_BYTES = RING_OFF + RING_BYTES;
  static constexpr int NQ = 22 * BY + 8 * NR;  // row copies per stage
  static_assert(STAGE_BYTES % 16 == 0 && GM_OFF % 16 == 0 && J_OFF % 16 == 0 &&
                    G0_OFF % 16 == 0,
                "stage regions must keep 16-byte alignment");
};

template <typename T, typename S, int BX, int BY, int NST>
constexpr size_t bulk_smem_bytes() {
  return BulkShape<T, S, BX, BY, NST>::SMEM_BYTES;
}

template <typename T, typename S, int BX, int BY, int NST>
__global__ void __launch_bounds__(BX* BY, 1)
    step3_bulk_kernel(const Args3<T, S> a, long long wait_cycles) {
  using SH = BulkShape<T, S, BX, BY, NST>;
  using Pair = typename N3<T>::pair;
  constexpr int NR = SH::NR;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* const bars = reinterpret_cast<uint64_t*>(smem + SH::BAR_OFF);
  Pair(*const ring)[NR][BX] = reinterpret_cast<Pair(*)[NR][BX]>(smem + SH::RING_OFF);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX, warp = tid >> 5, lane = tid & 31;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t P = a.plane;
  const int y0 = blockIdx.y * BY;
  const int zb = blockIdx.z * a.zc;
  const int ze = min(zb + a.zc, nz);
  const int nplanes = ze - zb;
  const bool colv = tx < nx;                    // a column of the box
  const bool act = colv && (y0 + ty < ny);      // a node this CTA updates
  // periodic neighbour columns inside a staged row
  const int xm = (tx == 0) ? nx - 1 : tx - 1;
  const int xp = (tx + 1 >= nx) ? 0 : tx + 1;
  // periodic wrap of row and plane indices (any number of periods: boxes may
  // be thinner than the rows and planes a CTA touches)
  auto wrapy = [&](int v) { return ((v % ny) + ny) % ny; };
  auto wrapz = [&](int v) { return ((v % nz) + nz) % nz; };
  auto colof = [&](int cx) { return cx == 1 ? xm : (cx == -1 ? xp : tx); };

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
    return reinterpret_cast<S*>(st + SH::F_OFF) + ((size_t)i * BY + r) * BX;
  };
  auto sGM = [&](unsigned char* st, int m, int r) {  // mover m = 1..6, phase-A row r
    return reinterpret_cast<S*>(st + SH::GM_OFF) + ((size_t)(m - 1) * NR + r) * BX;
  };
  auto sJ = [&](unsigned char* st, int c, int r) {
    return reinterpret_cast<T*>(st + SH::J_OFF) + ((size_t)c * BY + r) * BX;
  };
  auto sG0 = [&](unsigned char* st, int h, int r) {  // h = 0: g_0, 1: its low part
    return reinterpret_cast<T*>(st + SH::G0_OFF) + ((size_t)h * NR + r) * BX;
  };
  // first element of row (y, z) of a plane, both coordinates wrapped
  auto rowp = [&](int y, int z) -> int64_t {
    return ((int64_t)wrapz(z) * ny + wrapy(y)) * nx;
  };

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) lbmk::mbar_init(&bars[s], 1);
    lbmk::fence_mbar_init();
  }
  __syncthreads();

  // Row copies of local plane k (plane z = zb + k): f and phi*u of the BY
  // rows of plane z, the g of the NR phase-A rows of plane z + 1.  Warp 0.
  const uint32_t bytes_stage = (uint32_t)((19 * BY + 6 * NR) * nx * sizeof(S) +
                                          (3 * BY + 2 * NR) * nx * sizeof(T));
  auto issue = [&](int k) {
    unsigned char* st = stage(k);
    uint64_t* bar = &bars[k % NST];
    const int z = zb + k;
    if (lane == 0) lbmk::mbar_arrive_expect_tx(bar, bytes_stage);
    __syncwarp();
    for (int q = lane; q < SH::NQ; q += 32) {
      void* d;
      const void* s;
      uint32_t nb;
      if (q < 19 * BY) {
        const int i = q / BY, r = q % BY;
        d = sF(st, i, r);
        s = fs + (int64_t)i * P + rowp(y0 + r - bcy(i), z - bcz(i));
        nb = (uint32_t)(nx * sizeof(S));
      } else if (q < 19 * BY + 6 * NR) {
        const int u = q - 19 * BY, m = u / NR + 1, r = u % NR;
        d = sGM(st, m, r);
        s = gms + (int64_t)(m - 1) * P + rowp(y0 - 1 + r - bcy(m), z + 1 - bcz(m));
        nb = (uint32_t)(nx * sizeof(S));
      } else if (q < 22 * BY + 6 * NR) {
        const int u = q - 19 * BY - 6 * NR, c = u / BY, r = u % BY;
        d = sJ(st, c, r);
        s = js + (int64_t)c * P + rowp(y0 + r, z);
        nb = (uint32_t)(nx * sizeof(T));
      } else {
        const int u = q - 22 * BY - 6 * NR, h = u / NR, r = u % NR;
        d = sG0(st, h, r);
        s = (h == 0 ? g0s : g0ls) + rowp(y0 - 1 + r, z + 1);
        nb = (uint32_t)(nx * sizeof(T));
      }
      lbmk::bulk_g2s(d, s, nb, bar);
    }
  };

  // pulled g of column tx of phase-A row r from a staged plane
  auto staged_g = [&](unsigned char* st, int r, T (&G)[7], T& glo) {
    G[0] = sG0(st, 0, r)[tx];
    glo = sG0(st, 1, r)[tx];
#pragma unroll
    for (int m = 1; m < 7; ++m) G[m] = Conv<T, S>::ld(sGM(st, m, r) + colof(bcx(m)));
  };
  auto put = [&](int slot, int r, const T (&G)[7], T glo) {
    const T phi = phi_of(G, glo);
    Pair v;
    v.x = phi;
    v.y = psi3(phi, a.xi);
    ring[slot][r][tx] = v;
  };

  // ---- prologue: phase A of planes zb-1 and zb from global memory ----------
  T Gc[7], Gn[7], Gcl = T(0), Gnl = T(0);
  const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
  for (int q = 0; q < 2; ++q) {
    const int zl = zb - 1 + q;
    // own row (ty + 1) and, for the first and last thread rows, the halo rows
    for (int h = 0; h < 2; ++h) {
      int r;
      if (h == 0) r = ty + 1;
      else if (ty == 0) r = 0;
      else if (ty == BY - 1) r = NR - 1;
      else break;
      if (!colv) break;
      Offs o;
      set_xy(o, tx, wrapy(y0 - 1 + r), nx, ny);
      set_z(o, wrapz(zl), nz, nxy);
      T G[7], gl;
      pull_g(g0s, g0ls, gms, P, o, G, gl);
      put(zl & 3, r, G, gl);
      if (h == 0) {
#pragma unroll
        for (int i = 0; i < 7; ++i) (q == 0 ? Gn : Gc)[i] = G[i];
        (q == 0 ? Gnl : Gcl) = gl;
      }
    }
  }
  if (warp == 0)
    for (int k = 0; k < NST - 1 && k < nplanes; ++k) issue(k);
  int issued_last = min(NST - 1, nplanes) - 1;
  int landed = -1;
  const long long lim = wait_cycles;

  double vsum = 0.0;
  for (int k = 0; k < nplanes; ++k) {
    const int z = zb + k;
    unsigned char* st = stage(k);
    bool bad = !lbmk::mbar_wait_bounded(&bars[k % NST], (uint32_t)((k / NST) & 1), lim);
    if (!bad) {
      landed = k;
      // phase A of plane z + 1 from the staged g rows
      if (colv) {
        staged_g(st, ty + 1, Gn, Gnl);
        put((z + 1) & 3, ty + 1, Gn, Gnl);
        if (ty == 0 || ty == BY - 1) {
          const int r = ty == 0 ? 0 : NR - 1;
          T H[7], hl;
          staged_g(st, r, H, hl);
          put((z + 1) & 3, r, H, hl);
        }
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
      if (warp == 0) {
        lbmk::fence_proxy_async_smem();
        issue(nxt);
      }
      issued_last = nxt;
    }
    if (act) {
      T F[19], jp[3];
#pragma unroll
      for (int i = 0; i < 19; ++i) F[i] = Conv<T, S>::ld(sF(st, i, ty) + colof(bcx(i)));
#pragma unroll
      for (int c = 0; c < 3; ++c) jp[c] = sJ(st, c, ty)[tx];
      // stencils of plane z from the ring: planes z-1, z, z+1, rows ty..ty+2
      const int sm = (z + 3) & 3, s0 = z & 3, sp = (z + 1) & 3, j = ty + 1;
      const Pair c = ring[s0][j][tx], e = ring[s0][j][xp], w = ring[s0][j][xm];
      const Pair n = ring[s0][j + 1][tx], s = ring[s0][j - 1][tx];
      const Pair ne = ring[s0][j + 1][xp], nw = ring[s0][j + 1][xm];
      const Pair se = ring[s0][j - 1][xp], sw = ring[s0][j - 1][xm];
      const Pair u = ring[sp][j][tx], ue = ring[sp][j][xp], uw = ring[sp][j][xm];
      const Pair un = ring[sp][j + 1][tx], us = ring[sp][j - 1][tx];
      const Pair d = ring[sm][j][tx], de = ring[sm][j][xp], dw = ring[sm][j][xm];
      const Pair dn = ring[sm][j + 1][tx], ds = ring[sm][j - 1][tx];
      const St3<T> SP{c.x, e.x, w.x, n.x, s.x, ne.x, nw.x, se.x, sw.x, u.x, ue.x, uw.x,
                      un.x, us.x, d.x, de.x, dw.x, dn.x, ds.x};
      const St3<T> SQ{c.y, e.y, w.y, n.y, s.y, ne.y, nw.y, se.y, sw.y, u.y, ue.y, uw.y,
                      un.y, us.y, d.y, de.y, dw.y, dn.y, ds.y};
      const Out3<T> o = node3<T, S, kModeStep>(a, F, Gc, Gcl, jp, SP, SQ);
      const T phi = SP.C;
      if (!(isfinite(phi) && isfinite(o.ux + o.uy + o.uz))) atomicOr(a.flags, kFlagNonFinite);
      if (a.vol_part) vsum += (double)phi;
      const uint32_t node = (uint32_t)z * nxy + (uint32_t)(y0 + ty) * (uint32_t)nx + (uint32_t)tx;
      jd[node] = phi * o.ux;
      jd[P + node] = phi * o.uy;
      jd[2 * P + node] = phi * o.uz;
      g0d[node] = Gc[0];
      g0ld[node] = Gcl;
#pragma unroll
      for (int i = 1; i < 7; ++i) gmd[(i - 1) * P + node] = Conv<T, S>::st(Gc[i]);
#pragma unroll
      for (int i = 0; i < 19; ++i) fd[i * P + node] = Conv<T, S>::st(F[i]);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) Gc[i] = Gn[i];
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
