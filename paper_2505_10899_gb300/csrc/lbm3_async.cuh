// Asynchronous-copy variant of the three-dimensional step kernel (FP32
// storage and arithmetic).  Same per-node arithmetic as step3_kernel
// (node3, the same stencils and phase-A sums); the difference is how the
// pulled values reach the threads.
//
// Each thread copies the values it will consume -- its 19 pulled f, its
// phi*u of the previous step, and the 7 (+ low part of g_0) pulled g of its
// own node and of its halo node -- from global to shared memory with 4-byte
// cp.async copies, NST - 1 planes ahead of the plane it updates.  The copies
// need no registers while in flight, so the global-memory latency of plane
// z + NST - 1 overlaps the arithmetic of plane z without the register cost
// of a software pipeline.  Every thread reads back only the slots it copied
// itself, so the stage buffers need no barrier: cp.async.wait_group orders
// each thread's own copies, and a slot is refilled only after the same
// thread has read it (program order).  The (phi, psi) ring is shared and
// keeps one barrier per plane, as in step3_kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm3_kernels.cuh"

namespace lbmk3 {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory footprint of one stage: f (19), phi*u (3), own g (8 with the
// low part of g_0), halo g (8).
template <int BX, int BY>
struct AsyncShape {
  static constexpr int NT = BX * BY;
  static constexpr int NH = 2 * (BX + 2) + 2 * BY;
  static constexpr int STAGE = (19 + 3 + 8) * NT + 8 * NH;  // floats
};

template <int BX, int BY, int NST>
constexpr size_t async_smem_bytes() {
  return sizeof(Ring3<float, BX, BY>) + (size_t)NST * AsyncShape<BX, BY>::STAGE * sizeof(float);
}

template <int BX, int BY, int NST>
__global__ void __launch_bounds__(BX* BY) step3_async_kernel(
    const Args3<float, float> a, const float* __restrict__ g0s, const float* __restrict__ g0ls,
    const float* __restrict__ gms, const float* __restrict__ fs, const float* __restrict__ js,
    float* __restrict__ g0d, float* __restrict__ g0ld, float* __restrict__ gmd,
    float* __restrict__ fd, float* __restrict__ jd) {
  using Sh = AsyncShape<BX, BY>;
  constexpr int NT = Sh::NT, NH = Sh::NH;
  static_assert(NH <= NT, "tile too small for its halo");
  static_assert(NST >= 2, "at least two stages");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Ring3<float, BX, BY>& ring = *reinterpret_cast<Ring3<float, BX, BY>*>(smem_raw);
  float* stages = reinterpret_cast<float*>(smem_raw + sizeof(Ring3<float, BX, BY>));

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
  const int64_t P = a.plane;
  const int gx = blockIdx.x * BX + tx, gy = blockIdx.y * BY + ty;
  const bool valid = gx < nx && gy < ny;
  Offs own, hal;
  set_xy(own, gx % nx, gy % ny, nx, ny);
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
  auto zwrap = [&](int zl) { return zl < 0 ? zl + nz : (zl >= nz ? zl - nz : zl); };

  // slots of this thread in stage s
  auto sF = [&](int s, int i) { return stages + (size_t)s * Sh::STAGE + i * NT + tid; };
  auto sJ = [&](int s, int c) { return stages + (size_t)s * Sh::STAGE + (19 + c) * NT + tid; };
  auto sG = [&](int s, int i) { return stages + (size_t)s * Sh::STAGE + (22 + i) * NT + tid; };
  auto sH = [&](int s, int i) { return stages + (size_t)s * Sh::STAGE + 30 * NT + i * NH + tid; };

  auto copy_g = [&](const Offs& o, auto slot) {
    cp_async4(slot(0), g0s + src_of<0>(o));
    cp_async4(slot(1), gms + 0 * P + src_of<1>(o));
    cp_async4(slot(2), gms + 1 * P + src_of<2>(o));
    cp_async4(slot(3), gms + 2 * P + src_of<3>(o));
    cp_async4(slot(4), gms + 3 * P + src_of<4>(o));
    cp_async4(slot(5), gms + 4 * P + src_of<5>(o));
    cp_async4(slot(6), gms + 5 * P + src_of<6>(o));
    cp_async4(slot(7), g0ls + src_of<0>(o));
  };
  // group of plane zq: f and phi*u of plane zq (own node, valid threads), g of
  // plane zq + 1 (own and halo node); planes past the chunk copy nothing
  auto issue = [&](int zq, int s) {
    if (zq < ze && valid) {
      Offs o = own;
      set_z(o, zq, nz, nxy);
#define LBM3_CPF(I) cp_async4(sF(s, I), fs + (I) * P + src_of<I>(o))
      LBM3_CPF(0); LBM3_CPF(1); LBM3_CPF(2); LBM3_CPF(3); LBM3_CPF(4);
      LBM3_CPF(5); LBM3_CPF(6); LBM3_CPF(7); LBM3_CPF(8); LBM3_CPF(9);
      LBM3_CPF(10); LBM3_CPF(11); LBM3_CPF(12); LBM3_CPF(13); LBM3_CPF(14);
      LBM3_CPF(15); LBM3_CPF(16); LBM3_CPF(17); LBM3_CPF(18);
#undef LBM3_CPF
      const uint32_t node = o.z[1] + o.y[1] + o.x[1];
      cp_async4(sJ(s, 0), js + node);
      cp_async4(sJ(s, 1), js + P + node);
      cp_async4(sJ(s, 2), js + 2 * P + node);
    }
    if (zq < ze) {
      const int zg = zwrap(zq + 1);
      Offs o = own;
      set_z(o, zg, nz, nxy);
      copy_g(o, [&](int i) { return sG(s, i); });
      if (has_h) {
        Offs oh = hal;
        set_z(oh, zg, nz, nxy);
        copy_g(oh, [&](int i) { return sH(s, i); });
      }
    }
    cp_commit();
  };

  // phi, psi of one node from 8 values (7 populations + low part of g_0)
  auto put = [&](int slot, int j, int i, const float (&G)[7], float glo) {
    const float phi = phi_of(G, glo);
    float2 v;
    v.x = phi;
    v.y = psi3(phi, a.xi);
    ring.pq[slot][j][i] = v;
  };

  // planes zb - 1 and zb: direct loads (no prefetch yet)
  float Gc[7], Gn[7], Gcl, Gnl;
  {
    float H[7], Hl;
    for (int q = 0; q < 2; ++q) {
      const int zl = zb - 1 + q;
      Offs o = own;
      set_z(o, zwrap(zl), nz, nxy);
      if (q == 0) {
        pull_g(g0s, g0ls, gms, P, o, Gn, Gnl);
        put(zl & 3, ty + 1, tx + 1, Gn, Gnl);
      } else {
        pull_g(g0s, g0ls, gms, P, o, Gc, Gcl);
        put(zl & 3, ty + 1, tx + 1, Gc, Gcl);
      }
      if (has_h) {
        Offs oh = hal;
        set_z(oh, zwrap(zl), nz, nxy);
        pull_g(g0s, g0ls, gms, P, oh, H, Hl);
        const float phh = sum7(H) + Hl;
        ring.pq[zl & 3][hy + 1][hx + 1] = make_float2(phh, psi3(phh, a.xi));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NST - 1; ++q) issue(zb + q, q);

  double vsum = 0.0;
  int s = 0;
  for (int z = zb; z < ze; ++z) {
    issue(z + NST - 1, (s + NST - 1) % NST);
    cp_wait<NST - 1>();  // the group of plane z has landed
    // phase A for plane z + 1 from this thread's own copies
    {
#pragma unroll
      for (int i = 0; i < 7; ++i) Gn[i] = *sG(s, i);
      Gnl = *sG(s, 7);
      put((z + 1) & 3, ty + 1, tx + 1, Gn, Gnl);
      if (has_h) {  // halo phi: plain sum, as in step3_kernel
        float H[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) H[i] = *sH(s, i);
        const float phh = sum7(H) + *sH(s, 7);
        ring.pq[(z + 1) & 3][hy + 1][hx + 1] = make_float2(phh, psi3(phh, a.xi));
      }
    }
    __syncthreads();
    if (valid) {
      float F[19], jp[3];
#pragma unroll
      for (int i = 0; i < 19; ++i) F[i] = *sF(s, i);
#pragma unroll
      for (int c = 0; c < 3; ++c) jp[c] = *sJ(s, c);
      St3<float> SP, SQ;
      read_st(ring, (z + 3) & 3, z & 3, (z + 1) & 3, ty + 1, tx + 1, SP, SQ);
      const Out3<float> o = node3<float, float, kModeStep>(a, F, Gc, Gcl, jp, SP, SQ);
      const float phi = SP.C;
      if (!(isfinite(phi) && isfinite(o.ux + o.uy + o.uz))) atomicOr(a.flags, kFlagNonFinite);
      const uint32_t node = (uint32_t)z * nxy + own.y[1] + own.x[1];
      if (a.vol_part) vsum += (double)phi;
      jd[node] = phi * o.ux;
      jd[P + node] = phi * o.uy;
      jd[2 * P + node] = phi * o.uz;
      g0d[node] = Gc[0];
      g0ld[node] = Gcl;
#pragma unroll
      for (int i = 1; i < 7; ++i) gmd[(i - 1) * P + node] = Gc[i];
#pragma unroll
      for (int i = 0; i < 19; ++i) fd[i * P + node] = F[i];
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) Gc[i] = Gn[i];
    Gcl = Gnl;
    s = (s + 1) % NST;
  }
  cp_wait<0>();
  if (a.vol_part) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vsum += __shfl_down_sync(0xffffffffu, vsum, off);
    __shared__ double wsum[NT / 32];
    __syncthreads();
    if ((tid & 31) == 0) wsum[tid >> 5] = vsum;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += wsum[w];
      a.vol_part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
  }
}

}  // namespace lbmk3
