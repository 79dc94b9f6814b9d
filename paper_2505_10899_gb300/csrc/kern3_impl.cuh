// Launch wrappers of the three-dimensional kernels (see launch3.h).
#pragma once
#include <type_traits>

#include "launch3.h"
#include "lbm3_async.cuh"
#include "lbm3_bulk.cuh"
#include "lbm3_kernels.cuh"
#include "lbm3_strip.cuh"

namespace lbmk3 {

template <typename T, typename S>
static Args3<T, S> make_args(const Bufs& b, const Host3& h, int parity) {
  Args3<T, S> a{};
  for (int k = 0; k < 2; ++k) {
    a.f[k] = static_cast<S*>(b.f[k]);
    a.g[k] = static_cast<S*>(b.g[k]);
    a.g0[k] = static_cast<T*>(b.g0[k]);
    a.g0lo[k] = static_cast<T*>(b.g0lo[k]);
    a.J[k] = static_cast<T*>(b.J[k]);
  }
  a.plane = h.plane;
  a.nx = h.nx, a.ny = h.ny, a.nz = h.nz;
  a.parity = parity;
  a.var_tau = h.var_tau;
  a.beta4 = (T)h.beta4, a.kappa = (T)h.kappa, a.lambda = (T)h.lambda;
  a.lamW = (T)h.lamW, a.xi = (T)h.xi, a.tfac = (T)h.tfac;
  {
    // psi_k is ln(a/b) in FP64 and log2(a/b) in FP32, q = 12 grad(psi_k)
    const double qs = 48.0 * lbmk3::kNormalMin / (h.W * (sizeof(T) == 4 ? 0.69314718055994531 : 1.0));
    a.qmin2 = (T)(qs * qs);
  }
  a.wg = (T)h.wg, a.hg = (T)h.hg, a.wf = (T)h.wf, a.hf = (T)h.hf;
  a.rho_g = (T)h.rho_g, a.drho = (T)h.drho, a.mu_g = (T)h.mu_g, a.dmu = (T)h.dmu;
  a.wait = h.wait_cycles;
  return a;
}

template <typename T, typename S, int BX, int BY, int MODE>
static cudaError_t launch_tile(const Args3<T, S>& a, cudaStream_t st) {
  const dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY, (a.nz + a.zc - 1) / a.zc);
  const int par = a.parity, dst = par ^ 1;
  step3_kernel<T, S, BX, BY, MODE><<<grid, BX * BY, 0, st>>>(
      a, a.g0[par], a.g0lo[par], a.g[par], a.f[par], a.J[par], a.g0[dst], a.g0lo[dst], a.g[dst],
      a.f[dst], a.J[dst]);
  return cudaGetLastError();
}

template <int BX, int BY, int NST>
static cudaError_t launch_async(const Args3<float, float>& a, cudaStream_t st) {
  constexpr size_t bytes = async_smem_bytes<BX, BY, NST>();
  static bool attr_set = false;  // per instantiation, per process (one device)
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(step3_async_kernel<BX, BY, NST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY, (a.nz + a.zc - 1) / a.zc);
  const int par = a.parity, dst = par ^ 1;
  step3_async_kernel<BX, BY, NST><<<grid, BX * BY, bytes, st>>>(
      a, a.g0[par], a.g0lo[par], a.g[par], a.f[par], a.J[par], a.g0[dst], a.g0lo[dst], a.g[dst],
      a.f[dst], a.J[dst]);
  return cudaGetLastError();
}

template <typename T, typename S, int BX, int BY, int NST>
static cudaError_t launch_bulk(const Args3<T, S>& a, cudaStream_t st) {
  constexpr size_t bytes = bulk_smem_bytes<T, S, BX, BY, NST>();
  static bool attr_set = false;  // per instantiation, per process (one device)
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(step3_bulk_kernel<T, S, BX, BY, NST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (a.nx > BX) return cudaErrorInvalidValue;
  const dim3 grid(1, (a.ny + BY - 1) / BY, (a.nz + a.zc - 1) / a.zc);
  step3_bulk_kernel<T, S, BX, BY, NST><<<grid, BX * BY, bytes, st>>>(a, a.wait);
  return cudaGetLastError();
}

template <typename T, typename S, int BX, int BY, int NST, int MINB>
static cudaError_t launch_strip(const Args3<T, S>& a, cudaStream_t st) {
  constexpr size_t bytes = strip_smem_bytes<T, S, BX, BY, NST>();
  static bool attr_set = false;  // per instantiation, per process (one device)
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(step3_strip_kernel<T, S, BX, BY, NST, MINB>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (a.nx % BX != 0) return cudaErrorInvalidValue;
  const dim3 grid(a.nx / BX, (a.ny + BY - 1) / BY, (a.nz + a.zc - 1) / a.zc);
  step3_strip_kernel<T, S, BX, BY, NST, MINB><<<grid, BX * BY, bytes, st>>>(a, a.wait);
  return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t step_async(const Args3<T, S>& a, int variant, int bx, int by,
                              cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (variant == kVarBulk) {
      // stages: FP16 rows are half the size, so three fit beside the ring
      constexpr int NST = sizeof(S) == 2 ? 3 : 2;
      if (bx == 256 && by == 2) return launch_bulk<T, S, 256, 2, NST>(a, st);
      if (bx == 128 && by == 4) return launch_bulk<T, S, 128, 4, NST>(a, st);
      return cudaErrorInvalidValue;
    }
    if (variant == kVarStrip) {
      // about 90 KB per CTA of 256 threads: two CTAs per SM, with three FP16
      // stages or two FP32 ones per CTA
      constexpr int NST = sizeof(S) == 2 ? 3 : 2;
      if (bx == 32 && by == 8) return launch_strip<T, S, 32, 8, NST, 2>(a, st);
      if (bx == 64 && by == 4) return launch_strip<T, S, 64, 4, NST, 2>(a, st);
      return cudaErrorInvalidValue;
    }
    if (variant == kVarStripOcc) {
      // two stages per CTA and at most 80 (64 x 4) or 96 (64 x 2) registers:
      // three or five CTAs per SM where shared memory allows (FP16 storage)
      if (bx == 64 && by == 4) return launch_strip<T, S, 64, 4, 2, 3>(a, st);
      if (bx == 64 && by == 2) return launch_strip<T, S, 64, 2, 2, 5>(a, st);
      return cudaErrorInvalidValue;
    }
  }
  if constexpr (std::is_same<T, float>::value && std::is_same<S, float>::value) {
    if (variant == kVarAsync2) {
      if (bx == 32 && by == 4) return launch_async<32, 4, 2>(a, st);
      if (bx == 32 && by == 8) return launch_async<32, 8, 2>(a, st);
      if (bx == 64 && by == 4) return launch_async<64, 4, 2>(a, st);
    } else if (variant == kVarAsync3) {
      if (bx == 32 && by == 4) return launch_async<32, 4, 3>(a, st);
      if (bx == 32 && by == 8) return launch_async<32, 8, 3>(a, st);
      if (bx == 64 && by == 4) return launch_async<64, 4, 3>(a, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, typename S>
cudaError_t K3<T, S>::step(const Bufs& b, const Host3& h, int parity, int variant, int bx,
                           int by, int zc, int mode, int32_t* flags, double* vol_part,
                           double* out, int which, cudaStream_t st) {
  Args3<T, S> a = make_args<T, S>(b, h, parity);
  a.zc = zc;
  a.flags = flags;
  a.vol_part = vol_part;
  a.out = out;
  a.out_which = which;
  if (mode == kModeFields) return launch_tile<T, S, 32, 8, kModeFields>(a, st);
  if (variant != kVarRegs) return step_async(a, variant, bx, by, st);
  if (bx == 32 && by == 4) return launch_tile<T, S, 32, 4, kModeStep>(a, st);
  if (bx == 32 && by == 8) return launch_tile<T, S, 32, 8, kModeStep>(a, st);
  if (bx == 32 && by == 16) return launch_tile<T, S, 32, 16, kModeStep>(a, st);
  if (bx == 64 && by == 4) return launch_tile<T, S, 64, 4, kModeStep>(a, st);
  return cudaErrorInvalidValue;
}

static inline int aux_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

template <typename T, typename S>
cudaError_t K3<T, S>::init(const Bufs& b, const Host3& h, int parity, const double* d_phi0,
                           const double* d_u0, cudaStream_t st) {
  const Args3<T, S> a = make_args<T, S>(b, h, parity);
  const int64_t n = (int64_t)h.nx * h.ny * h.nz;
  init3_kernel<T, S><<<aux_blocks(n), 256, 0, st>>>(a, h.beta4, h.kappa, h.lambda, h.rho_g,
                                                     h.drho, d_phi0, d_u0);
  init3_rest_kernel<T, S><<<aux_blocks(n), 256, 0, st>>>(a, d_phi0);
  return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t K3<T, S>::plane(const Bufs& b, const Host3& h, int parity, int kind, int i,
                            double* d_buf, int to_device, cudaStream_t st) {
  const Args3<T, S> a = make_args<T, S>(b, h, parity);
  const int64_t n = (int64_t)h.nx * h.ny * h.nz;
  plane3_kernel<T, S><<<aux_blocks(n), 256, 0, st>>>(a, kind, i, d_buf, to_device);
  return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t K3<T, S>::volume(const Bufs& b, const Host3& h, int parity, const int8_t* labels,
                             int nregions, double* part, int nparts, double* out,
                             cudaStream_t st) {
  const Args3<T, S> a = make_args<T, S>(b, h, parity);
  volume3_kernel<T, S><<<nparts, 256, 0, st>>>(a, labels, nregions, part);
  volume3_final<<<nregions, 32, 0, st>>>(part, nparts, kMaxRegions, nregions, out);
  return cudaGetLastError();
}

}  // namespace lbmk3
