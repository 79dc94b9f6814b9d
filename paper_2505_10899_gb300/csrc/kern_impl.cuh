// Explicit instantiation of the launch wrappers for precision LBM_T.
// Included by kern_f32.cu (LBM_T = float) and kern_f64.cu (LBM_T = double).
#include <algorithm>
#include <type_traits>

#include "launch.h"
#include "lbm_aux.cuh"
#include "lbm_kernels.cuh"
#include "lbm_kernels_tma.cuh"

namespace lbmk {

namespace {
inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 65535 * 8) b = 65535 * 8;
  return (int)(b < 1 ? 1 : b);
}

// pipeline depth of the TMA kernel: 4 stages for narrow strips in FP32,
// 3 otherwise (keeps shared memory per CTA low enough for 5-6 CTAs per SM)
template <int BX>
constexpr int stages_for() {
  return (sizeof(LBM_T) == 4 && BX <= 64) ? 4 : 3;
}

template <int BX, bool COUPLED, int MODE>
cudaError_t step_tma(const StepArgs<LBM_T>& a, int n, cudaStream_t s) {
  using SH = TmaShape<LBM_T, BX, COUPLED, MODE, stages_for<BX>()>;
  step_kernel_tma<LBM_T, BX, COUPLED, MODE, stages_for<BX>()><<<n, BX, SH::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int BX, bool COUPLED, int MODE>
cudaError_t prep_one() {
  using SH = TmaShape<LBM_T, BX, COUPLED, MODE, stages_for<BX>()>;
  return cudaFuncSetAttribute(step_kernel_tma<LBM_T, BX, COUPLED, MODE, stages_for<BX>()>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::SMEM_BYTES);
}

template <int BX>
cudaError_t prep_bx() {
  cudaError_t e;
  if ((e = prep_one<BX, true, kModeStep>()) != cudaSuccess) return e;
  if ((e = prep_one<BX, true, kModeFields>()) != cudaSuccess) return e;
  if ((e = prep_one<BX, false, kModeStep>()) != cudaSuccess) return e;
  return prep_one<BX, false, kModeFields>();
}

template <int BX>
cudaError_t step_bx(const StepArgs<LBM_T>& a, bool coupled, int mode, bool tma, int n,
                    cudaStream_t s) {
  if (tma) {
    if (coupled)
      return mode == kModeStep ? step_tma<BX, true, kModeStep>(a, n, s)
                               : step_tma<BX, true, kModeFields>(a, n, s);
    return mode == kModeStep ? step_tma<BX, false, kModeStep>(a, n, s)
                             : step_tma<BX, false, kModeFields>(a, n, s);
  }
  if constexpr (BX != 32 && BX != 64 && BX != 128) {
    return cudaErrorInvalidValue;  // whole-row widths: bulk-copy kernel only
  } else {
  if (coupled) {
    if (mode == kModeStep)
      step_kernel<LBM_T, BX, true, kModeStep><<<n, BX, 0, s>>>(a);
    else
      step_kernel<LBM_T, BX, true, kModeFields><<<n, BX, 0, s>>>(a);
  } else {
    if (mode == kModeStep)
      step_kernel<LBM_T, BX, false, kModeStep><<<n, BX, 0, s>>>(a);
    else
      step_kernel<LBM_T, BX, false, kModeFields><<<n, BX, 0, s>>>(a);
  }
  return cudaGetLastError();
  }
}
}  // namespace

template <>
cudaError_t launch_step<LBM_T>(const StepArgs<LBM_T>& a, int bx, bool coupled, int mode,
                               bool tma, int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  switch (bx) {
    case 32: return step_bx<32>(a, coupled, mode, tma, n_items, s);
    case 64: return step_bx<64>(a, coupled, mode, tma, n_items, s);
    case 128: return step_bx<128>(a, coupled, mode, tma, n_items, s);
    case 96: return step_bx<96>(a, coupled, mode, tma, n_items, s);
    case 192: return step_bx<192>(a, coupled, mode, tma, n_items, s);
    case 256: return step_bx<256>(a, coupled, mode, tma, n_items, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int BX, bool COUPLED>
cudaError_t persist_bx(const StepArgs<LBM_T>& a, int n_items, int nsteps, int flip,
                       unsigned int* count, unsigned int* gen, cudaStream_t s) {
  auto kern = step_kernel_persistent<LBM_T, BX, COUPLED>;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BX, 0);
  if (e != cudaSuccess) return e;
  int grid = per_sm * nsm;
  if (grid > n_items) grid = n_items;
  if (grid < 1) return cudaErrorInvalidConfiguration;
  StepArgs<LBM_T> args = a;
  GridBar bar{count, gen};
  void* params[] = {(void*)&args, (void*)&n_items, (void*)&nsteps, (void*)&flip, (void*)&bar};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(BX), params, 0, s);
}

template <>
cudaError_t launch_persistent<LBM_T>(const StepArgs<LBM_T>& a, int bx, bool coupled, int n_items,
                                     int nsteps, int flip, unsigned int* count,
                                     unsigned int* gen, cudaStream_t s) {
  if (n_items <= 0 || nsteps <= 0) return cudaSuccess;
  switch (bx) {
    case 32: return coupled ? persist_bx<32, true>(a, n_items, nsteps, flip, count, gen, s)
                            : persist_bx<32, false>(a, n_items, nsteps, flip, count, gen, s);
    case 64: return coupled ? persist_bx<64, true>(a, n_items, nsteps, flip, count, gen, s)
                            : persist_bx<64, false>(a, n_items, nsteps, flip, count, gen, s);
    case 128: return coupled ? persist_bx<128, true>(a, n_items, nsteps, flip, count, gen, s)
                             : persist_bx<128, false>(a, n_items, nsteps, flip, count, gen, s);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t prepare_tma<LBM_T>() {
  cudaError_t e;
  if ((e = prep_bx<32>()) != cudaSuccess) return e;
  if ((e = prep_bx<64>()) != cudaSuccess) return e;
  if ((e = prep_bx<96>()) != cudaSuccess) return e;
  if ((e = prep_bx<192>()) != cudaSuccess) return e;
  if ((e = prep_bx<256>()) != cudaSuccess) return e;
  return prep_bx<128>();
}

template <>
size_t tma_smem_bytes<LBM_T>(int bx, bool coupled, int mode) {
  auto pick = [&](auto bxc) -> size_t {
    constexpr int B = decltype(bxc)::value;
    constexpr int S = stages_for<B>();
    if (coupled)
      return mode == kModeStep ? TmaShape<LBM_T, B, true, kModeStep, S>::SMEM_BYTES
                               : TmaShape<LBM_T, B, true, kModeFields, S>::SMEM_BYTES;
    return mode == kModeStep ? TmaShape<LBM_T, B, false, kModeStep, S>::SMEM_BYTES
                             : TmaShape<LBM_T, B, false, kModeFields, S>::SMEM_BYTES;
  };
  switch (bx) {
    case 32: return pick(std::integral_constant<int, 32>{});
    case 64: return pick(std::integral_constant<int, 64>{});
    case 128: return pick(std::integral_constant<int, 128>{});
    case 96: return pick(std::integral_constant<int, 96>{});
    case 192: return pick(std::integral_constant<int, 192>{});
    case 256: return pick(std::integral_constant<int, 256>{});
    default: return 0;
  }
}

template <>
cudaError_t launch_init_items<LBM_T>(const CaseDev<LBM_T>* cases, const Item* items, int n_items,
                                     int bx, const InitSrc* src, double beta4, double kappa,
                                     double lambda, int vortex, double vU, int parity,
                                     cudaStream_t s) {
  if (n_items < 1) return cudaSuccess;
  switch (bx) {
    case 32:
      init_items<LBM_T, 32><<<n_items, 32, 0, s>>>(cases, items, src, beta4, kappa, lambda,
                                                    vortex, vU, parity);
      break;
    case 64:
      init_items<LBM_T, 64><<<n_items, 64, 0, s>>>(cases, items, src, beta4, kappa, lambda,
                                                    vortex, vU, parity);
      break;
    case 96:
      init_items<LBM_T, 96><<<n_items, 96, 0, s>>>(cases, items, src, beta4, kappa, lambda,
                                                    vortex, vU, parity);
      break;
    case 128:
      init_items<LBM_T, 128><<<n_items, 128, 0, s>>>(cases, items, src, beta4, kappa, lambda,
                                                      vortex, vU, parity);
      break;
    case 192:
      init_items<LBM_T, 192><<<n_items, 192, 0, s>>>(cases, items, src, beta4, kappa, lambda,
                                                      vortex, vU, parity);
      break;
    case 256:
      init_items<LBM_T, 256><<<n_items, 256, 0, s>>>(cases, items, src, beta4, kappa, lambda,
                                                      vortex, vU, parity);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <>
cudaError_t launch_snapshot<LBM_T>(const LBM_T* f, const LBM_T* g, const LBM_T* J,
                                   const LBM_T* lo, int64_t P, int64_t n, LBM_T* out,
                                   cudaStream_t s) {
  const int planes = lo ? 21 : 20;
  const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 4096), planes);
  snapshot_kernel<LBM_T><<<grid, 256, 0, s>>>(f, g, J, lo, P, n, out);
  return cudaGetLastError();
}

template <>
cudaError_t launch_plane_import<LBM_T>(LBM_T* buf, int64_t P, const double* src, int i, int nx,
                                       int ny, int walls, cudaStream_t s) {
  plane_import<LBM_T><<<grid_for((int64_t)nx * ny, 256), 256, 0, s>>>(buf, P, src, i, nx, ny,
                                                                      walls);
  return cudaGetLastError();
}

template <>
cudaError_t launch_plane_export<LBM_T>(double* dst, const LBM_T* buf, int64_t P, int i, int nx,
                                       int ny, int walls, cudaStream_t s) {
  plane_export<LBM_T><<<grid_for((int64_t)nx * ny, 256), 256, 0, s>>>(dst, buf, P, i, nx, ny,
                                                                      walls);
  return cudaGetLastError();
}

template <>
cudaError_t launch_wall_f_fix<LBM_T>(double* v, const CaseDev<LBM_T>& cd, int par, int i,
                                     double sign, cudaStream_t s) {
  wall_f_fix<LBM_T><<<grid_for(2 * (int64_t)cd.nx, 256), 256, 0, s>>>(
      v, cd, par, i, (double)cd.rho_g, (double)cd.drho, sign);
  return cudaGetLastError();
}

template <>
cudaError_t launch_copy_to_T<LBM_T>(LBM_T* dst, const double* src, int64_t n, cudaStream_t s) {
  copy_to_T<LBM_T><<<grid_for(n, 256), 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

template <>
cudaError_t launch_copy_to_f64<LBM_T>(double* dst, const LBM_T* src, int64_t n, cudaStream_t s) {
  copy_to_f64<LBM_T><<<grid_for(n, 256), 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

template <>
cudaError_t launch_add_lo_f64<LBM_T>(double* v, const LBM_T* lo, int64_t n, cudaStream_t s) {
  add_lo_f64<LBM_T><<<grid_for(n, 256), 256, 0, s>>>(v, lo, n);
  return cudaGetLastError();
}

template <>
cudaError_t launch_lo_from_f64<LBM_T>(LBM_T* lo, const LBM_T* hi, const double* v, int64_t n,
                                      cudaStream_t s) {
  lo_from_f64<LBM_T><<<grid_for(n, 256), 256, 0, s>>>(lo, hi, v, n);
  return cudaGetLastError();
}

template <>
cudaError_t launch_volume_partial<LBM_T>(const CaseDev<LBM_T>* cases, const Item* items,
                                         int n_items, int bx, int parity, double* part,
                                         cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  switch (bx) {
    case 32: volume_partial<LBM_T, 32><<<n_items, 32, 0, s>>>(cases, items, parity, part); break;
    case 64: volume_partial<LBM_T, 64><<<n_items, 64, 0, s>>>(cases, items, parity, part); break;
    case 96: volume_partial<LBM_T, 96><<<n_items, 96, 0, s>>>(cases, items, parity, part); break;
    case 128: volume_partial<LBM_T, 128><<<n_items, 128, 0, s>>>(cases, items, parity, part); break;
    case 192: volume_partial<LBM_T, 192><<<n_items, 192, 0, s>>>(cases, items, parity, part); break;
    case 256: volume_partial<LBM_T, 256><<<n_items, 256, 0, s>>>(cases, items, parity, part); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <>
cudaError_t launch_volume_final<LBM_T>(const CaseDev<LBM_T>* cases, const int* case_ids,
                                       int ncases, const double* part, double* out,
                                       const int64_t* t, int64_t toff, int64_t slots,
                                       int64_t stride, cudaStream_t s) {
  if (ncases <= 0) return cudaSuccess;
  const int warps = 4;
  volume_final<LBM_T><<<(ncases + warps - 1) / warps, 32 * warps, 0, s>>>(
      cases, case_ids, ncases, part, out, t, toff, slots, stride);
  return cudaGetLastError();
}

}  // namespace lbmk
