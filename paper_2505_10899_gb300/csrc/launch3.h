// Host-side launch interface of the three-dimensional kernels, one explicit
// instantiation per (arithmetic, storage) pair in kern3_f64.cu, kern3_f32.cu
// and kern3_f16.cu.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmk3 {

struct Bufs {
  void* f[2];
  void* g[2];
  void* g0[2];
  void* g0lo[2];  // null under FP64 arithmetic
  void* J[2];
};

// Launch-uniform values in FP64; each instantiation rounds them once.
struct Host3 {
  int32_t nx, ny, nz, var_tau;
  int64_t plane;
  double beta4, kappa, lambda, lamW, xi, tfac, wg, hg, wf, hf, rho_g, drho, mu_g, dmu;
  double W;  // interface width (the threshold of the normal scales with it)
};

inline bool tile_ok(int bx, int by) {
  return (bx == 32 && (by == 4 || by == 8 || by == 16)) || (bx == 64 && by == 4);
}

inline int64_t n_ctas(int nx, int ny, int nz, int bx, int by, int zc) {
  return (int64_t)((nx + bx - 1) / bx) * ((ny + by - 1) / by) * ((nz + zc - 1) / zc);
}

// Step-kernel variants: register-pipelined loads (any precision), or
// asynchronous copies through shared memory with 2 or 3 stages (FP32 only).
enum { kVarRegs = 1, kVarAsync2 = 2, kVarAsync3 = 3 };

inline bool variant_ok(int variant, int precision_is_f32, int bx, int by) {
  if (variant == kVarRegs) return tile_ok(bx, by);
  if (variant == kVarAsync2 || variant == kVarAsync3)
    return precision_is_f32 && ((bx == 32 && (by == 4 || by == 8)) || (bx == 64 && by == 4));
  return false;
}

template <typename T, typename S>
struct K3 {
  static cudaError_t step(const Bufs& b, const Host3& h, int parity, int variant, int bx, int by,
                          int zc, int mode, int32_t* flags, double* vol_part, double* out,
                          int which, cudaStream_t st);
  static cudaError_t init(const Bufs& b, const Host3& h, int parity, const double* d_phi0,
                          const double* d_u0, cudaStream_t st);
  static cudaError_t plane(const Bufs& b, const Host3& h, int parity, int kind, int i,
                           double* d_buf, int to_device, cudaStream_t st);
  static cudaError_t volume(const Bufs& b, const Host3& h, int parity, const int8_t* labels,
                            int nregions, double* part, int nparts, double* out,
                            cudaStream_t st);
};

cudaError_t volume3_final_launch(const double* part, int nparts, int stride, int nregions,
                                 double* out, cudaStream_t st);

}  // namespace lbmk3
