// Host-side launch interface of the three-dimensional kernels, one explicit
// instantiation per (arithmetic, storage) pair in kern3_f64.cu, kern3_f32.cu
// and kern3_f16.cu.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm3_layout.h"

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
  long long wait_cycles = lbmk::kWaitCycles;  // bound of the bulk-copy kernels' waits
};

// Tiles of the register-pipelined and asynchronous-copy kernels.
inline bool tile_regs_ok(int bx, int by) {
  return (bx == 32 && (by == 4 || by == 8 || by == 16)) || (bx == 64 && by == 4);
}
// Tiles of the bulk-copy kernel: whole x-rows, 128 x 4 or 256 x 2.
inline bool tile_bulk_ok(int bx, int by) { return (bx == 128 && by == 4) || (bx == 256 && by == 2); }
// Tiles of the strip bulk-copy kernel (nx a multiple of bx, nx >= 2 bx).
inline bool tile_strip_ok(int bx, int by) { return (bx == 32 && by == 8) || (bx == 64 && by == 4); }
// Tiles of the strip kernel's occupancy form (two stages, more CTAs per SM).
inline bool tile_strip_occ_ok(int bx, int by) { return bx == 64 && (by == 4 || by == 2); }
inline bool tile_ok(int bx, int by) {
  return tile_regs_ok(bx, by) || tile_bulk_ok(bx, by) || tile_strip_ok(bx, by) ||
         tile_strip_occ_ok(bx, by);
}

inline int64_t n_ctas(int nx, int ny, int nz, int bx, int by, int zc) {
  return (int64_t)((nx + bx - 1) / bx) * ((ny + by - 1) / by) * ((nz + zc - 1) / zc);
}

// Step-kernel variants: register-pipelined loads (any precision);
// asynchronous copies through shared memory with 2 or 3 stages (FP32 only);
// bulk copies of whole rows into shared memory (FP32 arithmetic, FP32 or
// FP16 storage; rows of nx <= bx values, nx values a multiple of 16 bytes);
// bulk copies of padded strip-row segments (FP32 arithmetic, FP32 or FP16
// storage; nx a multiple of bx and at least two strips), with two or three
// stages and two CTAs per SM (5), or two stages and three (64 x 4) or five
// (64 x 2) CTAs per SM at fewer registers (6).
enum { kVarRegs = 1, kVarAsync2 = 2, kVarAsync3 = 3, kVarBulk = 4, kVarStrip = 5,
       kVarStripOcc = 6 };

// sbytes: bytes of a stored population (8 FP64, 4 FP32, 2 FP16).
inline bool variant_ok(int variant, int sbytes, int bx, int by, int nx) {
  if (variant == kVarRegs) return tile_regs_ok(bx, by);
  if (variant == kVarAsync2 || variant == kVarAsync3)
    return sbytes == 4 && ((bx == 32 && (by == 4 || by == 8)) || (bx == 64 && by == 4));
  if (variant == kVarBulk)
    return sbytes != 8 && tile_bulk_ok(bx, by) && nx <= bx && (nx * sbytes) % 16 == 0 &&
           (nx * 4) % 16 == 0;
  if (variant == kVarStrip)
    return sbytes != 8 && tile_strip_ok(bx, by) && nx % bx == 0 && nx >= 2 * bx;
  if (variant == kVarStripOcc)
    return sbytes != 8 && tile_strip_occ_ok(bx, by) && nx % bx == 0 && nx >= 2 * bx;
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
