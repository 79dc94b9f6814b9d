// Host-side launch wrappers of the device kernels (one translation unit per
// precision instantiates them).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_layout.h"

namespace lbmk {

// Strip widths of a tiling (threads per CTA of the step kernels).
inline bool valid_bx(int bx) { return bx == 32 || bx == 64 || bx == 128; }

// Strip widths the bulk-copy kernel also runs, for cases whose whole row is
// one strip of that width (their own chains, see lbm_api.cu).
inline bool row_bx(int bx) { return bx == 96 || bx == 192 || bx == 256; }

// tma: use the bulk-copy staged kernel (every case must have nx a multiple
// of 16 bytes of T and nx >= 4), else the register-pipelined kernel.
template <typename T>
cudaError_t launch_step(const StepArgs<T>& a, int bx, bool coupled, int mode, bool tma,
                        int n_items, cudaStream_t s);

// Persistent register-path kernel (cooperative launch): nsteps steps in one
// launch; grid = min(n_items, co-resident CTAs).  count/gen: grid-barrier
// words (zero-initialised, device).
template <typename T>
cudaError_t launch_persistent(const StepArgs<T>& a, int bx, bool coupled, int n_items,
                              int nsteps, int flip, unsigned int* count, unsigned int* gen,
                              cudaStream_t s);

// Allow the dynamic shared memory of every TMA kernel variant on the current
// device (call once per device before the first launch or graph capture).
template <typename T>
cudaError_t prepare_tma();

// Dynamic shared memory of the TMA kernel variant (0 if not available).
template <typename T>
size_t tma_smem_bytes(int bx, bool coupled, int mode);

// Initial state of every case in one launch over the work items (bx columns
// per CTA); src: per-case device-readable pointers to phi0 and u0.
template <typename T>
cudaError_t launch_init_items(const CaseDev<T>* cases, const Item* items, int n_items, int bx,
                              const InitSrc* src, double beta4, double kappa, double lambda,
                              int vortex, double vU, int parity, cudaStream_t s);

// buf: the 9-plane buffer with plane stride P (walls: bounce-back positions)
template <typename T>
cudaError_t launch_plane_import(T* buf, int64_t P, const double* src, int i, int nx, int ny,
                                int walls, cudaStream_t s);
template <typename T>
cudaError_t launch_plane_export(double* dst, const T* buf, int64_t P, int i, int nx, int ny,
                                int walls, cudaStream_t s);
// moving-wall term of f plane i at the wall rows, added (sign 1) or removed (-1)
template <typename T>
cudaError_t launch_wall_f_fix(double* v, const CaseDev<T>& cd, int par, int i, double sign,
                              cudaStream_t s);
// One case's snapshot (lbm_snapshot layout) in one launch; lo may be null.
template <typename T>
cudaError_t launch_snapshot(const T* f, const T* g, const T* J, const T* lo, int64_t P,
                            int64_t n, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_to_T(T* dst, const double* src, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_to_f64(double* dst, const T* src, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_add_lo_f64(double* v, const T* lo, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_lo_from_f64(T* lo, const T* hi, const double* v, int64_t n, cudaStream_t s);

// Per-item partial volumes (labelled regions) of the state in buffer parity.
template <typename T>
cudaError_t launch_volume_partial(const CaseDev<T>* cases, const Item* items, int n_items,
                                  int bx, int parity, double* part, cudaStream_t s);

// Per-case sums of the item partials (written by the step kernel's fused
// volume or by launch_volume_partial): the cases case_ids[0..ncases), or
// cases 0..ncases-1 with case_ids null.
template <typename T>
cudaError_t launch_volume_final(const CaseDev<T>* cases, const int* case_ids, int ncases,
                                const double* part, double* out, const int64_t* t, int64_t toff,
                                int64_t slots, int64_t stride, cudaStream_t s);

cudaError_t launch_clock(int64_t* t, int64_t n, cudaStream_t s);
cudaError_t launch_set_clock(int64_t* t, int64_t value, cudaStream_t s);

}  // namespace lbmk
