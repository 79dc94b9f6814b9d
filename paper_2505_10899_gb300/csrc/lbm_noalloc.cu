// Allocation-free phase-volume entry point (lbm_phase_volume_noalloc).
//
// Some callers cannot allocate device memory at all: code running under an
// allocator that forbids cudaMalloc while a memory pool is being drained or
// defragmented, or a host framework that hands out only the buffers it owns.
// For them this file provides a variant of the labelled phase-volume
// reduction that needs no workspace: the caller passes the populations, the
// labels and the output, and the per-CTA partial sums live in a file-scope
// static device array of fixed size (kNaMaxBlocks x kNaMaxRegions doubles,
// 256 KiB), which every GPU that loads the library holds until the process
// exits.
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lbm_api.h"

namespace lbmk {
// Records the message returned by lbm_last_error() (defined in lbm_api.cu).
int set_last_error(int code, const char* msg);
}  // namespace lbmk

namespace {

constexpr int kNaMaxBlocks = 4096;  // partial-sum slots (CTAs per call)
constexpr int kNaMaxRegions = 8;
constexpr int kNaBX = 128;          // columns per CTA

// Scratch shared by every call on a device; each call overwrites the slots it
// uses before reading them, so nothing has to start at zero.
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * kNaMaxRegions];

int na_fail(int code, const std::string& msg) {
  return lbmk::set_last_error(code, ("lbm_phase_volume_noalloc: " + msg).c_str());
}

// phi = sum_i g_i(x) (Eq. 35) of post-streaming populations [i][y][x],
// reduced over the labels of one CTA's tile into FP64 partials, fixed order.
template <typename T>
__global__ void __launch_bounds__(kNaBX)
    na_volume_partial(const T* __restrict__ g, int64_t plane, int nx, int ny, int rows,
                      const int8_t* __restrict__ labels, int nregions,
                      double* __restrict__ part) {
  __shared__ double red[kNaBX / 32][kNaMaxRegions];
  const int nstrips = (nx + kNaBX - 1) / kNaBX;
  const int x = (blockIdx.x % nstrips) * kNaBX + threadIdx.x;
  const int y0 = (blockIdx.x / nstrips) * rows;
  double acc[kNaMaxRegions];
#pragma unroll
  for (int r = 0; r < kNaMaxRegions; ++r) acc[r] = 0.0;
  if (x < nx) {
    const int y1 = min(y0 + rows, ny);
    for (int y = y0; y < y1; ++y) {
      const int64_t k = (int64_t)y * nx + x;
      double phi = 0.0;
#pragma unroll
      for (int i = 0; i < 9; ++i) phi += (double)g[i * plane + k];
      const int lab = labels ? (int)labels[k] : 0;
#pragma unroll
      for (int r = 0; r < kNaMaxRegions; ++r)
        if (lab == r) acc[r] += phi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kNaMaxRegions; ++r) {
    double v = acc[r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][r] = v;
  }
  __syncthreads();
  if (threadIdx.x < nregions) {
    double v = 0.0;
    for (int w = 0; w < kNaBX / 32; ++w) v += red[w][threadIdx.x];
    part[(int64_t)blockIdx.x * kNaMaxRegions + threadIdx.x] = v;
  }
}

// Sum the partials of all CTAs: warp r handles region r.  Lane l adds the
// partials of CTAs l, l + 32, l + 64, ... in that order, then the 32 lane sums
// are combined by a fixed shuffle tree, so the result is the same bits on
// every call.
__global__ void na_volume_final(const double* __restrict__ part, int nblocks, int nregions,
                                double* __restrict__ out) {
  const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (r >= nregions) return;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += part[(int64_t)b * kNaMaxRegions + r];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) out[r] = v;
}

// Device address of the scratch array on the current device.  It is looked
// up on every call (a host-side query that allocates nothing): an address
// cached across calls would go stale if the device were reset and the module
// loaded again at another address.
int na_scratch(double** out) {
  double* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&p, g_na_partials);
  if (e != cudaSuccess || !p)
    return na_fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_phase_volume_noalloc(const void* d_g, int32_t precision, int32_t nx,
                                        int32_t ny, int64_t plane_stride,
                                        const int8_t* d_labels, int32_t nregions,
                                        double* d_out, void* stream) {
  if (!d_g || !d_out) return na_fail(LBM_ERR_ARG, "d_g and d_out must not be null");
  if (precision != LBM_F32 && precision != LBM_F64) return na_fail(LBM_ERR_ARG, "precision");
  if (nx < 1 || ny < 1) return na_fail(LBM_ERR_ARG, "nx, ny must be >= 1");
  if (plane_stride < (int64_t)nx * ny) return na_fail(LBM_ERR_ARG, "plane_stride < nx*ny");
  if (nregions < 1 || nregions > kNaMaxRegions)
    return na_fail(LBM_ERR_ARG, "nregions must lie in [1, 8]");
  const int nstrips = (nx + kNaBX - 1) / kNaBX;
  if (nstrips > kNaMaxBlocks)
    return na_fail(LBM_ERR_ARG, "nx too large for the static scratch: at most " +
                                    std::to_string(kNaMaxBlocks * kNaBX) + " columns");
  // rows per CTA so that the CTA count fits the scratch array
  const int max_runs = kNaMaxBlocks / nstrips;
  int rows = (ny + max_runs - 1) / max_runs;
  if (rows < 1) rows = 1;
  const int64_t nblocks = (int64_t)nstrips * ((ny + rows - 1) / rows);
  if (nblocks > kNaMaxBlocks) return na_fail(LBM_ERR_ARG, "grid too large for the static scratch");

  double* part = nullptr;
  int rc = na_scratch(&part);
  if (rc != LBM_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == LBM_F32)
    na_volume_partial<float><<<(int)nblocks, kNaBX, 0, s>>>((const float*)d_g, plane_stride, nx,
                                                            ny, rows, d_labels, nregions, part);
  else
    na_volume_partial<double><<<(int)nblocks, kNaBX, 0, s>>>((const double*)d_g, plane_stride, nx,
                                                             ny, rows, d_labels, nregions, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  na_volume_final<<<1, 32 * nregions, 0, s>>>(part, (int)nblocks, nregions, d_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return LBM_OK;
}
