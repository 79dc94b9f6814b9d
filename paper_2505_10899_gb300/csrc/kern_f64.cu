// FP64 instantiation of the device kernels.
#define LBM_T double
#include "kern_impl.cuh"

namespace lbmk {
cudaError_t launch_clock(int64_t* t, int64_t n, cudaStream_t s) {
  clock_kernel<<<1, 32, 0, s>>>(t, n);
  return cudaGetLastError();
}
cudaError_t launch_set_clock(int64_t* t, int64_t value, cudaStream_t s) {
  set_clock_kernel<<<1, 32, 0, s>>>(t, value);
  return cudaGetLastError();
}
}  // namespace lbmk
