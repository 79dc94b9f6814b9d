// Three-dimensional kernels: arithmetic double, population storage double.
#include "kern3_impl.cuh"

namespace lbmk3 {
template struct K3<double, double>;
}  // namespace lbmk3

namespace lbmk3 {
cudaError_t volume3_final_launch(const double* part, int nparts, int stride, int nregions,
                                 double* out, cudaStream_t st) {
  volume3_final<<<nregions, 32, 0, st>>>(part, nparts, stride, nregions, out);
  return cudaGetLastError();
}
}  // namespace lbmk3
