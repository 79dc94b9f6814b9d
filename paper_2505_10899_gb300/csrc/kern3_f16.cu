// Three-dimensional kernels: arithmetic float, population storage __half.
#include "kern3_impl.cuh"

namespace lbmk3 {
template struct K3<float, __half>;
}  // namespace lbmk3
