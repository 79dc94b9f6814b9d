// Three-dimensional kernels: arithmetic float, population storage float.
#include "kern3_impl.cuh"

namespace lbmk3 {
template struct K3<float, float>;
}  // namespace lbmk3
