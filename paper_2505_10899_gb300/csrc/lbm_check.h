// Debug build with index checks (compile with -DLBM_CHECK_BOUNDS; the
// library then builds as liblbm_gb300_checked.so).  In that build every
// global load and store of the 2-D step kernels (bulk-copy, register-
// pipelined and persistent) and the source and target range of every bulk
// copy are compared with the extent of the array they address.  An index out of range raises
// kFlagBounds in the launch's flag word (reported as LBM_ERR_BOUNDS) and the
// access is skipped (a bulk copy is redirected to the start of its own
// buffer, so that its barrier still completes).  In the normal build the
// checks compile to nothing.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbmk {

enum { kFlagBounds = 4 };

#ifdef LBM_CHECK_BOUNDS
__device__ __forceinline__ bool bound_ok(int32_t* flags, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  if (flags) atomicOr(flags, kFlagBounds);
  return false;
}
#define LBM_BOUND(flags, i, n) (::lbmk::bound_ok((flags), (long long)(i), (long long)(n)))
#else
#define LBM_BOUND(flags, i, n) true
#endif

}  // namespace lbmk
