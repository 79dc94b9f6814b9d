// FP32 instantiation of the device kernels.
#define LBM_T float
#include "kern_impl.cuh"
