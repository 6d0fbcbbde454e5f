// Single-precision (FP32-bulk) instantiation of the libvlb kernels.
#define VLB_REAL float
#include "vlb_kernels_impl.cuh"
