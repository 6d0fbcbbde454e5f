// Single-precision (FP32-bulk) instantiation of the libvlb kernels.
#define VLB_REAL float
#define VLB_DEFINE_SHARED
#include "vlb_kernels_impl.cuh"
