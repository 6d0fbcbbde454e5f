// Double-precision instantiation of the libvlb kernels.
#define VLB_REAL double
#include "vlb_kernels_impl.cuh"
