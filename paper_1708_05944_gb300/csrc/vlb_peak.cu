// Measured FP64 FMA throughput of the current device: the denominator of the
// roofline of the double-precision stage kernels, which are bound by the FP64
// pipe rather than by memory.  Eight independent fma chains per thread keep the
// pipe busy; the result is written only when it cannot occur, so the chains are
// not removed.
#include <cuda_runtime.h>

#include "../../include/vlb.h"

namespace {

__global__ void fp64_fma_chains(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == -1.0) out[0] = s;
}

}  // namespace

extern "C" vlb_status vlb_peak_fp64(double* tflops) {
  if (!tflops) return VLB_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return VLB_ERR_CUDA;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) return VLB_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8, iters = 1 << 14;
  fp64_fma_chains<<<blocks, threads>>>(d, 256, 0.9999999, 1e-7);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    fp64_fma_chains<<<blocks, threads>>>(d, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return VLB_ERR_CUDA;
  *tflops = 2.0 * 8.0 * double(iters) * double(threads) * double(blocks) / (double(best) * 1e-3) / 1e12;
  return VLB_OK;
}
