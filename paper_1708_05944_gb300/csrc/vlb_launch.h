// Host-side launchers of the libvlb kernels (one translation unit per precision).
#pragma once
#include <cuda_runtime.h>

#include "vlb_device.cuh"

namespace vlb {

template <typename real>
struct StageArgs;

// Launch shape of the stage kernel: cells per tile and threads per CTA.
struct StageVariant {
  int tc, nt;
};

// The launch shapes available for a model shape (at most 8); the first is the default.
template <typename real>
int stage_variants(int nq0, int nq1, StageVariant* out);

// Dynamic shared memory the stage kernel needs for a variant and per-field stride Vp.
template <typename real>
size_t stage_smem_bytes(StageVariant v, int Vp);

// Launch one RK3 stage over a.n_tiles tiles of v.tc cells.
template <typename real>
cudaError_t launch_stage(StageVariant v, const StageArgs<real>& a, const ModelArgs& m, const KArgs<real>& k,
                         cudaStream_t s);

// f_eq(n0, (u0, u1), T0) in every cell.
template <typename real>
cudaError_t launch_init_equilibrium(real* F, long long cells, int Vp, const ModelArgs& m, double n0, double u0,
                                    double u1, double T0, cudaStream_t s);

// Per cell, FP64: n, u0, u1, T, T00, T01, T11, q0, q1 (stride 9).
template <typename real>
cudaError_t launch_moments(const real* F, long long cells, int Vp, const ModelArgs& m, double* out, cudaStream_t s);

// Per instance L2 norms of Eq. (msites_steady) between mom and prev (stride 9 per cell), into res (3 per instance).
cudaError_t launch_residual(const double* mom, const double* prev, const InstDesc* inst, const GeoCell* geo,
                            int n_inst, double* res, cudaStream_t s);

}  // namespace vlb
