// Host-side launchers of the libvlb kernels (one translation unit per precision).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "vlb_device.cuh"
#include "vlb_tables.h"

namespace vlb {

template <typename real>
struct StageArgs;

// Launch shape of the stage kernel: cells per tile and threads per CTA.
struct StageVariant {
  int tc, nt;
  int persist;  // 0: one CTA per tile; 1: persistent CTAs walk the tile list
};

// The launch shapes available for a model shape (at most 8); the first is the default.
template <typename real>
int stage_variants(int nq0, int nq1, StageVariant* out);

// Dynamic shared memory the stage kernel needs for a variant and per-field stride Vp.
template <typename real>
size_t stage_smem_bytes(StageVariant v, int Vp);

// Whether the stage kernels of a model shape are the fixed-shape ones, which read
// the force kernels in split form (KArgs::split); the others read them whole.
template <typename real>
bool stage_split_tables(int nq0, int nq1);

// Launch configuration of a stage launch shape on the current device: tile
// buffers (StageArgs::nbuf) and resident CTAs per SM (0 if none fit).  Also
// raises the kernel's dynamic shared-memory limit to what the configuration
// needs, which its launches rely on; a context computes it once per shape.
// ft: the f~ instance (the first launch shape of the velocity set's shape only).
template <typename real>
cudaError_t stage_config(StageVariant v, const ModelArgs& m, int Vp, int* nbuf, int* per_sm, bool ft = false);

// Launch one RK3 stage over a.n_tiles tiles of at most v.tc cells on `grid` CTAs
// (a.nbuf as stage_config gave it).
template <typename real>
cudaError_t launch_stage(StageVariant v, const StageArgs<real>& a, const ModelArgs& m, const KArgs<real>& k, int grid,
                         cudaStream_t s, bool ft = false);

// Launch shapes of the channel stage kernel: ts lambda rows per segment of a
// CTA's march (0: chosen by the host from the SM count; at least n_lambda: one
// segment), tp xi-columns per strip, nt threads ((tp + 1) x velocities).
struct ChanVariant {
  int ts, tp, nt;
  int tc;  // single precision: force contraction on the tensor cores (1) or the CUDA cores (0)
};
template <typename real>
struct ChanArgs;

// Channel launch shapes for a model shape (at most 8); 0 if the shape has no channel kernel.
int channel_variants(int nq0, int nq1, ChanVariant* out);
template <typename real>
size_t channel_smem_bytes(ChanVariant v, int nq0, int nq1);
// The ChanTables block of a model shape (bytes, bulk-copied by every CTA) for the
// axis tables, the model arguments and the reservoir / wall temperature T0; false
// if the shape has no channel kernel.
template <typename real>
bool channel_tables(int nq0, int nq1, const AxisTables* ax, const ModelArgs& m, double T0,
                    std::vector<unsigned char>* out);
// One channel stage on `grid` CTAs (a.nx / v.tp strips x a.nseg segments).
// The split force block (ChanKP) of a model shape from the full matrices of the two
// axes; false if the shape has no channel kernel or a matrix lacks the reflection
// symmetry the split relies on.
bool channel_force_pairs(int nq0, int nq1, const AxisTables* ax, std::vector<unsigned char>* out);
// clb: the Cartesian-split formulation on the same march (a.geo then holds its geometry records)
template <typename real>
cudaError_t launch_channel(ChanVariant v, const ChanArgs<real>& a, const void* kp, int nq0, int nq1, int grid,
                           cudaStream_t s, bool clb = false);

// Order of a context's cells in device buffers against the caller's order.
// Couette contexts keep the caller's order (nx = 0).  Channel contexts store cell
// (s, p) at s * nx + p (xi fastest, one lambda row of the channel after another)
// and callers see it at p * nl + s (one xi column after another).
struct CellMap {
  int nl = 0, nx = 0;
};
__host__ __device__ __forceinline__ long long caller_cell(const CellMap& m, long long q) {
  if (m.nx == 0) return q;
  const long long s = q / m.nx, p = q - s * m.nx;
  return p * m.nl + s;
}

// f_eq(n0, (u0, u1), T0) in every cell.
template <typename real>
cudaError_t launch_init_equilibrium(real* F, long long cells, int Vp, const ModelArgs& m, double n0, double u0,
                                    double u1, double T0, cudaStream_t s);

// Grad heat-flux form of n_c, (u0_c, u1_c), T_c, q0_c (q0 may be null: zero
// flux, the truncated equilibrium) projected on the model, per cell from device arrays.
template <typename real>
cudaError_t launch_seed(real* F, long long cells, int Vp, const ModelArgs& m, const double* n, const double* u0,
                        const double* u1, const double* T, const double* q0, cudaStream_t s, CellMap map = CellMap{});

// Caller layout F (per cell: f' then f'', V values each) to and from the device
// layout (per cell: Vp interleaved (f', f'') pairs of the deviation D = F - R;
// padding zero).  to_deviation = 1: caller -> device, 0: device -> caller; each
// element is summed in double.  src and dst may be the same buffer when V == Vp and
// the cell map is the identity.
template <typename real>
cudaError_t launch_deviation(const real* src, real* dst, long long cells, int Vp, const ModelArgs& m,
                             int to_deviation, cudaStream_t s, CellMap map = CellMap{});

// Shakhov correction of a stage (see shakhov_kernel): F_out += cc dt (1 - Pr) G[F_prev] / tau per
// cell, the moments taken from F_prev by the same kernel (device cell order); kn_fixed > 0:
// tau = kn_fixed / (n T) for every cell, else each cell's instance (Kn, tau convention); dt from
// the instance.
template <typename real>
cudaError_t launch_shakhov(real* Fout, const real* Fprev, long long cells, int Vp, const ModelArgs& m,
                           const InstDesc* inst, int n_inst, double cc, double one_minus_pr, double kn_fixed,
                           cudaStream_t s);

// Model tables of a Couette context beyond the fused kernels' 32 nodes per axis (device
// pointers; tab rows have stride MAXN; K0 is d/dp on axis 0, Kt1 d/dp (p .) on axis 1).
struct LargeModel {
  int nq0, nq1, V, Vp, N0, N1, kind0, kind1;
  const double *p0, *p1, *w0, *w1, *iw0, *iw1, *tab0, *tab1, *K0, *Kt1;
  // single precision: the symmetric scaling sqrt(w_k' / w_k) K of both matrices (entries of
  // order Q^(3/2); K itself reaches 1e117 at Q = 200), with sqrt(w) and 1/sqrt(w) (capped at 1e30)
  const float *K0f, *Kt1f, *s0f, *is0f, *s1f, *is1f;
  double ref_flux_neg, ref_flux_pos;  // outgoing particle flux of R at the inner / outer wall
  unsigned* err;
  // the f~ formulation (Eqs. boltz_couette_cons, boltz_couette_str_cons) when ftilde != 0: per
  // cell sqrt(g), the advection factors e_{s+1/2} / (d eta sqrt(g_s)) and e_{s-1/2} / (...),
  // and 1 / R_s of the force term
  int ftilde;
  const double *sqrtg, *advp, *advm, *inv_r;
  // per velocity (p1_j^2 (K0 R)_ij - p0_i (Kt1 R)_ij), R_ij = w0_i w1_j: the inertial term of the
  // rest state, which the chi form drops with the advection of R (they cancel) and f~ must keep
  const double* forceR;
};

// One RK3 stage of the large-set Couette path (see vlb_large.cu): walls holds per
// (instance, wall) g0 (nq0), g1 (nq1) of f_eq(1, (0, u_w), T_w), the incoming flux and T_w;
// rec (cells x (nq0 + nq1 + 2)), force (lm_force_reals) and part (lm_part_doubles) are scratch.
template <typename real>
cudaError_t lm_stage(const LargeModel& m, const real* Fprev, const real* Fl, real* Fout, long long cells,
                     const InstDesc* inst, int n_inst, const GeoCell* geo, const double* walls, double* nw,
                     real* rec, real* force, double* part, double ca, double cc, cudaStream_t s);
size_t lm_part_doubles(const LargeModel& m, long long cells, int n_inst);
size_t lm_force_reals(const LargeModel& m, long long cells);  // the force scratch, in reals
// The Cartesian-split channel (Sec. VII.G): geometry of the advection velocities
// V^lambda = va_p (p^x - lambda_{s+1/2} dph_p p^y) and V^xi = vx_{p+1/2} p^y, device arrays.
struct ClbGeom {
  int nl, nx;
  const double *va, *dph;  // [nx] 1 / (1 + phi(xi_p)), phi'(xi_p)
  const double* lf;        // [nl + 1] lambda_{s+1/2}
  const double* vx;        // [nx + 1] 1 + phi(xi_{p+1/2})
  const double *idl, *idx;  // [nl] 1 / d lambda_s, [nx] 1 / d chi_p
  const double* weq;       // [nq0 + nq1] factors of f_eq(1, 0, T0) (the wall)
  double kn, n_in, n_out, T0;
  const int* ibar;         // [nq0] the p^x mirror of each axis-0 node
};

// One RK3 stage of the Cartesian-split channel: rec (cells x (nq0 + nq1 + 2)) and res
// (nl x 2 x (nq0 + nq1)) are scratch; nw gets n_w per column.  Device cell s * nx + p.
template <typename real>
cudaError_t clb_stage(const LargeModel& m, const ClbGeom& g, const real* Fprev, const real* Fl, real* Fout, real* rec,
                      real* res, double* nw, double dt, double ca, double cc, cudaStream_t s);

template <typename real>
cudaError_t lm_deviation(const LargeModel& m, const real* src, real* dst, long long cells, int to_dev, cudaStream_t s);
template <typename real>
cudaError_t lm_init(const LargeModel& m, real* F, long long cells, double n, double u0, double u1, double T,
                    cudaStream_t s);
template <typename real>
cudaError_t lm_moments(const LargeModel& m, const real* F, long long cells, double* out, cudaStream_t s);

// Per cell, FP64: n, u0, u1, T, T00, T01, T11, q0, q1 (stride 9).
template <typename real>
cudaError_t launch_moments(const real* F, long long cells, int Vp, const ModelArgs& m, double* out, cudaStream_t s,
                           CellMap map = CellMap{});

// Per instance L2 norms of Eq. (msites_steady) between mom and prev (stride 9 per cell), into res (3 per instance).
cudaError_t launch_residual(const double* mom, const double* prev, const InstDesc* inst, const GeoCell* geo,
                            int n_inst, double* res, cudaStream_t s);
cudaError_t launch_channel_post(const double* mom, const double* tab, int nl, int nx, double dxi, double* ux,
                                double* uy, double* omega, double* psi, double* pw, cudaStream_t s);

}  // namespace vlb
