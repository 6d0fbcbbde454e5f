// Circular Couette stage for velocity sets beyond the fused stage kernel's 32 nodes per
// axis (the high-order half-range models of Sec. VI.D, e.g. HH(4;200) x HH(4;10), 8000
// velocities).  A cell row no longer fits a tile in shared memory, so the stage runs as
// four kernels over device memory (L2-resident at these sizes):
//
//   sums   -- per cell and chunk of 1024 velocities the sums of the moments (Eqs.
//             macro_red, mom_quad), and per wall and chunk the outgoing WENO-5 flux of the
//             extrapolated populations (Eqs. extrapol, nw), FP64, spread over many CTAs;
//   cell   -- per cell n, u, T from its chunk sums (in a fixed order), tau and the
//             truncated equilibrium factors (Sec. IV.D) normalised to sum n;
//   force  -- the radial part of the inertial term -(1/R)(p^phi)^2 K^R f (Eq.
//             boltz_couette_kom): per cell the contraction over the nq0 radial nodes is
//             a dense (nq0 x nq0) x (nq0 x 2 nq1) product, run as a shared-memory tiled
//             GEMM;
//   update -- one thread per (cell, velocity): WENO-5 at both interfaces along R from
//             the cell's neighbours or, past a wall, its ghosts (Eq. weno_populate: the
//             extrapolation of the outgoing half, n_w from the wall's chunk sums times the
//             wall equilibrium for the incoming half, built in place), the chi flux
//             difference, the azimuthal part of the inertial term (nq1 terms), BGK and
//             the RK3 combine, both fields as a pair.
// Every sum is taken in a fixed order, so results do not depend on scheduling.
//
// The same kernels run the f~ formulation (LargeModel::ftilde, Sec. VI.B): the stencils and
// the wall construction act on F~ = sqrt(g) f, whose flux difference e_{s+1/2} F~_{s+1/2} -
// e_{s-1/2} F~_{s-1/2} over d eta sqrt(g_s) is the advection of f; the force takes 1 / R_s.
//
// The arithmetic is that of the fused kernel: deviations D = F - R stored, the same
// epsilon-free pair WENO, the same wall construction.  In single precision the WENO
// indicator scale 1 / (w_i w_j) is capped at 1e30: tail populations below ~1e-38 are
// zero in single precision, and for the others the cap leaves the (scale-invariant)
// weights unchanged.
#include <cuda_runtime.h>

#include "vlb_launch.h"

namespace vlb {
namespace {

constexpr int kCellThreads = 256;  // per-cell and initial-state kernels
constexpr int kChunk = 1024;       // velocities per CTA of the partial-sum kernels (256 threads x 4)

// Sum over the block (all threads call it); warp 0 adds the warp partials.
__device__ double block_sum(double v, double* red) {
  v = warp_sum<double>(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum<double>(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ int instance_of(const InstDesc* inst, int n_inst, long long c) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].cell0 <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename real>
__device__ __forceinline__ real weno_scale(double iw) {
  if constexpr (sizeof(real) == 4) return real(iw < 1e30 ? iw : 1e30);
  else return real(iw);
}

// Equilibrium factors of (n, u0, u1, T) into g0 (carrying n, normalised so that
// sum_ij g0_i g1_j = n, reading of Sec. IV.D) and g1: shared arrays, whole block.
__device__ void eq_factors(const LargeModel& m, double n, double u0, double u1, double T, double* g0, double* g1,
                           double* mv, double* red) {
  if (threadIdx.x < 4) {
    const int ax = threadIdx.x >> 1, side = threadIdx.x & 1;
    const double u = (ax ? u1 : u0) * (side ? -1.0 : 1.0);
    eq_moment_vector<double>(ax ? m.kind1 : m.kind0, ax ? m.N1 : m.N0, u, T, mv + threadIdx.x * MAXN);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m.nq0 + m.nq1; k += blockDim.x) {
    const int ax = k >= m.nq0, j = ax ? k - m.nq0 : k;
    const double* tab = ax ? m.tab1 : m.tab0;
    const int kind = ax ? m.kind1 : m.kind0, N = ax ? m.N1 : m.N0;
    const double p = ax ? m.p1[j] : m.p0[j];
    const double* v = mv + (2 * ax + ((kind == 1 && p < 0.0) ? 1 : 0)) * MAXN;
    double g = 0.0;
    for (int s = 0; s <= N; ++s) g += tab[j * MAXN + s] * v[s];
    if (ax) g1[j] = g;
    else g0[j] = n * g;
  }
  __syncthreads();
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < m.nq0; k += blockDim.x) a += g0[k];
  for (int k = threadIdx.x; k < m.nq1; k += blockDim.x) b += g1[k];
  const double s0 = block_sum(a, red), s1 = block_sum(b, red);
  const double sc = n / (s0 * s1);
  for (int k = threadIdx.x; k < m.nq0; k += blockDim.x) g0[k] *= sc;
  __syncthreads();
}

// ---------------------------------------------------------------- partial sums
// part[(c NP + p) 4 + k]: over the velocities p kChunk .. (p + 1) kChunk of cell c, the sums
// of f', p^0 f', p^1 f' and (p^0^2 + p^1^2) f' + f'' (F = D + R), FP64
template <typename real>
__global__ void __launch_bounds__(256) lm_partial_kernel(const LargeModel m, const real* F, double* part) {
  __shared__ double red[4][8];
  const long long c = blockIdx.x;
  const int p = blockIdx.y, NP = gridDim.y;
  const real* f = F + c * 2 * m.Vp;
  double q[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < kChunk / 256; ++k) {
    const int v = p * kChunk + k * 256 + threadIdx.x;
    if (v >= m.V) break;
    const int i = v / m.nq1, j = v - i * m.nq1;
    const double r = m.w0[i] * m.w1[j];
    const double f1 = double(f[2 * v]) + r, f2 = double(f[2 * v + 1]) + r;
    const double a = m.p0[i], b = m.p1[j];
    q[0] += f1;
    q[1] += a * f1;
    q[2] += b * f1;
    q[3] += (a * a + b * b) * f1 + f2;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double t = warp_sum<double>(q[k]);
    if (lane == 0) red[k][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[threadIdx.x][k];
    part[(c * NP + p) * 4 + threadIdx.x] = t;
  }
}

// wpart[(ii 2 + wall) NP + p]: the outgoing particle flux at the wall of the WENO-5 interface
// values of the extrapolated populations (Eqs. extrapol, nw) over one chunk of velocities
template <typename real>
__global__ void __launch_bounds__(256) lm_wallpart_kernel(const LargeModel m, const real* F, const InstDesc* inst,
                                                          double* wpart) {
  __shared__ double red[8];
  using P = pair_t<real>;
  const int ii = blockIdx.x, wall = blockIdx.y, p = blockIdx.z, NP = gridDim.z;
  const InstDesc d = inst[ii];
  const long long edge = d.cell0 + (wall == 0 ? 0 : d.n_cells - 1);
  const int dir = wall == 0 ? 1 : -1;
  const double sgn = wall == 0 ? 1.0 : -1.0;  // incoming half: p^R > 0 at the inner wall
  const real* F0r = F + edge * 2 * m.Vp;
  const real* F1r = F + (edge + dir) * 2 * m.Vp;
  const real* F2r = F + (edge + 2 * dir) * 2 * m.Vp;
  double num = 0.0;
  for (int k = 0; k < kChunk / 256; ++k) {
    const int v = p * kChunk + k * 256 + threadIdx.x;
    if (v >= m.V) break;
    const int i = v / m.nq1, j = v - i * m.nq1;
    if (!(sgn * m.p0[i] < 0.0)) continue;
    P F0 = p_load(F0r + 2 * v), F1 = p_load(F1r + 2 * v), F2 = p_load(F2r + 2 * v);
    if (m.ftilde) {  // the walls act on F~ = sqrt(g) (D + R)
      const real R = real(m.w0[i] * m.w1[j]);
      F0 = p_mul(p_add(F0, p_set(R)), p_set(real(m.sqrtg[edge])));
      F1 = p_mul(p_add(F1, p_set(R)), p_set(real(m.sqrtg[edge + dir])));
      F2 = p_mul(p_add(F2, p_set(R)), p_set(real(m.sqrtg[edge + 2 * dir])));
    }
    const P G0 = p_fma(F1, p_set(real(-3)), p_fma(F0, p_set(real(3)), F2));
    const P G1 = p_fma(F1, p_set(real(-8)), p_fma(F0, p_set(real(6)), p_mul(F2, p_set(real(3)))));
    num += double(weno5p<real>(F2, F1, F0, G0, G1, weno_scale<real>(m.iw0[i] * m.iw1[j])).x) * m.p0[i];
  }
  num = warp_sum<double>(num);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = num;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    wpart[(size_t(ii) * 2 + wall) * NP + p] = t;
  }
}

// ---------------------------------------------------------------- cell kernel
// rec per cell: g0 (nq0, carrying n), g1 (nq1), T, 1/tau; moments from the partial sums
template <typename real>
__global__ void __launch_bounds__(kCellThreads) lm_cell_kernel(const LargeModel m, long long cells, int NP,
                                                               const double* part, const InstDesc* inst, int n_inst,
                                                               real* rec) {
  extern __shared__ double sh[];
  double* g0 = sh;
  double* g1 = g0 + m.nq0;
  double* mv = g1 + m.nq1;
  double* red = mv + 4 * MAXN;  // 33 entries
  double* q = red + 33;         // 4 entries
  const int stride = m.nq0 + m.nq1 + 2;
  for (long long c = blockIdx.x; c < cells; c += gridDim.x) {
    if (threadIdx.x < 4) {
      double t = 0.0;
      for (int p = 0; p < NP; ++p) t += part[(c * NP + p) * 4 + threadIdx.x];
      q[threadIdx.x] = t;
    }
    __syncthreads();
    const double n = q[0], u0 = q[1] / n, u1 = q[2] / n;
    const double T = (q[3] / n - u0 * u0 - u1 * u1) / 3.0;
    const InstDesc& d = inst[instance_of(inst, n_inst, c)];
    const double tau = relaxation_time<double>(d.tau_mode, d.kn, n, T);
    eq_factors(m, n, u0, u1, T, g0, g1, mv, red);
    real* o = rec + c * stride;
    for (int k = threadIdx.x; k < m.nq0 + m.nq1; k += blockDim.x) o[k] = real(k < m.nq0 ? g0[k] : g1[k - m.nq0]);
    if (threadIdx.x == 0) {
      o[m.nq0 + m.nq1] = real(T);
      o[m.nq0 + m.nq1 + 1] = real(1.0 / tau);
      if (!(n > 0.0) || !(T > 0.0)) atomicOr(m.err, ERR_NONFINITE);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- force kernel
// out[h][c][i][jd] = -inv_rbar_c p1_j^2 sum_{k in part h} K0[i][k] D[c][k][jd], jd = 2 j + d (the
// radial part of the inertial term, its k range split in KS parts that the update kernel adds in
// order; the azimuthal part, nq1 terms, is added there too).  CTA tile: TI rows x TJ columns of
// one cell and one k part, k in chunks of TK; 128 threads, each 2 rows x 5 columns.
constexpr int TI = 32, TJ = 40, TK = 32, FT = 128, KS = 4;
template <typename real>
__global__ void __launch_bounds__(FT) lm_force_kernel(const LargeModel m, const real* F, const GeoCell* geo, real* out) {
  __shared__ real Ks[TI][TK + 1];
  __shared__ real Ds[TK][TJ];
  const long long c = blockIdx.x;
  const int ncol = 2 * m.nq1, ntj = (ncol + TJ - 1) / TJ;
  const int i0 = blockIdx.y * TI, c0 = (blockIdx.z % ntj) * TJ, h = blockIdx.z / ntj;
  const int kchunks = (m.nq0 + TK - 1) / TK, per = (kchunks + KS - 1) / KS;
  const int kbeg = h * per * TK, kend = min(m.nq0, (h + 1) * per * TK);
  const real* D = F + c * 2 * m.Vp;  // [i][jd], row stride ncol
  constexpr bool F32 = sizeof(real) == 4;
  // single precision: the scaled matrix, inputs times 1/sqrt(w) of their node, output times sqrt(w)
  const real* K0 = F32 ? reinterpret_cast<const real*>(m.K0f) : reinterpret_cast<const real*>(m.K0);
  const int ti = threadIdx.x >> 3, tj = threadIdx.x & 7;  // rows ti, ti + 16; columns tj + 8 r
  real acc[2][5] = {};
  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    for (int x = threadIdx.x; x < TI * TK; x += FT) {
      const int r = x / TK, k = x - r * TK;
      Ks[r][k] = (i0 + r < m.nq0 && k0 + k < kend) ? K0[size_t(i0 + r) * m.nq0 + k0 + k] : real(0);
    }
    for (int x = threadIdx.x; x < TK * TJ; x += FT) {
      const int k = x / TJ, col = x - k * TJ;
      real dv = (k0 + k < kend && c0 + col < ncol) ? D[size_t(k0 + k) * ncol + c0 + col] : real(0);
      if constexpr (F32) dv *= (k0 + k < kend) ? real(m.is0f[k0 + k]) : real(0);
      Ds[k][col] = dv;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TK; ++k) {
      const real a0 = Ks[ti][k], a1 = Ks[ti + 16][k];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const real b = Ds[k][tj + 8 * r];
        acc[0][r] += a0 * b;
        acc[1][r] += a1 * b;
      }
    }
    __syncthreads();
  }
  const real irb = real(m.ftilde ? m.inv_r[c] : geo[c].inv_rbar);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = i0 + ti + 16 * q;
    if (i >= m.nq0) continue;
    const real si = F32 ? real(m.s0f[i]) : real(1);
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int col = c0 + tj + 8 * r;
      if (col >= ncol) continue;
      const real pj = real(m.p1[col >> 1]);
      out[(size_t(h) * gridDim.x + c) * 2 * m.Vp + size_t(i) * ncol + col] = -irb * pj * pj * (si * acc[q][r]);
    }
  }
}

// ---------------------------------------------------------------- update kernel
template <typename real>
__global__ void lm_update_kernel(const LargeModel m, const real* Fprev, const real* Fl, real* Fout, long long cells,
                                 const InstDesc* inst, int n_inst, const GeoCell* geo, const real* rec,
                                 const real* force, const double* walls, const double* wpart, int NP, double* nw,
                                 double ca, double cc) {
  using P = pair_t<real>;
  constexpr bool F32 = sizeof(real) == 4;
  const long long total = cells * m.V;
  const int stride = m.nq0 + m.nq1 + 2;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const long long c = x / m.V;
    const int v = int(x - c * m.V);
    const int i = v / m.nq1, j = v - i * m.nq1;
    const int ii = instance_of(inst, n_inst, c);
    const InstDesc& d = inst[ii];
    const int s = int(c - d.cell0), n = d.n_cells;
    const double Rd = m.w0[i] * m.w1[j];
    auto wall_density = [&](int wall) {  // n_w of Eq. (nw) from the chunk sums, in a fixed order
      double t = m.ftilde ? 0.0 : (wall == 0 ? m.ref_flux_neg : m.ref_flux_pos);  // f~: no R split
      for (int p = 0; p < NP; ++p) t += wpart[(size_t(ii) * 2 + wall) * NP + p];
      return -t / walls[(size_t(ii) * 2 + wall) * (m.nq0 + m.nq1 + 2) + m.nq0 + m.nq1];
    };
    // the advected value of a cell: D (chi), or F~ = sqrt(g) (D + R) (f~)
    auto cell = [&](long long cc) -> P {
      const P x = p_load(Fprev + cc * 2 * m.Vp + 2 * v);
      if (!m.ftilde) return x;
      return p_mul(p_add(x, p_set(real(Rd))), p_set(real(m.sqrtg[cc])));
    };
    auto ghost = [&](int wall, int dist) -> P {  // ghost at distance 1..3 past a wall (Eq. weno_populate)
      const double sgn = wall == 0 ? 1.0 : -1.0;
      if (sgn * m.p0[i] < 0.0) {  // outgoing: quadratic extrapolation (Eq. extrapol)
        const long long e0 = d.cell0 + (wall == 0 ? 0 : n - 1);
        const int dir = wall == 0 ? 1 : -1;
        const P F0 = cell(e0), F1 = cell(e0 + dir), F2 = cell(e0 + 2 * dir);
        if (dist == 1) return p_fma(F1, p_set(real(-3)), p_fma(F0, p_set(real(3)), F2));
        return p_fma(F1, p_set(real(-8)), p_fma(F0, p_set(real(6)), p_mul(F2, p_set(real(3)))));
      }
      const double* wt = walls + (size_t(ii) * 2 + wall) * (m.nq0 + m.nq1 + 2);
      const double e = wall_density(wall) * wt[i] * wt[m.nq0 + j];
      const double r = m.ftilde ? 0.0 : Rd;  // f~ ghosts are F~ itself
      return p_make(real(e - r), real(e * wt[m.nq0 + m.nq1 + 1] - r));
    };
    auto at = [&](int k) -> P {  // advected values of cell s + k, ghosts past the walls
      const int t = s + k;
      if (t < 0) return ghost(0, -t);
      if (t >= n) return ghost(1, t - n + 1);
      return cell(c + k);
    };
    if (v == 0 && (s == 0 || s == n - 1))  // the wall densities of the stage, for vlb_wall_density
      for (int wall = 0; wall < 2; ++wall)
        if ((wall == 0 && s == 0) || (wall == 1 && s == n - 1)) {
          const double nwv = wall_density(wall);
          nw[ii * 2 + wall] = nwv;
          if (!isfinite(nwv)) atomicOr(m.err, ERR_NONFINITE);
        }
    const P Fm3 = at(-3), Fm2 = at(-2), Fm1 = at(-1), S0 = at(0), Fp1 = at(1), Fp2 = at(2), Fp3 = at(3);
    const P F0 = p_load(Fprev + c * 2 * m.Vp + 2 * v);  // the cell's own D
    const real sc = weno_scale<real>(m.iw0[i] * m.iw1[j]);
    const real pr = real(m.p0[i]);
    P fm, fp;
    if (pr >= real(0)) {
      fm = weno5p<real>(Fm3, Fm2, Fm1, S0, Fp1, sc);
      fp = weno5p<real>(Fm2, Fm1, S0, Fp1, Fp2, sc);
    } else {
      fm = weno5p<real>(Fp2, Fp1, S0, Fm1, Fm2, sc);
      fp = weno5p<real>(Fp3, Fp2, Fp1, S0, Fm1, sc);
    }
    const GeoCell g = geo[c];
    // -adv = -p^R (cp F_{s+1/2} - cm F_{s-1/2}); f~: the factors e_{s+-1/2} / (d eta sqrt(g_s))
    const real cp = real(m.ftilde ? m.advp[c] : g.cp), cm = real(m.ftilde ? m.advm[c] : g.cm);
    const P nadv = p_mul(p_sub(p_mul(fp, p_set(cp)), p_mul(fm, p_set(cm))), p_set(-pr));
    // the azimuthal part of the inertial term, +inv_rbar p0_i sum_l Kt1[j][l] D[c][i][l]
    const real* Drow = Fprev + c * 2 * m.Vp + size_t(i) * 2 * m.nq1;
    P e = p_set(real(0));
    if constexpr (F32) {
      for (int l = 0; l < m.nq1; ++l) e = p_fma(p_set(real(m.Kt1f[j * m.nq1 + l]) * real(m.is1f[l])), p_load(Drow + 2 * l), e);
      e = p_mul(e, p_set(real(m.s1f[j])));
    } else {
      for (int l = 0; l < m.nq1; ++l) e = p_fma(p_set(real(m.Kt1[j * m.nq1 + l])), p_load(Drow + 2 * l), e);
    }
    P fr = p_load(force + c * 2 * m.Vp + 2 * v);
    for (int h = 1; h < KS; ++h) fr = p_add(fr, p_load(force + (size_t(h) * cells + c) * 2 * m.Vp + 2 * v));
    P frc = p_fma(e, p_set(real(m.ftilde ? m.inv_r[c] : g.inv_rbar) * pr), fr);
    if (m.ftilde) frc = p_add(frc, p_set(real(-m.inv_r[c] * m.forceR[v])));  // f~ advects R too
    const real* rc = rec + c * stride;
    const real geq = rc[i] * rc[m.nq0 + j];
    const real R = real(Rd);
    const P deq = p_make(geq - R, geq * rc[m.nq0 + m.nq1] - R);
    const real itau = rc[m.nq0 + m.nq1 + 1];
    const P Lv = p_fma(p_sub(F0, deq), p_set(-itau), p_add(nadv, frc));
    const real dt = F32 ? real(d.dt_f) : real(d.dt);
    P o = p_fma(Lv, p_set(real(cc) * dt), F0);
    if (ca != 0.0) o = p_fma(p_sub(p_load(Fl + c * 2 * m.Vp + 2 * v), F0), p_set(real(ca)), o);
    p_store(Fout + c * 2 * m.Vp + 2 * v, o);
  }
}

// ---------------------------------------------------------------- Cartesian-split channel (Sec. VII.G)
// Eq. (canalie_coord_beq_cons): no force term; the lambda flux upwinds by the sign of
// V^lambda = (p^x - lambda phi' p^y) / (1 + phi), a combination of both momenta that changes
// along the wall, so the wall's incoming half-plane is per column (Eq. canalie_coord_nw).
// The fluxes are taken of F = D + R: without a force term the rest state's advection does not
// cancel discretely, so R is kept.

// per cell: moments, tau = Kn / (n T), the equilibrium record; the end columns also the
// reservoir factors of f_eq(1, (0, u^y), T0) (u^y of that cell)
template <typename real>
__global__ void __launch_bounds__(kCellThreads) clb_cell_kernel(const LargeModel m, const ClbGeom g, const real* F,
                                                                real* rec, real* res) {
  extern __shared__ double sh[];
  double* g0 = sh;
  double* g1 = g0 + m.nq0;
  double* mv = g1 + m.nq1;
  double* red = mv + 4 * MAXN;
  const int stride = m.nq0 + m.nq1 + 2;
  const long long cells = (long long)g.nl * g.nx;
  for (long long c = blockIdx.x; c < cells; c += gridDim.x) {
    const real* f = F + c * 2 * m.Vp;
    double sn = 0, s0 = 0, s1 = 0, se = 0;
    for (int v = threadIdx.x; v < m.V; v += blockDim.x) {
      const int i = v / m.nq1, j = v - i * m.nq1;
      const double r = m.w0[i] * m.w1[j];
      const double f1 = double(f[2 * v]) + r, f2 = double(f[2 * v + 1]) + r;
      const double a = m.p0[i], b = m.p1[j];
      sn += f1;
      s0 += a * f1;
      s1 += b * f1;
      se += (a * a + b * b) * f1 + f2;
    }
    const double n = block_sum(sn, red), u0 = block_sum(s0, red) / n, u1 = block_sum(s1, red) / n;
    const double T = (block_sum(se, red) / n - u0 * u0 - u1 * u1) / 3.0;
    eq_factors(m, n, u0, u1, T, g0, g1, mv, red);
    real* o = rec + c * stride;
    for (int k = threadIdx.x; k < m.nq0 + m.nq1; k += blockDim.x) o[k] = real(k < m.nq0 ? g0[k] : g1[k - m.nq0]);
    if (threadIdx.x == 0) {
      o[m.nq0 + m.nq1] = real(T);
      o[m.nq0 + m.nq1 + 1] = real(n * T / g.kn);
      if (!(n > 0.0) || !(T > 0.0)) atomicOr(m.err, ERR_NONFINITE);
    }
    __syncthreads();
    const int s_ = int(c / g.nx), p = int(c - (long long)s_ * g.nx);
    for (int end = 0; end < 2; ++end) {  // uniform across the block
      if (p != (end == 0 ? 0 : g.nx - 1)) continue;
      eq_factors(m, 1.0, 0.0, u1, g.T0, g0, g1, mv, red);
      real* q = res + (size_t(s_) * 2 + end) * (m.nq0 + m.nq1);
      for (int k = threadIdx.x; k < m.nq0 + m.nq1; k += blockDim.x) q[k] = real(k < m.nq0 ? g0[k] : g1[k - m.nq0]);
      __syncthreads();
    }
  }
}

// per column: n_w of Eq. (canalie_coord_nw) from the leaving half (V^lambda > 0 at the wall)
template <typename real>
__global__ void __launch_bounds__(256) clb_wall_kernel(const LargeModel m, const ClbGeom g, const real* F, double* nw) {
  __shared__ double red[33];
  using P = pair_t<real>;
  const int p = blockIdx.x, nl = g.nl, nx = g.nx;
  const real* FN = F + ((long long)(nl - 1) * nx + p) * 2 * m.Vp;
  const real* FN1 = F + ((long long)(nl - 2) * nx + p) * 2 * m.Vp;
  const real* FN2 = F + ((long long)(nl - 3) * nx + p) * 2 * m.Vp;
  const double lw = g.lf[nl];
  double num = 0.0, den = 0.0;
  for (int v = threadIdx.x; v < m.V; v += blockDim.x) {
    const int i = v / m.nq1, j = v - i * m.nq1;
    const double V = g.va[p] * (m.p0[i] - lw * g.dph[p] * m.p1[j]);
    if (V > 0.0) {
      const P a = p_load(FN2 + 2 * v), b = p_load(FN1 + 2 * v), c0 = p_load(FN + 2 * v);
      const P e1 = p_fma(b, p_set(real(-3)), p_fma(c0, p_set(real(3)), a));
      const P e2 = p_fma(b, p_set(real(-8)), p_fma(c0, p_set(real(6)), p_mul(a, p_set(real(3)))));
      const double fx = double(weno5p<real>(a, b, c0, e1, e2, weno_scale<real>(m.iw0[i] * m.iw1[j])).x);
      num += (fx + m.w0[i] * m.w1[j]) * V;  // the flux of F = D + R
    } else {
      den += g.weq[i] * g.weq[m.nq0 + j] * V;
    }
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) {
    const double nwv = -num / den;
    nw[p] = nwv;
    if (!isfinite(nwv)) atomicOr(m.err, ERR_NONFINITE);
  }
}

template <typename real>
__global__ void clb_update_kernel(const LargeModel m, const ClbGeom g, const real* Fprev, const real* Fl, real* Fout,
                                  const real* rec, const real* res, const double* nw, double dt, double ca, double cc) {
  using P = pair_t<real>;
  const int nl = g.nl, nx = g.nx;
  const long long total = (long long)nl * nx * m.V;
  const int stride = m.nq0 + m.nq1 + 2;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const long long c = x / m.V;
    const int v = int(x - c * m.V);
    const int i = v / m.nq1, j = v - i * m.nq1;
    const int s = int(c / nx), p = int(c - (long long)s * nx);
    const double Rd = m.w0[i] * m.w1[j];
    const real R = real(Rd);
    auto D = [&](int r, int q, int vv) -> P { return p_load(Fprev + ((long long)r * nx + q) * 2 * m.Vp + 2 * vv); };
    // lambda column p: rows below 0 mirror p^x (specular centreline), rows past nl are wall ghosts
    const double Vw = g.va[p] * (m.p0[i] - g.lf[nl] * g.dph[p] * m.p1[j]);
    auto lam = [&](int r) -> P {
      if (r >= 0 && r < nl) return D(r, p, v);
      if (r < 0) return D(-r - 1, p, g.ibar[i] * m.nq1 + j);
      const int dist = r - nl + 1;
      if (Vw > 0.0) {  // leaving through the wall: quadratic extrapolation (Eq. extrapol)
        const P a = D(nl - 3, p, v), b = D(nl - 2, p, v), c0 = D(nl - 1, p, v);
        if (dist == 1) return p_fma(b, p_set(real(-3)), p_fma(c0, p_set(real(3)), a));
        return p_fma(b, p_set(real(-8)), p_fma(c0, p_set(real(6)), p_mul(a, p_set(real(3)))));
      }
      const double e = nw[p] * g.weq[i] * g.weq[m.nq0 + j];
      return p_make(real(e - Rd), real(e * g.T0 - Rd));
    };
    // xi row s: columns past the ends are the reservoirs for the entering populations
    auto xi = [&](int q) -> P {
      if (q >= 0 && q < nx) return D(s, q, v);
      const int end = q < 0 ? 0 : 1;
      const bool entering = end == 0 ? (m.p1[j] > 0.0) : (m.p1[j] < 0.0);
      if (!entering) return D(s, end == 0 ? 0 : nx - 1, v);
      const real* rr = res + (size_t(s) * 2 + end) * (m.nq0 + m.nq1);
      const double e = (end == 0 ? g.n_in : g.n_out) * double(rr[i]) * double(rr[m.nq0 + j]);
      return p_make(real(e - Rd), real(e * g.T0 - Rd));
    };
    const real sc = weno_scale<real>(m.iw0[i] * m.iw1[j]);
    const P L3 = lam(s - 3), L2 = lam(s - 2), L1 = lam(s - 1), C0 = lam(s), U1 = lam(s + 1), U2 = lam(s + 2), U3 = lam(s + 3);
    const double Vm = g.va[p] * (m.p0[i] - g.lf[s] * g.dph[p] * m.p1[j]);
    const double Vp = g.va[p] * (m.p0[i] - g.lf[s + 1] * g.dph[p] * m.p1[j]);
    const P fm = Vm >= 0.0 ? weno5p<real>(L3, L2, L1, C0, U1, sc) : weno5p<real>(U2, U1, C0, L1, L2, sc);
    const P fp = Vp >= 0.0 ? weno5p<real>(L2, L1, C0, U1, U2, sc) : weno5p<real>(U3, U2, U1, C0, L1, sc);
    const P X3 = xi(p - 3), X2 = xi(p - 2), X1 = xi(p - 1), X4 = xi(p + 1), X5 = xi(p + 2), X6 = xi(p + 3);
    const bool up = m.p1[j] >= 0.0;
    const P xm = up ? weno5p<real>(X3, X2, X1, C0, X4, sc) : weno5p<real>(X5, X4, C0, X1, X2, sc);
    const P xp = up ? weno5p<real>(X2, X1, C0, X4, X5, sc) : weno5p<real>(X6, X5, X4, C0, X1, sc);
    const P Rp = p_set(R);
    // -[V F]_{s-1/2}^{s+1/2} / d lambda - [V F]_{p-1/2}^{p+1/2} / d chi, F = D + R
    P nadv = p_mul(p_sub(p_mul(p_add(fp, Rp), p_set(real(Vp))), p_mul(p_add(fm, Rp), p_set(real(Vm)))),
                   p_set(real(-g.idl[s])));
    const real vxm = real(g.vx[p] * m.p1[j]), vxp = real(g.vx[p + 1] * m.p1[j]);
    nadv = p_fma(p_sub(p_mul(p_add(xp, Rp), p_set(vxp)), p_mul(p_add(xm, Rp), p_set(vxm))), p_set(real(-g.idx[p])), nadv);
    const real* rc = rec + c * stride;
    const real geq = rc[i] * rc[m.nq0 + j];
    const P deq = p_make(geq - R, geq * rc[m.nq0 + m.nq1] - R);
    const P Lv = p_fma(p_sub(C0, deq), p_set(-rc[m.nq0 + m.nq1 + 1]), nadv);
    P o = p_fma(Lv, p_set(real(cc * dt)), C0);
    if (ca != 0.0) o = p_fma(p_sub(p_load(Fl + c * 2 * m.Vp + 2 * v), C0), p_set(real(ca)), o);
    p_store(Fout + c * 2 * m.Vp + 2 * v, o);
  }
}

// ---------------------------------------------------------------- layout, initial state, moments
template <typename real>
__global__ void lm_deviation_kernel(const LargeModel m, const real* src, real* dst, long long cells, int to_dev) {
  const long long total = cells * 2 * m.Vp;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const long long c = x / (2 * m.Vp);
    const int e = int(x - c * 2 * m.Vp), v = e >> 1, f = e & 1;
    if (v >= m.V) {
      if (to_dev) dst[x] = real(0);
      continue;
    }
    const int i = v / m.nq1, j = v - i * m.nq1;
    const double r = m.w0[i] * m.w1[j];
    if (to_dev) dst[x] = real(double(src[c * 2 * m.V + f * m.V + v]) - r);
    else dst[c * 2 * m.V + f * m.V + v] = real(double(src[x]) + r);
  }
}

template <typename real>
__global__ void __launch_bounds__(kCellThreads) lm_init_kernel(const LargeModel m, real* F, long long cells, double n,
                                                               double u0, double u1, double T) {
  extern __shared__ double sh[];
  double* g0 = sh;
  double* g1 = g0 + m.nq0;
  double* mv = g1 + m.nq1;
  double* red = mv + 4 * MAXN;
  eq_factors(m, n, u0, u1, T, g0, g1, mv, red);
  for (long long c = blockIdx.x; c < cells; c += gridDim.x)
    for (int v = threadIdx.x; v < m.Vp; v += blockDim.x) {
      real a = real(0), b = real(0);
      if (v < m.V) {
        const int i = v / m.nq1, j = v - i * m.nq1;
        const double g = g0[i] * g1[j], r = m.w0[i] * m.w1[j];
        a = real(g - r);
        b = real(T * g - r);
      }
      F[c * 2 * m.Vp + 2 * v] = a;
      F[c * 2 * m.Vp + 2 * v + 1] = b;
    }
}

template <typename real>
__global__ void __launch_bounds__(kCellThreads) lm_moments_kernel(const LargeModel m, const real* F, long long cells,
                                                                  double* out) {
  __shared__ double red[33];
  for (long long c = blockIdx.x; c < cells; c += gridDim.x) {
    const real* f = F + c * 2 * m.Vp;
    double sn = 0, s0 = 0, s1 = 0;
    for (int v = threadIdx.x; v < m.V; v += blockDim.x) {
      const int i = v / m.nq1, j = v - i * m.nq1;
      const double f1 = double(f[2 * v]) + m.w0[i] * m.w1[j];
      sn += f1;
      s0 += m.p0[i] * f1;
      s1 += m.p1[j] * f1;
    }
    const double n = block_sum(sn, red), u0 = block_sum(s0, red) / n, u1 = block_sum(s1, red) / n;
    double t00 = 0, t01 = 0, t11 = 0, tr2 = 0, q0 = 0, q1 = 0;
    for (int v = threadIdx.x; v < m.V; v += blockDim.x) {
      const int i = v / m.nq1, j = v - i * m.nq1;
      const double r = m.w0[i] * m.w1[j];
      const double f1 = double(f[2 * v]) + r, f2 = double(f[2 * v + 1]) + r;
      const double x0 = m.p0[i] - u0, x1 = m.p1[j] - u1;
      t00 += x0 * x0 * f1;
      t01 += x0 * x1 * f1;
      t11 += x1 * x1 * f1;
      tr2 += f2;
      const double e = 0.5 * (x0 * x0 + x1 * x1) * f1 + 0.5 * f2;
      q0 += e * x0;
      q1 += e * x1;
    }
    t00 = block_sum(t00, red);
    t01 = block_sum(t01, red);
    t11 = block_sum(t11, red);
    tr2 = block_sum(tr2, red);
    q0 = block_sum(q0, red);
    q1 = block_sum(q1, red);
    if (threadIdx.x == 0) {
      double* o = out + c * 9;
      o[0] = n;
      o[1] = u0;
      o[2] = u1;
      o[3] = (t00 + t11 + tr2) / (3.0 * n);
      o[4] = t00;
      o[5] = t01;
      o[6] = t11;
      o[7] = q0;
      o[8] = q1;
    }
    __syncthreads();
  }
}

size_t cell_smem(const LargeModel& m) { return sizeof(double) * (m.nq0 + m.nq1 + 4 * MAXN + 33 + 4); }
int grid_for(long long work, int threads) {
  const long long b = (work + threads - 1) / threads;
  return int(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

int chunks(const LargeModel& m) { return (m.V + kChunk - 1) / kChunk; }

template <typename real>
cudaError_t lm_stage(const LargeModel& m, const real* Fprev, const real* Fl, real* Fout, long long cells,
                     const InstDesc* inst, int n_inst, const GeoCell* geo, const double* walls, double* nw,
                     real* rec, real* force, double* part, double ca, double cc, cudaStream_t s) {
  const int NP = chunks(m);
  double* wpart = part + cells * NP * 4;
  lm_partial_kernel<real><<<dim3(unsigned(cells), unsigned(NP)), 256, 0, s>>>(m, Fprev, part);
  lm_wallpart_kernel<real><<<dim3(unsigned(n_inst), 2, unsigned(NP)), 256, 0, s>>>(m, Fprev, inst, wpart);
  const int cgrid = int(cells < 152 * 8 ? cells : 152 * 8);
  lm_cell_kernel<real><<<cgrid, kCellThreads, cell_smem(m), s>>>(m, cells, NP, part, inst, n_inst, rec);
  const dim3 fg(unsigned(cells), unsigned((m.nq0 + TI - 1) / TI), unsigned((2 * m.nq1 + TJ - 1) / TJ) * KS);
  lm_force_kernel<real><<<fg, FT, 0, s>>>(m, Fprev, geo, force);
  lm_update_kernel<real><<<grid_for(cells * m.V, 256), 256, 0, s>>>(m, Fprev, Fl, Fout, cells, inst, n_inst, geo,
                                                                   rec, force, walls, wpart, NP, nw, ca, cc);
  return cudaGetLastError();
}

template <typename real>
cudaError_t clb_stage(const LargeModel& m, const ClbGeom& g, const real* Fprev, const real* Fl, real* Fout, real* rec,
                      real* res, double* nw, double dt, double ca, double cc, cudaStream_t s) {
  const long long cells = (long long)g.nl * g.nx;
  const int cg = int(cells < 152 * 8 ? cells : 152 * 8);
  clb_cell_kernel<real><<<cg, kCellThreads, cell_smem(m), s>>>(m, g, Fprev, rec, res);
  clb_wall_kernel<real><<<g.nx, 256, 0, s>>>(m, g, Fprev, nw);
  clb_update_kernel<real><<<grid_for(cells * m.V, 256), 256, 0, s>>>(m, g, Fprev, Fl, Fout, rec, res, nw, dt, ca, cc);
  return cudaGetLastError();
}

size_t lm_force_reals(const LargeModel& m, long long cells) { return size_t(KS) * cells * 2 * m.Vp; }

size_t lm_part_doubles(const LargeModel& m, long long cells, int n_inst) {
  return size_t(cells) * chunks(m) * 4 + size_t(n_inst) * 2 * chunks(m);
}

template <typename real>
cudaError_t lm_deviation(const LargeModel& m, const real* src, real* dst, long long cells, int to_dev, cudaStream_t s) {
  lm_deviation_kernel<real><<<grid_for(cells * 2 * m.Vp, 256), 256, 0, s>>>(m, src, dst, cells, to_dev);
  return cudaGetLastError();
}

template <typename real>
cudaError_t lm_init(const LargeModel& m, real* F, long long cells, double n, double u0, double u1, double T,
                    cudaStream_t s) {
  const int g = int(cells < 152 * 2 ? cells : 152 * 2);
  lm_init_kernel<real><<<g, kCellThreads, cell_smem(m), s>>>(m, F, cells, n, u0, u1, T);
  return cudaGetLastError();
}

template <typename real>
cudaError_t lm_moments(const LargeModel& m, const real* F, long long cells, double* out, cudaStream_t s) {
  const int g = int(cells < 152 * 2 ? cells : 152 * 2);
  lm_moments_kernel<real><<<g, kCellThreads, 0, s>>>(m, F, cells, out);
  return cudaGetLastError();
}

#define VLB_LM_INST(real)                                                                                          \
  template cudaError_t lm_stage<real>(const LargeModel&, const real*, const real*, real*, long long,               \
                                      const InstDesc*, int, const GeoCell*, const double*, double*, real*, real*,    \
                                      double*, double, double, cudaStream_t);                                        \
  template cudaError_t lm_deviation<real>(const LargeModel&, const real*, real*, long long, int, cudaStream_t);    \
  template cudaError_t clb_stage<real>(const LargeModel&, const ClbGeom&, const real*, const real*, real*, real*,  \
                                       real*, double*, double, double, double, cudaStream_t);                        \
  template cudaError_t lm_init<real>(const LargeModel&, real*, long long, double, double, double, double,          \
                                     cudaStream_t);                                                                  \
  template cudaError_t lm_moments<real>(const LargeModel&, const real*, long long, double*, cudaStream_t);
VLB_LM_INST(float)
VLB_LM_INST(double)

}  // namespace vlb
