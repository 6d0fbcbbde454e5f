// One TVD-RK3 stage of the chi-formulation circular Couette update, fused into
// one kernel per tile of up to TC cells of one instance (all momenta of those cells):
//
//   bulk-copy the tile, its three-cell halo and its cells' geometry to shared memory
//   -> moments per cell (Eq. macro_red), truncated equilibrium and tau; meanwhile,
//      on the warps without a cell, the inertial force
//      (1/R)[(p^phi)^2 K^R f - p^R K~^phi f] (Eq. boltz_couette_kom)
//   -> walls: extrapolated outgoing ghosts (Eq. extrapol), wall flux, n_w
//      (Eq. nw), incoming ghosts f_eq(n_w, u_w, T_w) (Eq. weno_populate)
//   -> WENO-5 fluxes along the cells, chi flux difference, BGK, RK3 combine
//      (Eqs. weno5_flux, flux_kom_R / flux_kom_eta, BGK, rk3) -> global.
//
// Every distribution buffer holds the deviation D = F - R from the rest state
// (ModelArgs): the operator is linear in R's part, which it leaves unchanged.
// A cell row holds Vp velocity pairs (f', f'') interleaved (see pair_t).
#pragma once
#include <type_traits>

#include "vlb_device.cuh"

namespace vlb {

template <typename real>
struct StageArgs {
  const real* Fprev;  // distribution L acts on
  const real* Fl;     // F_l of the step (read when ca != 0)
  real* Fout;
  // Fout = ca F_l + cb F_prev + cc dt L[F_prev] with cb = 1 - ca, evaluated as
  // F_prev + ca (F_l - F_prev) + cc dt L so that the weights on F sum to exactly
  // one in any precision (float(1/3) + float(2/3) = 1 + 3e-8 would add that much
  // mass every step).
  double ca, cb, cc;
  float caf, cbf, ccf;  // single-precision copies
  const InstDesc* inst;
  const TileDesc* tiles;
  int n_tiles;
  const GeoCell* geo;    // per global cell
  const GeoCellF* geof;  // single-precision copy
  double* nw;          // 2 per instance: inner, outer wall density
  const WallEq* wall;  // 2 per instance: inner, outer wall equilibrium
  const real* halo;    // 2 x 3 rows per instance: ghost cells of slab halo ends (InstDesc::halo)
  // the f~ formulation (the FT kernels): sqrt(g) per global cell and the inertial term of R per
  // velocity; geo / geof then hold e_{s+-1/2} / (d eta sqrt(g)) as cp / cm and 1 / R_s as inv_rbar
  const real* sqrtg;
  const real* forceR;
  unsigned* err;
  int Vp;              // velocities per cell row, padded (>= nq0 nq1, multiple of 4); a row holds 2 Vp reals
  int nbuf;            // tile buffers: 1, or 2 when a persistent CTA stages its next tile during this one
  unsigned long long max_polls;
};

// Shared-memory carve-up, identical on host and device: two mbarriers, nbuf tile
// buffers (the TC + 6 rows of a tile with its halo, then the geometry of its TC
// cells), the force buffer (TC rows), then doubles and reals.
template <typename real, int TC, int NT>
struct StageSmem {
  static constexpr int NW = NT / 32;
  using Geo = typename std::conditional<sizeof(real) == 4, GeoCellF, GeoCell>::type;
  __host__ __device__ static size_t tile_off() { return 16; }
  __host__ __device__ static size_t geo_off(int Vp) { return size_t(TC + 6) * 2 * Vp * sizeof(real); }
  __host__ __device__ static size_t buf_bytes(int Vp) { return geo_off(Vp) + size_t(TC) * sizeof(Geo); }
  __host__ __device__ static size_t lbuf_off(int Vp, int nbuf) { return tile_off() + size_t(nbuf) * buf_bytes(Vp); }
  __host__ __device__ static size_t dbl_off(int Vp, int nbuf) {
    size_t o = lbuf_off(Vp, nbuf) + size_t(TC) * 2 * Vp * sizeof(real);
    return (o + 15) & ~size_t(15);
  }
  // doubles: p0, p1 (MAXQ each), reduction (NW*4), wall equilibrium factors (2*MAXQ), scalars (16)
  static constexpr size_t n_dbl = 2 * MAXQ + NW * 4 + 2 * MAXQ + 16;
  __host__ __device__ static size_t real_off(int Vp, int nbuf) { return dbl_off(Vp, nbuf) + n_dbl * sizeof(double); }
  // reals: p0, p1, 1/w0, 1/w1 (MAXQ each), tab0, tab1 (MAXQ*MAXN each), then pairs: n g_R and g_phi
  // (TC*MAXQ each), (1, T), -1/tau, cp, -cm, 1/Rbar (TC each); then moment vectors (TC*4*MAXN),
  // w0, w1 (MAXQ each)
  static constexpr size_t n_real = 4 * MAXQ + 2 * MAXQ * MAXN + 4 * TC * MAXQ + 10 * TC + TC * 4 * MAXN + 2 * MAXQ;
  __host__ __device__ static size_t bytes(int Vp, int nbuf) { return real_off(Vp, nbuf) + n_real * sizeof(real); }
};

// CTAs per SM the register allocation is sized for, where shared memory would
// allow them but the compiler, left alone, takes too many registers a thread.  A
// single-precision CTA of 256 to 384 threads needs at most about 64 KB of shared
// memory for tiles up to 8 cells (three fit on an SM) and about 100 KB for 16
// (two fit) with the model shapes that have fixed node counts.
constexpr int stage_min_ctas(int real_bytes, int tc, int nt) {
  return (real_bytes == 4 && nt >= 256 && nt <= 384) ? (tc <= 8 ? 3 : 2) : 1;
}

// FT: the f~ formulation (Sec. VI.B, Eqs. boltz_couette_cons / boltz_couette_str_cons).  The
// stencils act on F~ = sqrt(g) (D + R), held during phase D as F~ - R so that the walls' ghost
// rows (stored the same way) need no sqrt(g); the walls extrapolate F~; the flux difference
// takes e / (d eta sqrt(g)) and the force 1 / R_s, with the rest state's own advection and
// inertial term added (F~ is not a deviation).  The moments, equilibrium and BGK act on D.
template <typename real, int TC, int Q0MAX, int Q1MAX, int NT, bool EXACT, bool FT = false>
__global__ void __launch_bounds__(NT, stage_min_ctas(int(sizeof(real)), TC, NT))
    couette_stage_kernel(const __grid_constant__ StageArgs<real> a, const __grid_constant__ ModelArgs m,
                         const __grid_constant__ KArgs<real> kk) {
  using L = StageSmem<real, TC, NT>;
  constexpr int NW = L::NW;
  constexpr int VPC = (Q0MAX * Q1MAX + 3) / 4 * 4;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // exact instantiations fix node counts and strides at compile time; the generic one reads them
  const int nq0 = EXACT ? Q0MAX : m.nq0;
  const int nq1 = EXACT ? Q1MAX : m.nq1;
  const int V = nq0 * nq1;
  const int Vp = EXACT ? VPC : a.Vp;
  const int row = 2 * Vp;

  const int nbuf = a.nbuf;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);  // one mbarrier per tile buffer
  real* tile0 = reinterpret_cast<real*>(smem + L::tile_off());
  const size_t bstride = L::buf_bytes(Vp) / sizeof(real);  // reals per tile buffer
  real* lbuf = reinterpret_cast<real*>(smem + L::lbuf_off(Vp, nbuf));
  double* p0d = reinterpret_cast<double*>(smem + L::dbl_off(Vp, nbuf));
  double* p1d = p0d + MAXQ;
  double* red = p1d + MAXQ;
  double* gw0 = red + NW * 4;  // wall equilibrium factors
  double* gw1 = gw0 + MAXQ;
  double* mw = gw1 + MAXQ;     // [0] incoming equilibrium flux, [1] n_w
  real* p0r = reinterpret_cast<real*>(smem + L::real_off(Vp, nbuf));
  real* p1r = p0r + MAXQ;
  real* iw0 = p1r + MAXQ;  // 1 / w_i
  real* iw1 = iw0 + MAXQ;  // 1 / w_j
  real* tabr0 = iw1 + MAXQ;  // equilibrium tables in the bulk type
  real* tabr1 = tabr0 + MAXQ * MAXN;
  // per-cell values of phase D as ready pairs (both lanes of a packed operand)
  using P2 = pair_t<real>;
  P2* gRn = reinterpret_cast<P2*>(tabr1 + MAXQ * MAXN);  // [t][i] n_t g_{R,i} twice
  P2* gP = gRn + TC * MAXQ;                              // [t][j] g_{phi,j} twice
  P2* cT1 = gP + TC * MAXQ;                              // (1, T)
  P2* cNtau = cT1 + TC;                                  // -1/tau twice
  P2* ccp = cNtau + TC;                                  // cp twice
  P2* cNcm = ccp + TC;                                   // -cm twice
  P2* cIR = cNcm + TC;                                   // 1/Rbar twice
  real* mv = reinterpret_cast<real*>(cIR + TC);          // [t][axis*2 + side][s]
  real* w0r = mv + TC * 4 * MAXN;  // weights: R_ij = w0_i w1_j in the bulk type
  real* w1r = w0r + MAXQ;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr bool F32 = sizeof(real) == 4;
  for (int x = tid; x < MAXQ; x += NT) {
    p0d[x] = m.p0[x];
    p1d[x] = m.p1[x];
    if constexpr (F32) {
      p0r[x] = m.p0f[x];
      p1r[x] = m.p1f[x];
      iw0[x] = m.iw0f[x];
      iw1[x] = m.iw1f[x];
      w0r[x] = m.w0f[x];
      w1r[x] = m.w1f[x];
    } else {
      p0r[x] = m.p0[x];
      p1r[x] = m.p1[x];
      iw0[x] = m.iw0[x];
      iw1[x] = m.iw1[x];
      w0r[x] = m.w0[x];
      w1r[x] = m.w1[x];
    }
  }
  for (int x = tid; x < MAXQ * MAXN; x += NT) {
    tabr0[x] = sizeof(real) == 4 ? real(m.tab0f[x]) : real(m.tab0[x]);
    tabr1[x] = sizeof(real) == 4 ? real(m.tab1f[x]) : real(m.tab1[x]);
  }
  __syncthreads();
  const bool need_fl = a.caf != 0.0f;
  using Geo = typename L::Geo;
  const Geo* geo_src =
      reinterpret_cast<const Geo*>(F32 ? static_cast<const void*>(a.geof) : static_cast<const void*>(a.geo));
  // warp 0 stages tile tx (cells lo..hi-1 at slots lo-c0+3 ..., then its cells' geometry) into
  // buffer b with bulk copies that complete on the buffer's mbarrier
  auto stage_tile = [&](const TileDesc& t, int b) {
    const InstDesc i = a.inst[t.inst];
    const int lo = max(t.c0 - 3, 0), hi = min(t.c0 + t.nc + 3, i.n_cells);
    real* dst = tile0 + b * bstride;
    const unsigned rbytes = unsigned(row * sizeof(real)), gbytes = unsigned(t.nc * sizeof(Geo));
    if (lane == 0) mbar_expect_tx(bar + b, rbytes * unsigned(hi - lo) + gbytes);
    __syncwarp();
    for (int c = lo + lane; c < hi; c += 32)
      bulk_g2s(dst + (c - t.c0 + 3) * row, a.Fprev + size_t(i.cell0 + c) * row, rbytes, bar + b);
    if (lane == 0) bulk_g2s(dst + L::geo_off(Vp) / sizeof(real), geo_src + i.cell0 + t.c0, gbytes, bar + b);
  };
  unsigned phase = 0;  // bit b: parity of buffer b's next completion
  // the next tile's descriptor is read during the current tile (its load latency hidden)
  TileDesc td_next = blockIdx.x < a.n_tiles ? a.tiles[blockIdx.x] : TileDesc{0, 0, 0};
  if (nbuf == 2 && warp == 0 && blockIdx.x < a.n_tiles) stage_tile(td_next, 0);
  // one tile per iteration: a launch with one CTA per tile runs the body once, a persistent
  // launch (grid sized by occupancy) walks the tile list, with two buffers staging the next
  // tile while this one is computed
  for (int tix = blockIdx.x, it = 0; tix < a.n_tiles; tix += gridDim.x, ++it) {
  const int b = nbuf == 2 ? (it & 1) : 0;
  real* tile = tile0 + b * bstride;
  const TileDesc td = td_next;
  const InstDesc in = a.inst[td.inst];
  const int n = in.n_cells, c0 = td.c0;
  const int TCe = td.nc;  // the host sizes tiles (1 <= nc <= TC) to fill the launch in whole rounds
  if (nbuf == 1 && warp == 0) stage_tile(td, 0);
  bool ok = mbar_wait(bar + b, (phase >> b) & 1u, a.max_polls);
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
    mbar_wait(bar + b, (phase >> b) & 1u, a.max_polls);  // let the copies land before the CTA exits
    if (tid == 0) bulk_wait_all();                        // and the stores read their source
    return;
  }
  phase ^= 1u << b;
  {  // the cells' geometry as pairs for phase D
    const Geo* g = reinterpret_cast<const Geo*>(tile + L::geo_off(Vp) / sizeof(real));
    for (int t = tid; t < TCe; t += NT) {
      ccp[t] = p_set(real(g[t].cp));
      cNcm[t] = p_set(real(-g[t].cm));
      cIR[t] = p_set(real(g[t].inv_rbar));
    }
  }

  // ==== phase A: per cell, one half-warp (16 lanes) with no CTA barrier: moments (Eq.
  // macro_red), tau, the equilibrium moment vectors and factors (Sec. IV.D) and their mass
  // normalisation.  A warp takes two cells, so each shuffle level and each per-cell scalar
  // step serves both; warps without a cell go on to the force contractions below.
  const int NA = (TCe + 1) >> 1;  // warps with cells
  for (int wa = warp; wa < NA; wa += NW) {
    const int hl = lane & 15;
    const int tc = 2 * wa + (lane >> 4);
    const bool has = tc < TCe;         // the upper half of the last warp of an odd tile has no cell:
    const int t = has ? tc : TCe - 1;  // it repeats the lower half's and writes nothing
    const real* F = tile + (t + 3) * row;
    real sn = 0, sr = 0, sp = 0, se = 0;  // per-lane partial sums over a sixteenth of the velocities
#pragma unroll 4
    for (int v = hl; v < V; v += 16) {
      const int i = v / nq1, j = v - i * nq1;
      const pair_t<real> f = p_load(F + 2 * v);
      const real f1 = f.x, f2 = f.y, pr = p0r[i], pp = p1r[j];
      sn += f1;
      sr += pr * f1;
      sp += pp * f1;
      se += (pr * pr + pp * pp) * f1 + f2;
    }
    // sums over the half-warp; then the sums of D plus those of R and the derived fields
    real nn, u0, u1, T;
    double dn = 0.0;  // FP64 path: sum of D (n - sum R)
    float en = 0.f;   // FP32 path: rounding error of the mass sum sn (float-float sn + en)
    if constexpr (F32) {
      // compensated FP32 butterflies leave the same sums on every lane of the half; n in
      // float-float, the other fields in FP32 through one reciprocal: no FP64 and no
      // broadcast on the dependency chain
      float er = 0.f, ep = 0.f, ee = 0.f;
      half_sum_comp(sn, en);
      half_sum_comp(sr, er);
      half_sum_comp(sp, ep);
      half_sum_comp(se, ee);
      float nh, nl;
      two_sum(sn, m.ref_nf[0], nh, nl);
      nn = nh + (nl + (en + m.ref_nf[1]));
      const float inv = 1.0f / nn;
      u0 = (sr + (er + m.ref_rf)) * inv;
      u1 = (sp + (ep + m.ref_pf)) * inv;
      T = ((se + (ee + m.ref_ef)) * inv - (u0 * u0 + u1 * u1)) * (1.0f / 3.0f);
    } else {
      dn = half_sum(double(sn));
      const double dr = half_sum(double(sr)), dpp = half_sum(double(sp)), de = half_sum(double(se));
      nn = real(dn + m.ref_n), u0 = real(dr + m.ref_r) / nn, u1 = real(dpp + m.ref_p) / nn;
      T = (real(de + m.ref_e) - nn * (u0 * u0 + u1 * u1)) / (real(3) * nn);
    }
    if (hl == 0 && has) {
      cT1[t] = p_make(real(1), T);
      cNtau[t] = p_set(-(real(1) / relaxation_time<real>(in.tau_mode, F32 ? real(in.kn_f) : real(in.kn), nn, T)));
    }
    real* mt = mv + t * 4 * MAXN;  // moment vectors [axis * 2 + side][s]
    if (hl < 4 && has) {
      const int ax = hl >> 1, side = hl & 1;
      const real u = (ax ? u1 : u0) * (side ? real(-1) : real(1));
      eq_moment_vector<real>(ax ? m.kind1 : m.kind0, ax ? m.N1 : m.N0, u, T, mt + hl * MAXN);
    }
    __syncwarp();
    // equilibrium factors: lane hl takes g_R[k] and g_phi[k] for k = hl and hl + 16
    real gr[2] = {real(0), real(0)}, gp[2] = {real(0), real(0)};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = hl + 16 * q;
      if (16 * q < Q0MAX && k < nq0) {
        const real* mm = mt + ((m.kind0 == 1 && p0r[k] < real(0)) ? 1 : 0) * MAXN;
        for (int s2 = 0; s2 <= m.N0; ++s2) gr[q] += tabr0[k * MAXN + s2] * mm[s2];
        gr[q] *= nn;
      }
      if (16 * q < Q1MAX && k < nq1) {
        const real* mm = mt + (2 + ((m.kind1 == 1 && p1r[k] < real(0)) ? 1 : 0)) * MAXN;
        for (int s2 = 0; s2 <= m.N1; ++s2) gp[q] += tabr1[k * MAXN + s2] * mm[s2];
      }
    }
    // rescale g_R so that sum_i g_R sum_j g_phi is exactly the target sum D + sum R (f_eq - R
    // of phase D then carries the cell's mass; see normalise_equilibrium): g_R <- g_R (1 - delta)
    real scale0;  // FP64 path: the factor of g_R
    float delta = 0.f;
    if constexpr (F32) {
      // A = sum g_R sum g_phi and the target sum D + sum R, both in float-float;
      // delta = (A - target) / A, where A_hi - target_hi is exact (the two are close)
      float a0, a0e, a1, a1e;
      two_sum(gr[0], gr[1], a0, a0e);
      two_sum(gp[0], gp[1], a1, a1e);
      half_sum_comp(a0, a0e);
      half_sum_comp(a1, a1e);
      const float Ah = a0 * a1;
      const float Al = fmaf(a0, a1e, fmaf(a0e, a1, fmaf(a0, a1, -Ah)));
      float th, tl;
      two_sum(sn, m.ref_sumf[0], th, tl);
      tl = tl + (en + m.ref_sumf[1]);
      delta = (__fsub_rn(Ah, th) + (Al - tl)) / Ah;
      scale0 = real(0);
    } else {
      const double a0 = half_sum(double(gr[0]) + double(gr[1])), a1 = half_sum(double(gp[0]) + double(gp[1]));
      scale0 = real((dn + m.ref_n) / (a0 * a1));
    }
    if (has) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = hl + 16 * q;
        if (16 * q < Q0MAX && k < nq0)
          gRn[t * MAXQ + k] = p_set(F32 ? real(fmaf(-float(gr[q]), delta, float(gr[q]))) : gr[q] * scale0);
        if (16 * q < Q1MAX && k < nq1) gP[t * MAXQ + k] = p_set(gp[q]);
      }
    }
  }
  // Single-precision fixed-shape kernels contract both fields of a velocity in one task
  // (packed FP32x2 against duplicated coefficients); the others one field per task.
  constexpr bool PAIRED = F32 && EXACT;
  constexpr int TPF = PAIRED ? 1 : 2;  // tasks per (cell, column) and per (cell, row)
  constexpr int HQ = KArgs<real>::HQ;
  // lbuf = -(p^phi)^2 K^R f (one task per (cell, [field,] j): a column of nq0 values)
  auto force_R = [&](int x) {
    if constexpr (PAIRED) {  // even and odd parts under the reflection of axis 0 (KArgs)
      constexpr int H = Q0MAX / 2;
      const int j = x % Q1MAX, t = x / Q1MAX;
      const real* F = tile + (t + 3) * row;
      real* Lr = lbuf + t * row;
      // node k of the first half and its mirror refl(k) = k + H (half range) or Q - 1 - k
      // (full range): the mirror's pair sits at r0 + k rs
      const int rs = m.kind0 == 1 ? 2 * Q1MAX : -2 * Q1MAX;
      const int r0 = 2 * refl(m.kind0, Q0MAX, 0) * Q1MAX + 2 * j;
      pair_t<real> e[H], o[H];
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const pair_t<real> fk = p_load(F + 2 * j + 2 * k * Q1MAX), fr = p_load(F + r0 + k * rs);
        e[k] = p_add(fk, fr);
        o[k] = p_sub(fk, fr);
      }
      const pair_t<real> w = p_set(-p1r[j] * p1r[j]);
#pragma unroll
      for (int i = 0; i < H; ++i) {
        pair_t<real> pe = p_set(real(0)), mo = p_set(real(0));
#pragma unroll
        for (int k = 0; k < H; ++k) {
          pe = p_fma(kk.pairs.P0[i * HQ + k], e[k], pe);
          mo = p_fma(kk.pairs.M0[i * HQ + k], o[k], mo);
        }
        p_store(Lr + 2 * j + 2 * i * Q1MAX, p_mul(w, p_add(mo, pe)));
        p_store(Lr + r0 + i * rs, p_mul(w, p_sub(mo, pe)));
      }
    } else {
      const int j = x % nq1, td2 = x / nq1, d = td2 & 1, t = td2 >> 1;
      const real* F = tile + (t + 3) * row + d;
      real* Lr = lbuf + t * row + d;
      const real w = -p1r[j] * p1r[j];
      if constexpr (EXACT) {  // as above, one field
        constexpr int H = Q0MAX / 2;
        const int rs = m.kind0 == 1 ? 2 * Q1MAX : -2 * Q1MAX;
        const int r0 = 2 * refl(m.kind0, Q0MAX, 0) * Q1MAX + 2 * j;
        real e[H], o[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
          const real fk = F[2 * j + 2 * k * Q1MAX], fr = F[r0 + k * rs];
          e[k] = fk + fr;
          o[k] = fk - fr;
        }
#pragma unroll
        for (int i = 0; i < H; ++i) {
          real pe = 0, mo = 0;
#pragma unroll
          for (int k = 0; k < H; ++k) {
            pe += kk.split.P0[i * HQ + k] * e[k];
            mo += kk.split.M0[i * HQ + k] * o[k];
          }
          Lr[2 * j + 2 * i * Q1MAX] = w * (mo + pe);
          Lr[r0 + i * rs] = w * (mo - pe);
        }
      } else {
        real col[Q0MAX];
#pragma unroll
        for (int ip = 0; ip < Q0MAX; ++ip) col[ip] = ip < nq0 ? F[2 * (ip * nq1 + j)] : real(0);
#pragma unroll
        for (int i = 0; i < Q0MAX; ++i) {
          if (i < nq0) {
            real acc = 0;
#pragma unroll
            for (int ip = 0; ip < Q0MAX; ++ip)
              if (ip < nq0) acc += kk.full.K0[i * MAXQ + ip] * col[ip];
            Lr[2 * (i * nq1 + j)] = w * acc;
          }
        }
      }
    }
  };
  // lbuf += p^R K~^phi f (one task per (cell, [field,] i): a row of nq1 values)
  auto force_phi = [&](int x) {
    if constexpr (PAIRED) {  // even and odd parts under the reflection of axis 1 (KArgs)
      constexpr int H = Q1MAX / 2;
      const int i = x % Q0MAX, t = x / Q0MAX;
      const real* F = tile + (t + 3) * row + 2 * i * Q1MAX;
      real* Lr = lbuf + t * row + 2 * i * Q1MAX;
      const int rs = m.kind1 == 1 ? 2 : -2;  // the mirror of node k sits at r0 + k rs
      const int r0 = 2 * refl(m.kind1, Q1MAX, 0);
      pair_t<real> e[H], o[H];
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const pair_t<real> fk = p_load(F + 2 * k), fr = p_load(F + r0 + k * rs);
        e[k] = p_add(fk, fr);
        o[k] = p_sub(fk, fr);
      }
      const pair_t<real> pr = p_set(p0r[i]);
#pragma unroll
      for (int j = 0; j < H; ++j) {
        pair_t<real> pe = p_set(real(0)), mo = p_set(real(0));
#pragma unroll
        for (int k = 0; k < H; ++k) {
          pe = p_fma(kk.pairs.P1[j * HQ + k], e[k], pe);
          mo = p_fma(kk.pairs.M1[j * HQ + k], o[k], mo);
        }
        p_store(Lr + 2 * j, p_fma(pr, p_add(pe, mo), p_load(Lr + 2 * j)));
        p_store(Lr + r0 + j * rs, p_fma(pr, p_sub(pe, mo), p_load(Lr + r0 + j * rs)));
      }
    } else {
      const int i = x % nq0, td2 = x / nq0, d = td2 & 1, t = td2 >> 1;
      const real* F = tile + (t + 3) * row + d + 2 * i * nq1;
      real* Lr = lbuf + t * row + d + 2 * i * nq1;
      const real pr = p0r[i];
      if constexpr (EXACT) {  // as above, one field
        constexpr int H = Q1MAX / 2;
        const int rs = m.kind1 == 1 ? 2 : -2;
        const int r0 = 2 * refl(m.kind1, Q1MAX, 0);
        real e[H], o[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
          const real fk = F[2 * k], fr = F[r0 + k * rs];
          e[k] = fk + fr;
          o[k] = fk - fr;
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
          real pe = 0, mo = 0;
#pragma unroll
          for (int k = 0; k < H; ++k) {
            pe += kk.split.P1[j * HQ + k] * e[k];
            mo += kk.split.M1[j * HQ + k] * o[k];
          }
          Lr[2 * j] += pr * (pe + mo);
          Lr[r0 + j * rs] += pr * (pe - mo);
        }
      } else {
        real rw[Q1MAX];
#pragma unroll
        for (int jp = 0; jp < Q1MAX; ++jp) rw[jp] = jp < nq1 ? F[2 * jp] : real(0);
#pragma unroll
        for (int j = 0; j < Q1MAX; ++j) {
          if (j < nq1) {
            real acc = 0;
#pragma unroll
            for (int jp = 0; jp < Q1MAX; ++jp)
              if (jp < nq1) acc += kk.full.Kt1[j * MAXQ + jp] * rw[jp];
            Lr[2 * j] += pr * acc;
          }
        }
      }
    }
  };
  // Both contractions read only the owned cells, which phase A does not change.  When
  // some warps have no cell and the tasks come to at most six per idle thread, those
  // warps run all of them during phase A (the K~^phi tasks after a barrier among those
  // warps only); otherwise every thread takes K^R tasks after phase A and K~^phi tasks
  // after a CTA barrier.
  const int nR = TCe * TPF * nq1, nP = TCe * TPF * nq0;
  const int nfree = NA < NW ? NT - 32 * NA : 0;
  const bool early = nR + nP <= 6 * nfree;  // uniform across the CTA
  const bool runs = !early || warp >= NA;
  const int f0 = early ? tid - 32 * NA : tid, fs = early ? nfree : NT;
  if (runs)
    for (int x = f0; x < nR; x += fs) force_R(x);
  if (!early) __syncthreads();
  else if (runs) asm volatile("bar.sync 1, %0;" ::"r"(nfree) : "memory");
  if (runs)
    for (int x = f0; x < nP; x += fs) force_phi(x);
  __syncthreads();

  if (tix + int(gridDim.x) < a.n_tiles) td_next = a.tiles[tix + gridDim.x];

  // stage the next tile into the other buffer, the source of the previous tile's store
  if (nbuf == 2 && warp == 0 && tix + int(gridDim.x) < a.n_tiles) {
    if (lane == 0) bulk_wait_read_all();
    __syncwarp();
    stage_tile(td_next, b ^ 1);
  }

  // ==== phase B: the walls
  for (int wall = 0; wall < 2; ++wall) {
    // every tile whose stencils reach a ghost cell fills the ghosts itself
    const bool active = wall == 0 ? (c0 < 3) : (c0 + TCe + 3 > n);
    if (!active) continue;  // uniform across the CTA
    if (in.halo & (1 << wall)) {
      // a slab end: the three ghost cells are the neighbouring slab's, in increasing
      // radius (below the slab at the inner end, above it at the outer end)
      const real* hb = a.halo + (size_t(td.inst) * 2 + wall) * 3 * row;
      const int sA = wall == 0 ? 3 - c0 : (n - 1 - c0 + 3);  // slot of the edge cell
      for (int x = tid; x < 3 * V; x += NT) {
        const int q = x / V, v = x - q * V;  // ghost q (increasing radius), velocity v
        const int slot = wall == 0 ? sA - 3 + q : sA + 1 + q;
        if (slot >= 0 && slot < TC + 6) p_store(tile + slot * row + 2 * v, p_load(hb + q * row + 2 * v));
      }
      continue;
    }
    const double Tw = wall == 0 ? in.T_in : in.T_out;
    const double sgn = wall == 0 ? 1.0 : -1.0;  // incoming half: p^R > 0 at the inner wall
    __syncthreads();
    {  // the wall's equilibrium factors and incoming flux, computed by the host
      const WallEq& we = a.wall[td.inst * 2 + wall];
      for (int k = tid; k < nq0 + nq1; k += NT) {
        if (k < nq0) gw0[k] = we.g0[k];
        else gw1[k - nq0] = we.g1[k - nq0];
      }
      if (tid == 0) mw[0] = we.in_flux;
    }
    __syncthreads();
    // outgoing wall flux of f' (field 0) and the incoming equilibrium flux, FP64 sums
    const int sA = wall == 0 ? 3 - c0 : (n - 1 - c0 + 3);  // slot of the wall-adjacent cell
    const int dir = wall == 0 ? 1 : -1;                // towards the interior
    double num = 0;
    for (int v = tid; v < V; v += NT) {
      const int i = v / nq1, j = v - i * nq1;
      if (!(sgn * p0d[i] < 0.0)) continue;
      // the same pair reconstruction as phase D (field 0 enters n_w)
      pair_t<real> F0 = p_load(tile + sA * row + 2 * v);
      pair_t<real> F1 = p_load(tile + (sA + dir) * row + 2 * v);
      pair_t<real> F2 = p_load(tile + (sA + 2 * dir) * row + 2 * v);
      if constexpr (FT) {  // F~ of the three wall-adjacent cells
        const long long e0 = in.cell0 + (wall == 0 ? 0 : n - 1);
        const pair_t<real> R2 = p_set(w0r[i] * w1r[j]);
        F0 = p_mul(p_add(F0, R2), p_set(a.sqrtg[e0]));
        F1 = p_mul(p_add(F1, R2), p_set(a.sqrtg[e0 + dir]));
        F2 = p_mul(p_add(F2, R2), p_set(a.sqrtg[e0 + 2 * dir]));
      }
      const pair_t<real> G0 = p_fma(F1, p_set(real(-3)), p_fma(F0, p_set(real(3)), F2));
      const pair_t<real> G1 = p_fma(F1, p_set(real(-8)), p_fma(F0, p_set(real(6)), p_mul(F2, p_set(real(3)))));
      num += double(weno5p<real>(F2, F1, F0, G0, G1, iw0[i] * iw1[j]).x) * p0d[i];
    }
    num = warp_sum<real>(num);
    if (lane == 0) red[warp] = num;
    __syncthreads();
    if (tid == 0) {
      double sacc = FT ? 0.0 : (wall == 0 ? m.ref_flux_neg : m.ref_flux_pos);  // chi: the outgoing flux of R
      for (int w = 0; w < NW; ++w) sacc += red[w];
      const double nwv = -sacc / mw[0];
      mw[1] = nwv;
      a.nw[td.inst * 2 + wall] = nwv;
      if (!isfinite(nwv)) atomicOr(a.err, ERR_NONFINITE);
    }
    __syncthreads();
    const double nwd = mw[1];
    for (int v = tid; v < V; v += NT) {
      const int i = v / nq1, j = v - i * nq1;
      pair_t<real> g1, g2, g3;  // ghosts at distance 1, 2, 3 from the wall
      if (sgn * p0d[i] < 0.0) {
        pair_t<real> F0 = p_load(tile + sA * row + 2 * v);
        pair_t<real> F1 = p_load(tile + (sA + dir) * row + 2 * v);
        pair_t<real> F2 = p_load(tile + (sA + 2 * dir) * row + 2 * v);
        if constexpr (FT) {
          const long long e0 = in.cell0 + (wall == 0 ? 0 : n - 1);
          const pair_t<real> R2 = p_set(w0r[i] * w1r[j]);
          F0 = p_mul(p_add(F0, R2), p_set(a.sqrtg[e0]));
          F1 = p_mul(p_add(F1, R2), p_set(a.sqrtg[e0 + dir]));
          F2 = p_mul(p_add(F2, R2), p_set(a.sqrtg[e0 + 2 * dir]));
        }
        g1 = p_fma(F1, p_set(real(-3)), p_fma(F0, p_set(real(3)), F2));
        g2 = p_fma(F1, p_set(real(-8)), p_fma(F0, p_set(real(6)), p_mul(F2, p_set(real(3)))));
        if constexpr (FT) {  // stored as F~ - R
          const pair_t<real> nR = p_set(-(w0r[i] * w1r[j]));
          g1 = p_add(g1, nR);
          g2 = p_add(g2, nR);
        }
        g3 = g2;  // never read by an outgoing stencil
      } else {  // f_eq(n_w, u_w, T_w) - R
        const double e = nwd * gw0[i] * gw1[j], r = m.w0[i] * m.w1[j];
        g1 = g2 = g3 = p_make(real(e - r), real(e * Tw - r));
      }
      const int s1 = sA - dir, s2 = sA - 2 * dir, s3 = sA - 3 * dir;
      if (s1 >= 0 && s1 < TC + 6) p_store(tile + s1 * row + 2 * v, g1);
      if (s2 >= 0 && s2 < TC + 6) p_store(tile + s2 * row + 2 * v, g2);
      if (s3 >= 0 && s3 < TC + 6) p_store(tile + s3 * row + 2 * v, g3);
    }
  }
  // phase D reads the ghost rows the walls wrote; an interior tile wrote nothing since the
  // barrier after phase A (warp 0's staging goes to the other buffer)
  if (c0 < 3 || c0 + TCe + 3 > n) __syncthreads();  // uniform across the CTA
  real* sgs = nullptr;  // f~: sqrt(g) of the tile's slots, 1 past the walls (ghost rows hold F~ - R)
  if constexpr (FT) {
    __shared__ real sgs_[TC + 6];
    sgs = sgs_;
    for (int q = tid; q < TC + 6; q += NT) {
      const int cell = c0 - 3 + q;
      sgs_[q] = (cell >= 0 && cell < n) ? a.sqrtg[in.cell0 + cell] : real(1);
    }
    __syncthreads();
  }

  // ==== phase D: WENO-5 fluxes along the cells, flux difference, BGK, RK3 combine (in place)
  const real dtr = F32 ? real(in.dt_f) : real(in.dt);
  const real ca = F32 ? real(a.caf) : real(a.ca);
  const real cc = (F32 ? real(a.ccf) : real(a.cc)) * dtr;
  using P = pair_t<real>;
  for (int v = tid; v < V; v += NT) {  // one velocity, both fields, walking the tile's cells
    const int i = v / nq1, j = v - i * nq1;
    const real pr = p0r[i];
    const bool up = pr >= real(0);
    const real sc = iw0[i] * iw1[j];
    const P nrij = p_set(-(w0r[i] * w1r[j]));
    const P npr = p_set(-pr);
    real* S = tile + 2 * v;
    const real* Fl = a.Fl + size_t(in.cell0 + c0) * row + 2 * v;  // F_l of the owned cells, read once
    // the advected value of slot q: D (chi), F~ - R = (D + R) sqrt(g) - R (f~)
    const real Rr = w0r[i] * w1r[j];
    auto adv_val = [&](const real* x, int q) -> P {
      if constexpr (FT) return p_fma(p_load(x), p_set(sgs[q]), p_set(Rr * (sgs[q] - real(1))));
      else return p_load(x);
    };
    P FRv = p_set(real(0));  // f~: the inertial term of R for this velocity
    if constexpr (FT) FRv = p_set(a.forceR[v]);
    P w0 = adv_val(S, 0), w1 = adv_val(S + row, 1), w2 = adv_val(S + 2 * row, 2), w3 = adv_val(S + 3 * row, 3);
    P w4 = adv_val(S + 4 * row, 4), w5 = adv_val(S + 5 * row, 5);
    // upwind stencil: (w0..w4) for p^R >= 0, mirrored (w5..w1) otherwise
    P fm = weno5p<real>(p_sel(up, w0, w5), p_sel(up, w1, w4), p_sel(up, w2, w3), p_sel(up, w3, w2),
                        p_sel(up, w4, w1), sc);
    // F_l of the next cell is loaded one cell ahead (a global load, the only one of the walk)
    P fl_next = need_fl ? p_load(Fl) : p_set(real(0));
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      if (t < TCe) {
        const P fl = fl_next;
        if (need_fl && t + 1 < TCe) fl_next = p_load(Fl + (t + 1) * row);
        const P w6 = adv_val(S + (t + 6) * row, t + 6);
        const P fp = weno5p<real>(p_sel(up, w1, w6), p_sel(up, w2, w5), p_sel(up, w3, w4), p_sel(up, w4, w3),
                                  p_sel(up, w5, w2), sc);
        // -adv = -p^R (cp F_{s+1/2} - cm F_{s-1/2}); per-cell factors: shared-memory broadcasts
        P nadv = p_mul(p_fma(fp, ccp[t], p_mul(fm, cNcm[t])), npr);
        P Dc = w3;  // the cell's D
        if constexpr (FT) {
          nadv = p_fma(p_mul(npr, p_set(Rr)), p_add(ccp[t], cNcm[t]), nadv);  // the advection of R
          Dc = p_load(S + (t + 3) * row);
        }
        // f_eq - R for both fields: (g, T g) - R
        const P deq = p_fma(p_mul(gRn[t * MAXQ + i], gP[t * MAXQ + j]), cT1[t], nrij);
        P force = p_load(lbuf + t * row + 2 * v);
        if constexpr (FT) force = p_sub(force, FRv);
        // L = -adv + force / Rbar - (D - D_eq) / tau
        const P Lv = p_fma(p_sub(Dc, deq), cNtau[t], p_fma(force, cIR[t], nadv));
        P o = p_fma(Lv, p_set(cc), Dc);
        if (need_fl) o = p_fma(p_sub(fl, Dc), p_set(ca), o);
        p_store(S + (t + 3) * row, o);  // in place: this column's slot t+3 is not read again
        w0 = w1;
        w1 = w2;
        w2 = w3;
        w3 = w4;
        w4 = w5;
        w5 = w6;
        fm = fp;
      }
    }
  }
  // ---- bulk store of the owned cells (generic-proxy writes made visible to the async proxy first)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    bulk_s2g(a.Fout + size_t(in.cell0 + c0) * row, tile + 3 * row, unsigned(TCe * row * sizeof(real)));
    bulk_commit();
    if (nbuf == 1) bulk_wait_read_all();
  }
  if (nbuf == 1) __syncthreads();  // the next tile is staged into this buffer
  }
  if (tid == 0) bulk_wait_all();  // the stores have read their source before the CTA exits
}

}  // namespace vlb
