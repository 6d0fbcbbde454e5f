// One TVD-RK3 stage of the chi-formulation circular Couette update, fused into
// one kernel per tile of TC cells of one instance (all momenta of those cells):
//
//   bulk-copy the tile and its three-cell halo to shared memory
//   -> moments per cell (Eq. macro_red)          -> truncated equilibrium and tau
//   -> walls: extrapolated outgoing ghosts (Eq. extrapol), wall flux, n_w
//      (Eq. nw), incoming ghosts f_eq(n_w, u_w, T_w) (Eq. weno_populate)
//   -> inertial force (1/R)[(p^phi)^2 K^R f - p^R K~^phi f] (Eq. boltz_couette_kom)
//   -> WENO-5 fluxes along the cells, chi flux difference, BGK, RK3 combine
//      (Eqs. weno5_flux, flux_kom_R / flux_kom_eta, BGK, rk3) -> global.
#pragma once
#include "vlb_device.cuh"

namespace vlb {

template <typename real>
struct StageArgs {
  const real* Fprev;  // distribution L acts on
  const real* Fl;     // F_l of the step (read when ca != 0)
  real* Fout;
  double ca, cb, cc;  // Fout = ca F_l + cb F_prev + cc dt L[F_prev]
  const InstDesc* inst;
  const TileDesc* tiles;
  int n_tiles;
  const GeoCell* geo;  // per global cell
  double* nw;          // 2 per instance: inner, outer wall density
  unsigned* err;
  int Vp;              // per-field stride of a cell row (>= nq0 nq1, multiple of 4)
  unsigned long long max_polls;
};

// Shared-memory carve-up, identical on host and device.
template <typename real, int TC, int NT>
struct StageSmem {
  static constexpr int NW = NT / 32;
  __host__ __device__ static size_t tile_off() { return 16; }
  __host__ __device__ static size_t lbuf_off(int Vp) { return tile_off() + size_t(TC + 6) * 2 * Vp * sizeof(real); }
  __host__ __device__ static size_t fl_off(int Vp) { return lbuf_off(Vp) + size_t(TC) * 2 * Vp * sizeof(real); }
  __host__ __device__ static size_t dbl_off(int Vp) {
    size_t o = fl_off(Vp) + size_t(TC) * 2 * Vp * sizeof(real);
    return (o + 15) & ~size_t(15);
  }
  // doubles: p0, p1 (MAXQ each), tab0, tab1 (MAXQ*MAXN each, wall equilibria), reduction (NW*4),
  // wall scratch (2*MAXQ + 16)
  static constexpr size_t n_dbl = 2 * MAXQ + 2 * MAXQ * MAXN + NW * 4 + 2 * MAXQ + 16;
  __host__ __device__ static size_t real_off(int Vp) { return dbl_off(Vp) + n_dbl * sizeof(double); }
  // reals: p0, p1, 1/w0, 1/w1 (MAXQ each), tab0, tab1 (MAXQ*MAXN each), n g_R and g_phi (TC*MAXQ each),
  // cell n, T, u0, u1, 1/tau, cp, cm, 1/Rbar (TC each), moment vectors (TC*4*MAXN)
  static constexpr size_t n_real = 4 * MAXQ + 2 * MAXQ * MAXN + 2 * TC * MAXQ + 8 * TC + TC * 4 * MAXN;
  __host__ __device__ static size_t bytes(int Vp) { return real_off(Vp) + n_real * sizeof(real); }
};

template <typename real, int TC, int Q0MAX, int Q1MAX, int NT, bool EXACT>
__global__ void __launch_bounds__(NT) couette_stage_kernel(const __grid_constant__ StageArgs<real> a,
                                                           const __grid_constant__ ModelArgs m,
                                                           const __grid_constant__ KArgs<real> kk) {
  using L = StageSmem<real, TC, NT>;
  constexpr int NW = L::NW;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // exact instantiations fix the node counts at compile time; the generic one reads them
  const int nq0 = EXACT ? Q0MAX : m.nq0;
  const int nq1 = EXACT ? Q1MAX : m.nq1;
  const int V = nq0 * nq1, Vp = a.Vp;
  const size_t row = 2 * size_t(Vp);

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  real* tile = reinterpret_cast<real*>(smem + L::tile_off());
  real* lbuf = reinterpret_cast<real*>(smem + L::lbuf_off(Vp));
  real* flb = reinterpret_cast<real*>(smem + L::fl_off(Vp));  // F_l of the owned cells (stages 2, 3)
  double* dp = reinterpret_cast<double*>(smem + L::dbl_off(Vp));
  double* p0d = dp;
  double* p1d = p0d + MAXQ;
  double* tab0 = p1d + MAXQ;
  double* tab1 = tab0 + MAXQ * MAXN;
  double* red = tab1 + MAXQ * MAXN;
  double* wl = red + NW * 4;      // wall scratch
  real* rp = reinterpret_cast<real*>(smem + L::real_off(Vp));
  real* p0r = rp;
  real* p1r = p0r + MAXQ;
  real* iw0 = p1r + MAXQ;  // 1 / w_i
  real* iw1 = iw0 + MAXQ;  // 1 / w_j
  real* tabr0 = iw1 + MAXQ;  // equilibrium tables in the bulk type
  real* tabr1 = tabr0 + MAXQ * MAXN;
  real* gRn = tabr1 + MAXQ * MAXN;  // [t][i] n_t g_{R,i}
  real* gP = gRn + TC * MAXQ;
  real* cn = gP + TC * MAXQ;
  real* cTr = cn + TC;
  real* cu0 = cTr + TC;
  real* cu1 = cu0 + TC;
  real* cItau = cu1 + TC;
  real* ccp = cItau + TC;
  real* ccm = ccp + TC;
  real* cIR = ccm + TC;
  real* mv = cIR + TC;  // [t][axis*2 + side][s]

  const TileDesc td = a.tiles[blockIdx.x];
  const InstDesc in = a.inst[td.inst];
  const int n = in.n_cells, c0 = td.c0;
  const int TCe = min(TC, n - c0);
  const int lo = max(c0 - 3, 0), hi = min(c0 + TC + 3, n);

  // ---- stage the tile (cells lo..hi-1 at slots lo-c0+3 ...) with bulk copies
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool need_fl = a.ca != 0.0;
  if (warp == 0) {
    const unsigned rbytes = unsigned(row * sizeof(real));
    if (lane == 0) mbar_expect_tx(bar, rbytes * unsigned(hi - lo + (need_fl ? TCe : 0)));
    __syncwarp();
    for (int c = lo + lane; c < hi; c += 32)
      bulk_g2s(tile + size_t(c - c0 + 3) * row, a.Fprev + size_t(in.cell0 + c) * row, rbytes, bar);
    if (need_fl)
      for (int t = lane; t < TCe; t += 32)
        bulk_g2s(flb + size_t(t) * row, a.Fl + size_t(in.cell0 + c0 + t) * row, rbytes, bar);
  }
  for (int x = tid; x < MAXQ; x += NT) {
    p0d[x] = m.p0[x];
    p1d[x] = m.p1[x];
    p0r[x] = real(m.p0[x]);
    p1r[x] = real(m.p1[x]);
    iw0[x] = m.w0[x] > 0.0 ? real(1) / real(m.w0[x]) : real(0);
    iw1[x] = m.w1[x] > 0.0 ? real(1) / real(m.w1[x]) : real(0);
  }
  for (int x = tid; x < MAXQ * MAXN; x += NT) {
    tab0[x] = m.tab0[x];
    tab1[x] = m.tab1[x];
    tabr0[x] = sizeof(real) == 4 ? real(m.tab0f[x]) : real(m.tab0[x]);
    tabr1[x] = sizeof(real) == 4 ? real(m.tab1f[x]) : real(m.tab1[x]);
  }
  for (int t = tid; t < TCe; t += NT) {
    const GeoCell g = a.geo[in.cell0 + c0 + t];
    ccp[t] = real(g.cp);
    ccm[t] = real(g.cm);
    cIR[t] = real(g.inv_rbar);
  }
  bool ok = mbar_wait(bar, 0, a.max_polls);
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
    mbar_wait(bar, 0, a.max_polls);  // let the copies land before the CTA exits
    return;
  }

  // ---- moments per cell: per-lane partial sums in the bulk type, FP64 across lanes
  for (int t = warp; t < TCe; t += NW) {
    const real* F = tile + size_t(t + 3) * row;
    real sn = 0, sr = 0, sp = 0, se = 0;
    for (int v = lane; v < V; v += 32) {
      const int i = v / nq1, j = v - i * nq1;
      const real f1 = F[v], f2 = F[Vp + v], pr = p0r[i], pp = p1r[j];
      sn += f1;
      sr += pr * f1;
      sp += pp * f1;
      se += (pr * pr + pp * pp) * f1 + f2;
    }
    const double dn = warp_sum<real>(double(sn)), dr = warp_sum<real>(double(sr));
    const double dpp = warp_sum<real>(double(sp)), de = warp_sum<real>(double(se));
    if (lane == 0) {  // the sums are FP64; the derived fields are formed in the bulk type
      const real n = real(dn), u0 = real(dr) / n, u1 = real(dpp) / n;
      const real T = (real(de) - n * (u0 * u0 + u1 * u1)) / (real(3) * n);
      cn[t] = n;
      cu0[t] = u0;
      cu1[t] = u1;
      cTr[t] = T;
      cItau[t] = real(1) / relaxation_time<real>(in.tau_mode, real(in.kn), n, T);
    }
  }
  __syncthreads();
  for (int x = tid; x < TCe * 4; x += NT) {
    const int t = x >> 2, ax = (x >> 1) & 1, side = x & 1;
    const real u = (ax ? cu1[t] : cu0[t]) * (side ? real(-1) : real(1));
    eq_moment_vector<real>(ax ? m.kind1 : m.kind0, ax ? m.N1 : m.N0, u, cTr[t], mv + (t * 4 + ax * 2 + side) * MAXN);
  }
  __syncthreads();
  for (int x = tid; x < TCe * (nq0 + nq1); x += NT) {
    const int t = x / (nq0 + nq1);
    int k = x - t * (nq0 + nq1);
    if (k < nq0) {
      const int side = (m.kind0 == 1 && p0r[k] < real(0)) ? 1 : 0;
      const real* mm = mv + (t * 4 + side) * MAXN;
      real g = 0;
      for (int s = 0; s <= m.N0; ++s) g += tabr0[k * MAXN + s] * mm[s];
      gRn[t * MAXQ + k] = cn[t] * g;
    } else {
      k -= nq0;
      const int side = (m.kind1 == 1 && p1r[k] < real(0)) ? 1 : 0;
      const real* mm = mv + (t * 4 + 2 + side) * MAXN;
      real g = 0;
      for (int s = 0; s <= m.N1; ++s) g += tabr1[k * MAXN + s] * mm[s];
      gP[t * MAXQ + k] = g;
    }
  }

  // ---- diffuse-reflection walls
  for (int wall = 0; wall < 2; ++wall) {
    const bool active = wall == 0 ? (c0 == 0) : (c0 + TC + 3 > n);
    if (!active) continue;  // uniform across the CTA
    const double uw = wall == 0 ? in.u_in : in.u_out;
    const double Tw = wall == 0 ? in.T_in : in.T_out;
    const double sgn = wall == 0 ? 1.0 : -1.0;  // incoming half: p^R > 0 at the inner wall
    double* gw0 = wl;
    double* gw1 = wl + MAXQ;
    double* mw = wl + 2 * MAXQ;  // [0] incoming equilibrium flux, [1] n_w
    __syncthreads();
    if (tid == 0) {
      double m0p[MAXN], m0m[MAXN], m1p[MAXN], m1m[MAXN];
      eq_moment_vector<double>(m.kind0, m.N0, 0.0, Tw, m0p);
      eq_moment_vector<double>(m.kind0, m.N0, -0.0, Tw, m0m);
      eq_moment_vector<double>(m.kind1, m.N1, uw, Tw, m1p);
      eq_moment_vector<double>(m.kind1, m.N1, -uw, Tw, m1m);
      for (int k = 0; k < nq0; ++k) {
        const double* mm = (m.kind0 == 1 && p0d[k] < 0.0) ? m0m : m0p;
        double g = 0;
        for (int s = 0; s <= m.N0; ++s) g += tab0[k * MAXN + s] * mm[s];
        gw0[k] = g;
      }
      double s1 = 0;
      for (int k = 0; k < nq1; ++k) {
        const double* mm = (m.kind1 == 1 && p1d[k] < 0.0) ? m1m : m1p;
        double g = 0;
        for (int s = 0; s <= m.N1; ++s) g += tab1[k * MAXN + s] * mm[s];
        gw1[k] = g;
        s1 += g;
      }
      double s0 = 0;
      for (int k = 0; k < nq0; ++k)
        if (sgn * p0d[k] > 0.0) s0 += gw0[k] * p0d[k];
      mw[0] = s0 * s1;  // flux of f_eq(1, u_w, T_w) through the wall, incoming half
    }
    __syncthreads();
    // outgoing wall flux of f' (field 0)
    const int sA = wall == 0 ? 3 : (n - 1 - c0 + 3);  // slot of the wall-adjacent cell
    const int dir = wall == 0 ? 1 : -1;                // towards the interior
    double num = 0;
    for (int v = tid; v < V; v += NT) {
      const int i = v / nq1, j = v - i * nq1;
      if (!(sgn * p0d[i] < 0.0)) continue;
      const real F0 = tile[size_t(sA) * row + v];
      const real F1 = tile[size_t(sA + dir) * row + v];
      const real F2 = tile[size_t(sA + 2 * dir) * row + v];
      const real G0 = real(3) * F0 - real(3) * F1 + F2;
      const real G1 = real(6) * F0 - real(8) * F1 + real(3) * F2;
      num += double(weno5<real>(F2, F1, F0, G0, G1, iw0[i] * iw1[j])) * p0d[i];
    }
    num = warp_sum<real>(num);
    if (lane == 0) red[warp] = num;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < NW; ++w) s += red[w];
      const double nwv = -s / mw[0];
      mw[1] = nwv;
      a.nw[td.inst * 2 + wall] = nwv;
      if (!isfinite(nwv)) atomicOr(a.err, ERR_NONFINITE);
    }
    __syncthreads();
    const double nwv = mw[1];
    for (int x = tid; x < 2 * V; x += NT) {
      const int d = x >= V, v = x - d * V;
      const int i = v / nq1, j = v - i * nq1;
      real g1, g2, g3;  // ghosts at distance 1, 2, 3 from the wall
      if (sgn * p0d[i] < 0.0) {
        const real F0 = tile[size_t(sA) * row + d * Vp + v];
        const real F1 = tile[size_t(sA + dir) * row + d * Vp + v];
        const real F2 = tile[size_t(sA + 2 * dir) * row + d * Vp + v];
        g1 = real(3) * F0 - real(3) * F1 + F2;
        g2 = real(6) * F0 - real(8) * F1 + real(3) * F2;
        g3 = g2;  // never read by an outgoing stencil
      } else {
        const double f = nwv * gw0[i] * gw1[j] * (d ? Tw : 1.0);
        g1 = g2 = g3 = real(f);
      }
      const int s1 = sA - dir, s2 = sA - 2 * dir, s3 = sA - 3 * dir;
      if (s1 >= 0 && s1 < TC + 6) tile[size_t(s1) * row + d * Vp + v] = g1;
      if (s2 >= 0 && s2 < TC + 6) tile[size_t(s2) * row + d * Vp + v] = g2;
      if (s3 >= 0 && s3 < TC + 6) tile[size_t(s3) * row + d * Vp + v] = g3;
    }
  }
  __syncthreads();

  // ---- inertial force: lbuf = -(p^phi)^2 K^R f + p^R K~^phi f  (times 1/Rbar later)
  for (int x = tid; x < TCe * 2 * nq1; x += NT) {
    const int j = x % nq1, td2 = x / nq1, d = td2 & 1, t = td2 >> 1;
    const real* F = tile + size_t(t + 3) * row + d * Vp;
    real col[Q0MAX];
#pragma unroll
    for (int ip = 0; ip < Q0MAX; ++ip) col[ip] = ip < nq0 ? F[ip * nq1 + j] : real(0);
    real* Lr = lbuf + size_t(t * 2 + d) * Vp;
    const real w = -p1r[j] * p1r[j];
#pragma unroll
    for (int i = 0; i < Q0MAX; ++i) {
      if (i < nq0) {
        real acc = 0;
#pragma unroll
        for (int ip = 0; ip < Q0MAX; ++ip)
          if (ip < nq0) acc += kk.K0[i * MAXQ + ip] * col[ip];
        Lr[i * nq1 + j] = w * acc;
      }
    }
  }
  __syncthreads();
  for (int x = tid; x < TCe * 2 * nq0; x += NT) {
    const int i = x % nq0, td2 = x / nq0, d = td2 & 1, t = td2 >> 1;
    const real* F = tile + size_t(t + 3) * row + d * Vp + i * nq1;
    real rw[Q1MAX];
#pragma unroll
    for (int jp = 0; jp < Q1MAX; ++jp) rw[jp] = jp < nq1 ? F[jp] : real(0);
    real* Lr = lbuf + size_t(t * 2 + d) * Vp + i * nq1;
    const real pr = p0r[i];
#pragma unroll
    for (int j = 0; j < Q1MAX; ++j) {
      if (j < nq1) {
        real acc = 0;
#pragma unroll
        for (int jp = 0; jp < Q1MAX; ++jp)
          if (jp < nq1) acc += kk.Kt1[j * MAXQ + jp] * rw[jp];
        Lr[j] += pr * acc;
      }
    }
  }
  __syncthreads();

  // ---- WENO-5 fluxes along the cells, flux difference, BGK, RK3 combine
  const real dtr = real(in.dt);
  const real ca = real(a.ca), cb = real(a.cb), cc = real(a.cc) * dtr;
  for (int x = tid; x < 2 * V; x += NT) {
    const int d = x >= V, v = x - d * V;
    const int i = v / nq1, j = v - i * nq1;
    const real pr = p0r[i];
    const bool up = pr >= real(0);
    const real sc = iw0[i] * iw1[j];
    real* S = tile + d * Vp + v;
    const real* Fl = flb + d * Vp + v;
    real w0 = S[0], w1 = S[row], w2 = S[2 * row], w3 = S[3 * row], w4 = S[4 * row], w5 = S[5 * row];
    // upwind stencil: (w0..w4) for p^R >= 0, mirrored (w5..w1) otherwise
    real fm = weno5<real>(up ? w0 : w5, up ? w1 : w4, up ? w2 : w3, up ? w3 : w2, up ? w4 : w1, sc);
    for (int t = 0; t < TCe; ++t) {
      const real w6 = S[size_t(t + 6) * row];
      const real fp = weno5<real>(up ? w1 : w6, up ? w2 : w5, up ? w3 : w4, up ? w4 : w3, up ? w5 : w2, sc);
      const real adv = pr * (ccp[t] * fp - ccm[t] * fm);
      const real feq = gRn[t * MAXQ + i] * gP[t * MAXQ + j] * (d ? cTr[t] : real(1));
      const real Lv = -adv + lbuf[size_t(t * 2 + d) * Vp + v] * cIR[t] - (w3 - feq) * cItau[t];
      real o = cb * w3 + cc * Lv;
      if (need_fl) o += ca * Fl[size_t(t) * row];
      S[size_t(t + 3) * row] = o;  // in place: this column's slot t+3 is not read again
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = w4;
      w4 = w5;
      w5 = w6;
      fm = fp;
    }
  }
  // ---- bulk store of the owned cells (generic-proxy writes made visible to the async proxy first)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    bulk_s2g(a.Fout + size_t(in.cell0 + c0) * row, tile + 3 * row, unsigned(TCe * row * sizeof(real)));
    bulk_commit_and_wait_read();
  }
}

}  // namespace vlb
