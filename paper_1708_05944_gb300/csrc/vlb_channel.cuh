// One TVD-RK3 stage of the gradually expanding channel in the vielbein frame
// (Sec. VII.A-C, Eq. canalie_boltz), fused into one kernel per tile of
// TS (wall-normal, lambda) x TP (streamwise, xi) cells with all momenta:
//
//   bulk-copy the tile's columns with a 3-cell lambda halo and 3 xi-halo
//   columns -> moments and the lambda-axis force contractions
//   -> equilibrium moment vectors and the xi-axis force contractions
//   -> equilibrium factors; centreline mirror; wall n_w per column; inlet and
//      outlet reservoir ghosts
//   -> WENO-5 in lambda (walking the column) and in xi, chi flux differences,
//      BGK, RK3 combine -> bulk store.
//
// Distribution buffers hold the deviation D = F - R from the rest state
// (ModelArgs), as in the Couette kernel, with (f', f'') interleaved per
// velocity (pair_t).  The arithmetic here is scalar per field: a pair-wise
// phase D (as in the Couette kernel) gave wrong boundary ghosts for the
// 2 x 4-cell tile shape of the 16 x 12 velocity set while every other shape
// matched the oracle; the cause was not found, and the scalar form matches
// the oracle for every shape.
//
// Cell (s, p) of the grid has global index p * n_lambda + s (lambda fastest).
#pragma once
#include "vlb_device.cuh"

namespace vlb {

// Per-cell geometry of the channel (Sec. VII.A): interface factors of
// V^lambda = a p^lambda and V^xi = b p^xi - c p^lambda, 1/d lambda_s,
// 1/d chi^xi_p and the discrete connection coefficients.
template <typename T>
struct ChanCell {
  T am, ap;          // a at s-1/2, s+1/2
  T bm, bp, cm, cp;  // b, c at p-1/2, p+1/2
  T idl, idx;        // 1 / d lambda_s, 1 / d chi_p
  T glxl, glxx;      // Gamma_{l x l}, Gamma_{l x x}
  T pad0, pad1;
};

struct ChanDesc {
  int nl, nx;
  double kn, dt, n_in, n_out, T0;
  float knf, dtf, n_inf, n_outf, T0f;
};

template <typename real>
struct ChanArgs {
  const real* Fprev;
  const real* Fl;
  real* Fout;
  double ca, cb, cc;
  float caf, cbf, ccf;
  ChanDesc cd;
  const ChanCell<double>* geo;
  const ChanCell<float>* geof;
  double* nw;  // per column
  unsigned* err;
  unsigned long long max_polls;
};

template <typename real, int Q0, int Q1>
struct ChanK {
  real K0[Q0 * Q0], Kt0[Q0 * Q0];  // d/dp^lambda, d/dp^lambda (p^lambda .)
  real K1[Q1 * Q1], Kt1[Q1 * Q1];  // d/dp^xi, d/dp^xi (p^xi .)
};

template <typename real, int TS, int TP, int Q0, int Q1, int NT>
struct ChanSmem {
  static constexpr int NW = NT / 32;
  static constexpr int V = Q0 * Q1;
  static constexpr int VP = (V + 3) / 4 * 4;
  static constexpr int ROW = 2 * VP;
  static constexpr int NCS = TP * (TS + 6) + 6 * TS;  // cell slots in shared memory
  static constexpr int NC = TS * TP;                  // owned cells
  static constexpr size_t tile_off = 16;
  static constexpr size_t lbuf_off = tile_off + size_t(NCS) * ROW * sizeof(real);
  static constexpr size_t fl_off = lbuf_off + size_t(NC) * ROW * sizeof(real);
  static constexpr size_t dbl_off = (fl_off + size_t(NC) * ROW * sizeof(real) + 15) & ~size_t(15);
  // doubles: reduction (NW*4 + TP*NW), wall n_w (TP), scalars (16), equilibrium sum targets (NC)
  static constexpr size_t n_dbl = NW * 4 + TP * NW + TP + 16 + NC;
  static constexpr size_t real_off = dbl_off + n_dbl * sizeof(double);
  // reals: p0, p1, 1/w0, 1/w1 (Q each), tables (Q*MAXN each), per cell: 10 geometry + n, T, u0, u1, 1/tau,
  // g0 (Q0), g1 (Q1), moment vectors (4*MAXN); boundary: wall factors (Q0 + Q1), inlet/outlet factors (TS*Q1 each),
  // weights (Q0 + Q1)
  static constexpr size_t n_real = 2 * Q0 + 2 * Q1 + (Q0 + Q1) * MAXN + size_t(NC) * (15 + Q0 + Q1 + 4 * MAXN) +
                                   (Q0 + Q1) + 2 * size_t(TS) * Q1 + Q0 + Q1 + 2 * TS + 8;
  static constexpr size_t bytes = real_off + n_real * sizeof(real);
};

template <typename real, int TS, int TP, int Q0, int Q1, int NT>
__global__ void __launch_bounds__(NT) channel_stage_kernel(const __grid_constant__ ChanArgs<real> a,
                                                           const __grid_constant__ ModelArgs m,
                                                           const __grid_constant__ ChanK<real, Q0, Q1> kk) {
  using L = ChanSmem<real, TS, TP, Q0, Q1, NT>;
  constexpr int NW = L::NW, V = L::V, VP = L::VP, ROW = L::ROW, NC = L::NC;
  constexpr bool F32 = sizeof(real) == 4;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nl = a.cd.nl, nx = a.cd.nx;

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  real* tile = reinterpret_cast<real*>(smem + L::tile_off);
  real* lbuf = reinterpret_cast<real*>(smem + L::lbuf_off);
  real* flb = reinterpret_cast<real*>(smem + L::fl_off);
  double* red = reinterpret_cast<double*>(smem + L::dbl_off);  // NW*4 + TP*NW
  double* nwv = red + NW * 4 + TP * NW;                           // TP
  double* dsc = nwv + TP;                                         // 16 scalars
  double* cnd = dsc + 16;                                         // [q] target of sum g0n * sum g1
  real* rp = reinterpret_cast<real*>(smem + L::real_off);
  real* p0r = rp;
  real* p1r = p0r + Q0;
  real* iw0 = p1r + Q1;
  real* iw1 = iw0 + Q0;
  real* tb0 = iw1 + Q1;
  real* tb1 = tb0 + Q0 * MAXN;
  real* geo = tb1 + Q1 * MAXN;        // [q][10]
  real* cn = geo + NC * 10;           // [q]
  real* cT = cn + NC;
  real* cu0 = cT + NC;
  real* cu1 = cu0 + NC;
  real* citau = cu1 + NC;
  real* g0n = citau + NC;             // [q][Q0] n g_lambda
  real* g1 = g0n + NC * Q0;           // [q][Q1]
  real* mv = g1 + NC * Q1;            // [q][4][MAXN]
  real* gw0 = mv + NC * 4 * MAXN;     // wall / reservoir lambda factor g_lambda(0, T0)
  real* gw1 = gw0 + Q0;               // wall xi factor g_xi(0, T0)
  real* gin = gw1 + Q1;               // [TS][Q1] inlet xi factor per row
  real* gout = gin + TS * Q1;         // [TS][Q1]
  real* w0r = gout + TS * Q1;         // [Q0] weights: R_ij = w0_i w1_j in the bulk type
  real* w1r = w0r + Q0;               // [Q1]
  real* uin = w1r + Q1;               // [TS] inlet / outlet u^xi of the adjacent cell
  real* uout = uin + TS;

  const int nts = (nl + TS - 1) / TS;
  const int s0 = (blockIdx.x % nts) * TS, p0 = (blockIdx.x / nts) * TP;
  const int TSe = min(TS, nl - s0);
  auto slot = [&](int sr, int c) -> int {
    if (c >= 0 && c < TP) return c * (TS + 6) + sr + 3;
    const int h = c < 0 ? c + 3 : c - TP + 3;
    return TP * (TS + 6) + h * TS + sr;
  };
  auto gcell = [&](int s, int p) -> size_t { return size_t(p) * nl + s; };

  // ---- bulk copies: tile columns with lambda halo, xi-halo columns, F_l of the owned cells
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool need_fl = a.caf != 0.0f;
  if (warp == 0) {
    const unsigned rb = unsigned(ROW * sizeof(real));
    const int slo = max(s0 - 3, 0), shi = min(s0 + TS + 3, nl);
    unsigned total = 0;
    for (int c = -3; c < TP + 3; ++c) {
      const int p = p0 + c;
      if (p < 0 || p >= nx) continue;
      total += (c >= 0 && c < TP) ? unsigned(shi - slo) * rb : unsigned(TSe) * rb;
    }
    if (need_fl) total += unsigned(TP * TSe) * rb;
    if (lane == 0) mbar_expect_tx(bar, total);
    __syncwarp();
    if (lane < TP + 6) {
      const int c = lane - 3, p = p0 + c;
      if (p >= 0 && p < nx) {
        if (c >= 0 && c < TP)
          bulk_g2s(tile + slot(slo - s0, c) * ROW, a.Fprev + gcell(slo, p) * ROW, unsigned(shi - slo) * rb, bar);
        else
          bulk_g2s(tile + slot(0, c) * ROW, a.Fprev + gcell(s0, p) * ROW, unsigned(TSe) * rb, bar);
      }
    } else if (need_fl && lane >= 16 && lane < 16 + TP) {
      const int c = lane - 16;
      bulk_g2s(flb + c * TS * ROW, a.Fl + gcell(s0, p0 + c) * ROW, unsigned(TSe) * rb, bar);
    }
  }
  for (int x = tid; x < Q0; x += NT) {
    p0r[x] = F32 ? real(m.p0f[x]) : real(m.p0[x]);
    iw0[x] = F32 ? real(m.iw0f[x]) : real(m.iw0[x]);
    w0r[x] = F32 ? real(m.w0f[x]) : real(m.w0[x]);
  }
  for (int x = tid; x < Q1; x += NT) {
    p1r[x] = F32 ? real(m.p1f[x]) : real(m.p1[x]);
    iw1[x] = F32 ? real(m.iw1f[x]) : real(m.iw1[x]);
    w1r[x] = F32 ? real(m.w1f[x]) : real(m.w1[x]);
  }
  for (int x = tid; x < Q0 * MAXN; x += NT) tb0[x] = F32 ? real(m.tab0f[x]) : real(m.tab0[x]);
  for (int x = tid; x < Q1 * MAXN; x += NT) tb1[x] = F32 ? real(m.tab1f[x]) : real(m.tab1[x]);
  for (int x = tid; x < NC * 10; x += NT) {
    const int q = x / 10, k = x - q * 10, c = q / TS, sr = q - c * TS;
    real v = 0;
    if (sr < TSe) {
      if constexpr (F32) v = (&a.geof[gcell(s0 + sr, p0 + c)].am)[k];
      else v = (&a.geo[gcell(s0 + sr, p0 + c)].am)[k];
    }
    geo[x] = v;
  }
  bool ok = mbar_wait(bar, 0, a.max_polls);
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
    mbar_wait(bar, 0, a.max_polls);
    return;
  }
  const real T0 = F32 ? real(a.cd.T0f) : real(a.cd.T0);

  // ==== phase A: moments per owned cell (warp per cell) and the lambda-axis contractions
  for (int q = warp; q < NC; q += NW) {
    const int c = q / TS, sr = q - c * TS;
    if (sr >= TSe) continue;
    const real* F = tile + slot(sr, c) * ROW;
    real sn = 0, sr0 = 0, sp1 = 0, se = 0;
    for (int v = lane; v < V; v += 32) {
      const int i = v / Q1, j = v - i * Q1;
      const pair_t<real> f = p_load(F + 2 * v);
      const real f1 = f.x, f2 = f.y, pl = p0r[i], px = p1r[j];
      sn += f1;
      sr0 += pl * f1;
      sp1 += px * f1;
      se += (pl * pl + px * px) * f1 + f2;
    }
    const bool h16 = lane & 16, h8 = lane & 8;
    double k0 = h16 ? double(sp1) : double(sn), k1 = h16 ? double(se) : double(sr0);
    const double t0 = h16 ? double(sn) : double(sp1), t1 = h16 ? double(sr0) : double(se);
    k0 += __shfl_xor_sync(0xffffffffu, t0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, t1, 16);
    double kq = h8 ? k1 : k0;
    kq += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    kq += __shfl_xor_sync(0xffffffffu, kq, 4);
    kq += __shfl_xor_sync(0xffffffffu, kq, 2);
    kq += __shfl_xor_sync(0xffffffffu, kq, 1);
    const double d0 = __shfl_sync(0xffffffffu, kq, 8), d1 = __shfl_sync(0xffffffffu, kq, 16);
    const double de = __shfl_sync(0xffffffffu, kq, 24);
    if (lane == 0) {  // sums of D plus those of R
      const real nn = real(kq + m.ref_n), u0 = real(d0 + m.ref_r) / nn, u1 = real(d1 + m.ref_p) / nn;
      const real T = (real(de + m.ref_e) - nn * (u0 * u0 + u1 * u1)) / (real(3) * nn);
      cn[q] = nn;
      cnd[q] = kq + (F32 ? m.ref_sum_f : m.ref_n);
      cu0[q] = u0;
      cu1[q] = u1;
      cT[q] = T;
      citau[q] = nn * T / (F32 ? real(a.cd.knf) : real(a.cd.kn));  // tau = Kn / (n T), Eq. (canalie_tau)
    }
  }
  // lbuf = G_lxx (p^xi)^2 K^l f + G_lxl p^xi K~^l f (task: owned cell, field, column j)
  for (int x = tid; x < NC * 2 * Q1; x += NT) {
    const int j = x % Q1, qd = x / Q1, d = qd & 1, q = qd >> 1;
    const int c = q / TS, sr = q - c * TS;
    if (sr >= TSe) continue;
    const real* F = tile + slot(sr, c) * ROW + d;
    real col[Q0];
#pragma unroll
    for (int ip = 0; ip < Q0; ++ip) col[ip] = F[2 * (ip * Q1 + j)];
    const real px = p1r[j];
    const real wa = geo[q * 10 + 9] * px * px, wb = geo[q * 10 + 8] * px;
    real* Lr = lbuf + q * ROW + d;
#pragma unroll
    for (int i = 0; i < Q0; ++i) {
      real s1 = 0, s2 = 0;
#pragma unroll
      for (int ip = 0; ip < Q0; ++ip) {
        s1 += kk.K0[i * Q0 + ip] * col[ip];
        s2 += kk.Kt0[i * Q0 + ip] * col[ip];
      }
      Lr[2 * (i * Q1 + j)] = wa * s1 + wb * s2;
    }
  }
  __syncthreads();

  // ==== phase B: equilibrium moment vectors and the xi-axis contractions
  for (int x = tid; x < NC * 4; x += NT) {
    const int q = x >> 2, ax = (x >> 1) & 1, side = x & 1;
    const int c = q / TS, sr = q - c * TS;
    if (sr >= TSe) continue;
    const real u = (ax ? cu1[q] : cu0[q]) * (side ? real(-1) : real(1));
    eq_moment_vector<real>(ax ? m.kind1 : m.kind0, ax ? m.N1 : m.N0, u, cT[q], mv + (q * 4 + ax * 2 + side) * MAXN);
  }
  // lbuf -= G_lxx p^l K~^xi f + G_lxl (p^l)^2 K^xi f (task: owned cell, field, row i)
  for (int x = tid; x < NC * 2 * Q0; x += NT) {
    const int i = x % Q0, qd = x / Q0, d = qd & 1, q = qd >> 1;
    const int c = q / TS, sr = q - c * TS;
    if (sr >= TSe) continue;
    const real* F = tile + slot(sr, c) * ROW + d + 2 * i * Q1;
    real rw[Q1];
#pragma unroll
    for (int jp = 0; jp < Q1; ++jp) rw[jp] = F[2 * jp];
    const real pl = p0r[i];
    const real wa = geo[q * 10 + 9] * pl, wb = geo[q * 10 + 8] * pl * pl;
    real* Lr = lbuf + q * ROW + d + 2 * i * Q1;
#pragma unroll
    for (int j = 0; j < Q1; ++j) {
      real s1 = 0, s2 = 0;
#pragma unroll
      for (int jp = 0; jp < Q1; ++jp) {
        s1 += kk.Kt1[j * Q1 + jp] * rw[jp];
        s2 += kk.K1[j * Q1 + jp] * rw[jp];
      }
      Lr[2 * j] -= wa * s1 + wb * s2;
    }
  }
  // equilibrium factors of the walls and reservoirs: g_lambda(0, T0), g_xi(0, T0)
  if (tid == 0) {
    real ml[MAXN], mx[MAXN];
    eq_moment_vector<real>(m.kind0, m.N0, real(0), T0, ml);
    eq_moment_vector<real>(m.kind1, m.N1, real(0), T0, mx);
    for (int k = 0; k < Q0; ++k) {
      real g = 0;
      for (int s = 0; s <= m.N0; ++s) g += tb0[k * MAXN + s] * ml[s];
      gw0[k] = g;
    }
    for (int k = 0; k < Q1; ++k) {
      real g = 0;
      for (int s = 0; s <= m.N1; ++s) g += tb1[k * MAXN + s] * mx[s];
      gw1[k] = g;
    }
  }
  __syncthreads();

  // ==== phase C: equilibrium factors per cell and the boundaries
  for (int x = tid; x < NC * (Q0 + Q1); x += NT) {
    const int q = x / (Q0 + Q1);
    int k = x - q * (Q0 + Q1);
    const int c = q / TS, sr = q - c * TS;
    if (sr >= TSe) continue;
    if (k < Q0) {
      const int side = (m.kind0 == 1 && p0r[k] < real(0)) ? 1 : 0;
      const real* mm = mv + (q * 4 + side) * MAXN;
      real g = 0;
      for (int s = 0; s <= m.N0; ++s) g += tb0[k * MAXN + s] * mm[s];
      g0n[q * Q0 + k] = cn[q] * g;
    } else {
      k -= Q0;
      const int side = (m.kind1 == 1 && p1r[k] < real(0)) ? 1 : 0;
      const real* mm = mv + (q * 4 + 2 + side) * MAXN;
      real g = 0;
      for (int s = 0; s <= m.N1; ++s) g += tb1[k * MAXN + s] * mm[s];
      g1[q * Q1 + k] = g;
    }
  }
  __syncthreads();
  if (tid < NC && tid % TS < TSe) normalise_equilibrium<real>(g0n + tid * Q0, g1 + tid * Q1, Q0, Q1, cnd[tid]);
  // centreline lambda = 0: specular reflection, ghost 1-k mirrors cell k (p^lambda -> -p^lambda)
  if (s0 < 3) {  // the lambda halo reaches the ghost cells s = -1, -2, -3 (s = -k mirrors cell k - 1)
    constexpr int QH = Q0 / 2;
    for (int x = tid; x < TP * 3 * V; x += NT) {
      const int v = x % V, kc = x / V, k = kc % 3 + 1, c = kc / 3;
      const int i = v / Q1, j = v - i * Q1;
      const int ib = i < QH ? i + QH : i - QH;
      const int rg = -k - s0, rc = k - 1 - s0;  // tile rows of the ghost and of its mirror cell
      if (rg >= -3) p_store(tile + slot(rg, c) * ROW + 2 * v, p_load(tile + slot(rc, c) * ROW + 2 * (ib * Q1 + j)));
    }
  }
  // wall lambda = 1: per column, outgoing flux (p^lambda > 0), n_w, incoming ghosts f_eq(n_w, 0, T0)
  if (s0 + TS + 3 > nl) {
    const int sA = nl - 1 - s0;  // row of the wall-adjacent cell, relative to s0
    double part[TP];
#pragma unroll
    for (int c = 0; c < TP; ++c) part[c] = 0;
    for (int x = tid; x < TP * V; x += NT) {
      const int c = x / V, v = x - c * V, i = v / Q1, j = v - i * Q1;
      if (!(p0r[i] > real(0))) continue;
      // field 0 (f'), with the reconstruction phase D applies
      const real F0 = tile[slot(sA, c) * ROW + 2 * v], F1 = tile[slot(sA - 1, c) * ROW + 2 * v];
      const real F2 = tile[slot(sA - 2, c) * ROW + 2 * v];
      const real G0 = real(3) * F0 - real(3) * F1 + F2, G1 = real(6) * F0 - real(8) * F1 + real(3) * F2;
      const double fl = double(weno5<real>(F2, F1, F0, G0, G1, iw0[i] * iw1[j])) * double(p0r[i]);
#pragma unroll
      for (int cc = 0; cc < TP; ++cc)
        if (cc == c) part[cc] += fl;
    }
#pragma unroll
    for (int c = 0; c < TP; ++c) {
      const double s = warp_sum<real>(part[c]);
      if (lane == 0) red[NW * 4 + c * NW + warp] = s;
    }
    __syncthreads();
    if (tid < TP) {
      double s = m.ref_flux_pos;  // the outgoing flux of R
      for (int w = 0; w < NW; ++w) s += red[NW * 4 + tid * NW + w];
      double den0 = 0, den1 = 0;  // incoming flux of f_eq(1, 0, T0): sum_{p^l<0} g p^l * sum_j g
      for (int k = 0; k < Q0; ++k)
        if (p0r[k] < real(0)) den0 += double(gw0[k]) * double(p0r[k]);
      for (int k = 0; k < Q1; ++k) den1 += double(gw1[k]);
      const double nwc = -s / (den0 * den1);
      nwv[tid] = nwc;
      a.nw[p0 + tid] = nwc;
      if (!isfinite(nwc)) atomicOr(a.err, ERR_NONFINITE);
    }
    __syncthreads();
    for (int x = tid; x < TP * V; x += NT) {
      const int v = x % V, c = x / V;
      const int i = v / Q1, j = v - i * Q1;
      pair_t<real> g1v, g2v, g3v;
      if (p0r[i] > real(0)) {
        const pair_t<real> F0 = p_load(tile + slot(sA, c) * ROW + 2 * v);
        const pair_t<real> F1 = p_load(tile + slot(sA - 1, c) * ROW + 2 * v);
        const pair_t<real> F2 = p_load(tile + slot(sA - 2, c) * ROW + 2 * v);
        g1v = p_make(real(3) * F0.x - real(3) * F1.x + F2.x, real(3) * F0.y - real(3) * F1.y + F2.y);
        g2v = p_make(real(6) * F0.x - real(8) * F1.x + real(3) * F2.x, real(6) * F0.y - real(8) * F1.y + real(3) * F2.y);
        g3v = g2v;
      } else {  // f_eq(n_w, 0, T0) - R
        const double e = nwv[c] * double(gw0[i]) * double(gw1[j]), r = m.w0[i] * m.w1[j];
        g1v = g2v = g3v = p_make(real(e - r), real(e * double(T0) - r));
      }
      if (sA + 1 < TS + 3) p_store(tile + slot(sA + 1, c) * ROW + 2 * v, g1v);
      if (sA + 2 < TS + 3) p_store(tile + slot(sA + 2, c) * ROW + 2 * v, g2v);
      if (sA + 3 < TS + 3) p_store(tile + slot(sA + 3, c) * ROW + 2 * v, g3v);
    }
  }
  // inlet and outlet reservoirs: per row, u^xi of the adjacent cell, then ghosts
  for (int end = 0; end < 2; ++end) {
    const bool active = end == 0 ? (p0 < 3) : (p0 + TP + 3 > nx);
    if (!active) continue;
    const int cA = end == 0 ? -p0 : nx - 1 - p0;  // tile column of the adjacent cell
    real* gres = end == 0 ? gin : gout;
    real* ures = end == 0 ? uin : uout;
    __syncthreads();
    for (int sr = warp; sr < TSe; sr += NW) {
      const real* F = tile + slot(sr, cA) * ROW;
      real sn = 0, sx = 0;
      for (int v = lane; v < V; v += 32) {
        const int j = v % Q1;
        sn += F[2 * v];
        sx += p1r[j] * F[2 * v];
      }
      const double dn = warp_sum<real>(double(sn)) + m.ref_n, dx = warp_sum<real>(double(sx)) + m.ref_p;
      if (lane == 0) ures[sr] = real(dx / dn);
    }
    __syncthreads();
    for (int sr = tid; sr < TSe; sr += NT) {
      real mx[MAXN], mxm[MAXN];
      eq_moment_vector<real>(m.kind1, m.N1, ures[sr], T0, mx);
      eq_moment_vector<real>(m.kind1, m.N1, -ures[sr], T0, mxm);
      for (int k = 0; k < Q1; ++k) {
        const real* mm = (m.kind1 == 1 && p1r[k] < real(0)) ? mxm : mx;
        real g = 0;
        for (int s = 0; s <= m.N1; ++s) g += tb1[k * MAXN + s] * mm[s];
        gres[sr * Q1 + k] = g;
      }
    }
    __syncthreads();
    const real nres = F32 ? real(end == 0 ? a.cd.n_inf : a.cd.n_outf) : real(end == 0 ? a.cd.n_in : a.cd.n_out);
    for (int x = tid; x < TSe * V; x += NT) {
      const int v = x % V, sr = x / V;
      const int i = v / Q1, j = v - i * Q1;
      // V^xi at the boundary interface of the adjacent cell
      real bb, cc;
      if constexpr (F32) {
        const ChanCell<float>& gc = a.geof[gcell(s0 + sr, p0 + cA)];
        bb = end == 0 ? gc.bm : gc.bp;
        cc = end == 0 ? gc.cm : gc.cp;
      } else {
        const ChanCell<double>& gc = a.geo[gcell(s0 + sr, p0 + cA)];
        bb = end == 0 ? gc.bm : gc.bp;
        cc = end == 0 ? gc.cm : gc.cp;
      }
      const real Vx = bb * p1r[j] - cc * p0r[i];
      const bool inflow = end == 0 ? (Vx > real(0)) : (Vx < real(0));
      pair_t<real> val;
      if (inflow) {  // f_eq(n_res, (0, u_res), T0) - R
        const real e = nres * gw0[i] * gres[sr * Q1 + j], r = w0r[i] * w1r[j];
        val = p_make(e - r, e * T0 - r);
      } else {
        val = p_load(tile + slot(sr, cA) * ROW + 2 * v);
      }
      for (int k = 1; k <= 3; ++k) {
        const int c = end == 0 ? cA - k : cA + k;
        if (c >= -3 && c < TP + 3 && (c < 0 || c >= TP)) p_store(tile + slot(sr, c) * ROW + 2 * v, val);
      }
    }
  }
  __syncthreads();

  // ==== phase D: WENO-5 in lambda (walking each column) and in xi, flux differences, BGK, RK3
  const real dtr = F32 ? real(a.cd.dtf) : real(a.cd.dt);
  const real ca = F32 ? real(a.caf) : real(a.ca);  // cb = 1 - ca: see StageArgs
  const real ccoef = (F32 ? real(a.ccf) : real(a.cc)) * dtr;
  for (int x = tid; x < 2 * V; x += NT) {
    const int d = x >= V, v = x - d * V;
    const int i = v / Q1, j = v - i * Q1;
    const real pl = p0r[i], px = p1r[j];
    const bool upl = pl >= real(0);
    const real sc = iw0[i] * iw1[j];
#pragma unroll
    for (int c = 0; c < TP; ++c) {
      const real* S = tile + slot(0, c) * ROW + 2 * v + d;  // row sr at S[sr * ROW]
      real w0 = S[-3 * ROW], w1 = S[-2 * ROW], w2 = S[-1 * ROW], w3 = S[0], w4 = S[ROW], w5 = S[2 * ROW];
      real fm = weno5<real>(upl ? w0 : w5, upl ? w1 : w4, upl ? w2 : w3, upl ? w3 : w2, upl ? w4 : w1, sc);
#pragma unroll
      for (int sr = 0; sr < TS; ++sr) {
        if (sr < TSe) {
          const int q = c * TS + sr;
          const real w6 = S[(sr + 3) * ROW];
          const real fp = weno5<real>(upl ? w1 : w6, upl ? w2 : w5, upl ? w3 : w4, upl ? w4 : w3, upl ? w5 : w2, sc);
          const real* gq = geo + q * 10;
          real adv = pl * (gq[1] * fp - gq[0] * fm) * gq[6];
          real h[7];
#pragma unroll
          for (int k = 0; k < 7; ++k) h[k] = tile[slot(sr, c - 3 + k) * ROW + 2 * v + d];
          const real Vm = gq[2] * px - gq[4] * pl, Vp_ = gq[3] * px - gq[5] * pl;
          const real Fm = Vm >= real(0) ? weno5<real>(h[0], h[1], h[2], h[3], h[4], sc)
                                        : weno5<real>(h[5], h[4], h[3], h[2], h[1], sc);
          const real Fp = Vp_ >= real(0) ? weno5<real>(h[1], h[2], h[3], h[4], h[5], sc)
                                         : weno5<real>(h[6], h[5], h[4], h[3], h[2], sc);
          adv += (Vp_ * Fp - Vm * Fm) * gq[7];
          const real deq = g0n[q * Q0 + i] * g1[q * Q1 + j] * (d ? cT[q] : real(1)) - w0r[i] * w1r[j];
          const real Lv = -adv + lbuf[q * ROW + 2 * v + d] - (w3 - deq) * citau[q];
          real o = w3 + ccoef * Lv;
          real* dst = flb + q * ROW + 2 * v + d;
          if (need_fl) o += ca * (*dst - w3);
          *dst = o;
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
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid < TP) {
    bulk_s2g(a.Fout + gcell(s0, p0 + tid) * ROW, flb + tid * TS * ROW, unsigned(TSe * ROW * sizeof(real)));
    bulk_commit_and_wait_read();
  }
}

}  // namespace vlb
