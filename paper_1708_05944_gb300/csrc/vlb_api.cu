// C ABI of libvlb (declared in include/vlb.h): contexts, buffers, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "vlb_ctx.h"


namespace {

thread_local std::string g_err;

vlb_status fail(vlb_ctx* c, vlb_status s, const std::string& msg) {
  if (c) c->err = msg;
  g_err = msg;
  return s;
}

vlb_status cuda_fail(vlb_ctx* c, cudaError_t e, const char* where) {
  return fail(c, VLB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define VLB_CUDA(c, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

bool valid_model(const vlb_model* m, std::string* why) {
  for (int a = 0; a < 2; ++a) {
    if (m->kind[a] != VLB_FULL && m->kind[a] != VLB_HALF) {
      *why = "quadrature kind must be VLB_FULL or VLB_HALF";
      return false;
    }
    if (m->Q[a] < 1 || m->N[a] < 0 || m->N[a] >= m->Q[a]) {
      *why = "each axis needs 0 <= N < Q (Eq. norder_limit)";
      return false;
    }
  }
  return true;
}

int axis_nodes(const vlb_model* m, int a) { return m->kind[a] == VLB_HALF ? 2 * m->Q[a] : m->Q[a]; }

// geometry of one Couette instance: chi-formulation factors per cell
void couette_geometry(const vlb_couette_grid& g, GeoCell* out) {
  const int n = g.n_cells;
  std::vector<double> Rf(n + 1), Rc(n), wres(n);
  const double L = g.r_out - g.r_in;
  if (g.stretch_A == 0.0) {
    for (int s = 0; s <= n; ++s) Rf[s] = g.r_in + L * s / n;
    for (int s = 0; s < n; ++s) {
      Rc[s] = g.r_in + (s + 0.5) / n * L;
      wres[s] = Rc[s] * L / n;
    }
  } else {
    const double A = g.stretch_A, dl = g.stretch_delta;
    const double A0 = dl > 1.0 - dl ? dl : 1.0 - dl;
    const double e_in = -atanh(A * dl / A0), e_out = atanh(A * (1.0 - dl) / A0);
    const double de = (e_out - e_in) / n;
    auto R = [&](double eta) { return g.r_in + L * (dl + A0 / A * tanh(eta)); };
    for (int s = 0; s <= n; ++s) Rf[s] = R(e_in + s * de);
    Rf[0] = g.r_in;
    Rf[n] = g.r_out;
    for (int s = 0; s < n; ++s) {
      const double ec = e_in + (s + 0.5) * de;
      Rc[s] = R(ec);
      wres[s] = A0 / A * L * Rc[s] * de / (cosh(ec) * cosh(ec));
    }
  }
  for (int s = 0; s < n; ++s) {
    const double rp = Rf[s + 1], rm = Rf[s];
    const double den = (rp - rm) * (rp + rm);
    out[s].cp = 2.0 * rp / den;
    out[s].cm = 2.0 * rm / den;
    out[s].inv_rbar = 2.0 / (rp + rm);
    out[s].wres = wres[s];
  }
}

// K J = sgn J K for the reflection J of an axis (KArgs), to rounding, and the
// nodes mirror each other: the fixed-shape kernels rely on both.
bool force_reflection_symmetric(const std::vector<double>& p, const std::vector<double>& K, int kind, int nq,
                                double sgn) {
  double kmax = 0.0, pmax = 0.0;
  for (double x : K) kmax = std::max(kmax, std::fabs(x));
  for (double x : p) pmax = std::max(pmax, std::fabs(x));
  for (int a = 0; a < nq; ++a) {
    if (std::fabs(p[refl(kind, nq, a)] + p[a]) > 1e-13 * pmax) return false;
    for (int b = 0; b < nq; ++b)
      if (std::fabs(K[refl(kind, nq, a) * nq + refl(kind, nq, b)] - sgn * K[a * nq + b]) > 1e-12 * kmax) return false;
  }
  return true;
}

// The force kernels in the form the stage kernels of this shape read (KArgs):
// full matrices, or the half-size blocks P, M of their even and odd parts.
template <typename real>
void fill_force_tables(KArgs<real>& k, const std::vector<double>& K0, const std::vector<double>& Kt1, int kind0,
                       int kind1, int nq0, int nq1, bool split) {
  memset(&k, 0, sizeof(k));
  if (!split) {
    for (int i = 0; i < nq0; ++i)
      for (int ip = 0; ip < nq0; ++ip) k.full.K0[i * MAXQ + ip] = real(K0[i * nq0 + ip]);
    for (int j = 0; j < nq1; ++j)
      for (int jp = 0; jp < nq1; ++jp) k.full.Kt1[j * MAXQ + jp] = real(Kt1[j * nq1 + jp]);
    return;
  }
  constexpr int HQ = KArgs<real>::HQ;
  // single precision: every coefficient duplicated (KArgs::SplitPairs)
  const bool paired = sizeof(real) == 4;
  for (int i = 0; i < nq0 / 2; ++i)
    for (int c = 0; c < nq0 / 2; ++c) {
      const double a = K0[i * nq0 + c], b = K0[i * nq0 + refl(kind0, nq0, c)];
      if (paired) {
        k.pairs.P0[i * HQ + c].x = k.pairs.P0[i * HQ + c].y = real(0.5 * (a + b));
        k.pairs.M0[i * HQ + c].x = k.pairs.M0[i * HQ + c].y = real(0.5 * (a - b));
      } else {
        k.split.P0[i * HQ + c] = real(0.5 * (a + b));
        k.split.M0[i * HQ + c] = real(0.5 * (a - b));
      }
    }
  for (int j = 0; j < nq1 / 2; ++j)
    for (int c = 0; c < nq1 / 2; ++c) {
      const double a = Kt1[j * nq1 + c], b = Kt1[j * nq1 + refl(kind1, nq1, c)];
      if (paired) {
        k.pairs.P1[j * HQ + c].x = k.pairs.P1[j * HQ + c].y = real(0.5 * (a + b));
        k.pairs.M1[j * HQ + c].x = k.pairs.M1[j * HQ + c].y = real(0.5 * (a - b));
      } else {
        k.split.P1[j * HQ + c] = real(0.5 * (a + b));
        k.split.M1[j * HQ + c] = real(0.5 * (a - b));
      }
    }
}

}  // namespace

cudaError_t stage_launch_config(vlb_ctx* c, int n_tiles, int* nbuf, int* grid) {
  const int v = c->variant;
  if (c->ftilde && c->ft_fused) {  // the f~ kernel of launch shape 0 (plain or persistent)
    if (c->cfg_ft_nbuf[v] == 0) {
      int nb = 1, per_sm = 0;
      const cudaError_t e = c->prec == VLB_FP64
                                ? stage_config<double>(c->variants[v], c->margs, c->Vp, &nb, &per_sm, true)
                                : stage_config<float>(c->variants[v], c->margs, c->Vp, &nb, &per_sm, true);
      if (e != cudaSuccess) return e;
      c->cfg_ft_nbuf[v] = nb;
      c->cfg_ft_per_sm[v] = per_sm;
    }
    *nbuf = c->cfg_ft_nbuf[v];
    const int cap = c->cfg_ft_per_sm[v] * c->sms;
    *grid = c->variants[v].persist && cap > 0 && cap < n_tiles ? cap : n_tiles;
    return cudaSuccess;
  }
  if (c->cfg_nbuf[v] == 0) {  // first use of this launch shape
    cudaError_t e;
    if (c->sms == 0) {
      int dev = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    }
    int nb = 1, per_sm = 0;
    e = c->prec == VLB_FP64 ? stage_config<double>(c->variants[v], c->margs, c->Vp, &nb, &per_sm)
                            : stage_config<float>(c->variants[v], c->margs, c->Vp, &nb, &per_sm);
    if (e != cudaSuccess) return e;
    c->cfg_nbuf[v] = nb;
    c->cfg_per_sm[v] = per_sm;
  }
  *nbuf = c->cfg_nbuf[v];
  const int cap = c->cfg_per_sm[v] * c->sms;  // persistent: as many CTAs as are resident at once
  *grid = c->variants[v].persist && cap > 0 && cap < n_tiles ? cap : n_tiles;
  return cudaSuccess;
}

namespace {

// Tiles over every instance for the current launch shape.  One-CTA-per-tile
// launches take tiles of the shape's full size TC.  A persistent launch walks
// the tile list in rounds of `slots` CTAs, so the tile size s <= TC is chosen to
// minimise rounds x (s + 3): the makespan in cell-times with the three halo
// cells as the fixed cost of a tile (for 5 x 1024 cells on 456 CTAs: 6-cell
// tiles in two rounds instead of 8-cell tiles in two).  CTA b takes the tiles
// b, b + slots, ...; when the last round is not full, the tiles that reach a
// wall (and so also fill its ghost cells, several times the work of an interior
// tile's phase in between) are placed in the first round of the CTAs that have
// no tile in the last round.
void build_tiles(vlb_ctx* c) {
  const StageVariant& v = c->variants[c->variant];
  int s = v.tc;
  int slots = 0;
  if (v.persist) {
    int nbuf = 1;
    if (stage_launch_config(c, 1 << 30, &nbuf, &slots) != cudaSuccess) slots = 0;
    if (slots > 0) {
      long long best = -1;
      for (int cand = v.tc; cand >= std::max(3, (v.tc + 1) / 2); --cand) {
        long long count = 0;
        for (int i = 0; i < c->n_inst; ++i) count += (c->inst[i].n_cells + cand - 1) / cand;
        const long long cost = ((count + slots - 1) / slots) * (cand + 3);
        if (best < 0 || cost < best) best = cost, s = cand;
      }
    }
  }
  c->tiles.clear();
  for (int i = 0; i < c->n_inst; ++i)
    for (int c0 = 0; c0 < c->inst[i].n_cells; c0 += s)
      c->tiles.push_back(TileDesc{i, c0, std::min(s, c->inst[i].n_cells - c0)});
  const int T = int(c->tiles.size());
  if (slots <= 0 || T <= slots || T % slots == 0) return;
  const int full = T - (T - 1) / slots * slots;  // CTAs 0 .. full-1 take a tile in the last round
  std::vector<TileDesc> wall, rest;
  for (const TileDesc& t : c->tiles) {
    const int n = c->inst[t.inst].n_cells;
    (t.c0 < 3 || t.c0 + t.nc + 3 > n ? wall : rest).push_back(t);
  }
  std::vector<TileDesc> out(T);
  std::vector<char> used(T, 0);
  size_t w = 0, r = 0;
  for (int b = full; b < slots && w < wall.size(); ++b) out[b] = wall[w++], used[b] = 1;
  for (int p = 0; p < T; ++p)
    if (!used[p]) out[p] = w < wall.size() ? wall[w++] : rest[r++];
  c->tiles.swap(out);
}

template <typename real>
vlb_status do_stage(vlb_ctx* c, int k, int prev, int out) {
  StageArgs<real> a{};
  a.Fprev = static_cast<const real*>(c->F[prev]);
  a.Fl = static_cast<const real*>(c->F[c->cur]);
  a.Fout = static_cast<real*>(c->F[out]);
  if (k == 1) {
    a.ca = 0.0, a.cb = 1.0, a.cc = 1.0;
  } else if (k == 2) {
    a.ca = 0.75, a.cb = 0.25, a.cc = 0.25;
  } else {
    a.ca = 1.0 / 3.0, a.cb = 2.0 / 3.0, a.cc = 2.0 / 3.0;
  }
  a.caf = float(a.ca), a.cbf = float(a.cb), a.ccf = float(a.cc);
  a.geof = c->d_geof;
  a.inst = c->d_inst;
  a.tiles = c->d_tiles;
  a.n_tiles = int(c->tiles.size());
  a.geo = c->d_geo;
  a.nw = c->d_nw;
  a.wall = c->d_wall;
  a.halo = static_cast<const real*>(c->d_halo);
  a.err = c->d_err;
  a.Vp = c->Vp;
  a.max_polls = 1ull << 26;
  const bool ft = c->ftilde && c->ft_fused;
  if (ft) {
    a.geo = c->d_ftgeo;
    a.geof = c->d_ftgeof;
    a.sqrtg = static_cast<const real*>(c->d_ftsg);
    a.forceR = static_cast<const real*>(c->d_ftfr);
  }
  const KArgs<real>* kk;
  if constexpr (sizeof(real) == 4) kk = c->k32.get(); else kk = c->k64.get();
  int grid = 0;
  cudaError_t e = stage_launch_config(c, a.n_tiles, &a.nbuf, &grid);
  if (e == cudaSuccess) e = launch_stage<real>(c->variants[c->variant], a, c->margs, *kk, grid, c->stream, ft);
  if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel launch");
  c->launches += 1;
  return VLB_OK;
}

template <typename real>
vlb_status do_clb_stage(vlb_ctx* c, int k, int prev, int out) {
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cc[3] = {1.0, 0.25, 2.0 / 3.0};
  ClbGeom g = c->clbg;
  g.kn = c->cdesc.kn, g.n_in = c->cdesc.n_in, g.n_out = c->cdesc.n_out, g.T0 = c->cdesc.T0;
  cudaError_t e = clb_stage<real>(c->lm, g, static_cast<const real*>(c->F[prev]), static_cast<const real*>(c->F[c->cur]),
                                  static_cast<real*>(c->F[out]), static_cast<real*>(c->d_clbrec),
                                  static_cast<real*>(c->d_clbres), c->d_nw, c->inst[0].dt, ca[k - 1], cc[k - 1],
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "Cartesian-split stage launch");
  c->launches += 3;
  return VLB_OK;
}

template <typename real>
vlb_status do_large_stage(vlb_ctx* c, int k, int prev, int out) {
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cc[3] = {1.0, 0.25, 2.0 / 3.0};
  cudaError_t e = lm_stage<real>(c->lm, static_cast<const real*>(c->F[prev]), static_cast<const real*>(c->F[c->cur]),
                                 static_cast<real*>(c->F[out]), c->total_cells, c->d_inst, c->n_inst, c->d_geo,
                                 c->d_lwall, c->d_nw, static_cast<real*>(c->d_lrec), static_cast<real*>(c->d_lforce),
                                 c->d_lpart, ca[k - 1], cc[k - 1], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "large-set stage launch");
  c->launches += 5;
  return VLB_OK;
}

// Model tables of a large velocity set in device memory (LargeModel), from the axis tables.
vlb_status setup_large(vlb_ctx* c) {
  const AxisTables &a0 = c->ax[0], &a1 = c->ax[1];
  const int nq0 = c->nq0, nq1 = c->nq1;
  std::vector<double> d;
  auto put = [&](const std::vector<double>& v) { size_t o = d.size(); d.insert(d.end(), v.begin(), v.end()); return o; };
  std::vector<double> iw0(nq0), iw1(nq1), t0(size_t(nq0) * MAXN, 0.0), t1(size_t(nq1) * MAXN, 0.0);
  for (int k = 0; k < nq0; ++k) iw0[k] = 1.0 / a0.w[k];
  for (int k = 0; k < nq1; ++k) iw1[k] = 1.0 / a1.w[k];
  for (int k = 0; k < nq0; ++k)
    for (int s2 = 0; s2 <= a0.N; ++s2) t0[size_t(k) * MAXN + s2] = a0.eqtab[size_t(k) * (a0.N + 1) + s2];
  for (int k = 0; k < nq1; ++k)
    for (int s2 = 0; s2 <= a1.N; ++s2) t1[size_t(k) * MAXN + s2] = a1.eqtab[size_t(k) * (a1.N + 1) + s2];
  const size_t op0 = put(a0.p), op1 = put(a1.p), ow0 = put(a0.w), ow1 = put(a1.w), oi0 = put(iw0), oi1 = put(iw1);
  const size_t ot0 = put(t0), ot1 = put(t1), oK = put(a0.K), oKt = put(a1.Kt);
  // single precision: sqrt(w_k' / w_k) K and the scale vectors (see LargeModel)
  std::vector<float> f;
  for (int k = 0; k < nq0; ++k)
    for (int kp = 0; kp < nq0; ++kp) f.push_back(float(a0.K[size_t(k) * nq0 + kp] * std::sqrt(a0.w[kp] / a0.w[k])));
  const size_t ofKt = f.size();
  for (int k = 0; k < nq1; ++k)
    for (int kp = 0; kp < nq1; ++kp) f.push_back(float(a1.Kt[size_t(k) * nq1 + kp] * std::sqrt(a1.w[kp] / a1.w[k])));
  const size_t os0 = f.size();
  for (int k = 0; k < nq0; ++k) f.push_back(float(std::sqrt(a0.w[k])));
  const size_t ois0 = f.size();
  for (int k = 0; k < nq0; ++k) f.push_back(float(std::min(1.0 / std::sqrt(a0.w[k]), 1e30)));
  const size_t os1 = f.size();
  for (int k = 0; k < nq1; ++k) f.push_back(float(std::sqrt(a1.w[k])));
  const size_t ois1 = f.size();
  for (int k = 0; k < nq1; ++k) f.push_back(float(std::min(1.0 / std::sqrt(a1.w[k]), 1e30)));
  const size_t dbytes = d.size() * sizeof(double);
  VLB_CUDA(c, cudaMalloc(&c->d_lm, dbytes + f.size() * sizeof(float)));
  VLB_CUDA(c, cudaMemcpy(c->d_lm, d.data(), dbytes, cudaMemcpyHostToDevice));
  VLB_CUDA(c, cudaMemcpy(static_cast<char*>(c->d_lm) + dbytes, f.data(), f.size() * sizeof(float),
                         cudaMemcpyHostToDevice));
  const double* D = static_cast<const double*>(c->d_lm);
  const float* Fp = reinterpret_cast<const float*>(static_cast<const char*>(c->d_lm) + dbytes);
  LargeModel& m = c->lm;
  m.nq0 = nq0, m.nq1 = nq1, m.V = c->V, m.Vp = c->Vp, m.N0 = a0.N, m.N1 = a1.N, m.kind0 = a0.kind, m.kind1 = a1.kind;
  m.p0 = D + op0, m.p1 = D + op1, m.w0 = D + ow0, m.w1 = D + ow1, m.iw0 = D + oi0, m.iw1 = D + oi1;
  m.tab0 = D + ot0, m.tab1 = D + ot1, m.K0 = D + oK, m.Kt1 = D + oKt, m.K0f = Fp, m.Kt1f = Fp + ofKt;
  m.s0f = Fp + os0, m.is0f = Fp + ois0, m.s1f = Fp + os1, m.is1f = Fp + ois1;
  double sw1 = 0, pos = 0, neg = 0;
  for (int k = 0; k < nq1; ++k) sw1 += a1.w[k];
  for (int k = 0; k < nq0; ++k) {
    if (a0.p[k] > 0.0) pos += a0.p[k] * a0.w[k];
    if (a0.p[k] < 0.0) neg += a0.p[k] * a0.w[k];
  }
  m.ref_flux_pos = pos * sw1;
  m.ref_flux_neg = neg * sw1;
  return VLB_OK;
}

// Rows per lambda segment and segments of a channel launch shape.  A fixed ts
// is used as given (at least 3 rows per segment, the last one included); ts = 0
// picks the segment count that minimises waves x (rows + 6) over the SMs of the
// device, one resident CTA each: the 6 rows are the warm-up of a segment (window
// rows below it and the equilibria of its first three rows).
void channel_segments(const vlb_ctx* c, const ChanVariant& v, int* seglen, int* nseg) {
  const int nl = c->cdesc.nl, nstrips = c->cdesc.nx / v.tp;
  auto count = [&](int L) {  // segments of L rows, 0 if the last would be shorter than 3
    const int n = (nl + L - 1) / L;
    return nl - (n - 1) * L >= 3 ? n : 0;
  };
  if (v.ts > 0) {
    int L = std::max(3, std::min(v.ts, nl));
    int n = count(L);
    if (n == 0) L = nl, n = 1;
    *seglen = L, *nseg = n;
    return;
  }
  const int sms = c->sms > 0 ? c->sms : 1;
  long long best = -1;
  *seglen = nl, *nseg = 1;
  for (int want = 1; want <= nl / 3; ++want) {
    const int L = (nl + want - 1) / want;
    const int n = count(L);
    if (n == 0) continue;
    const long long waves = (static_cast<long long>(nstrips) * n + sms - 1) / sms;
    const long long cost = waves * (L + 6);
    if (best < 0 || cost < best) best = cost, *seglen = L, *nseg = n;
  }
}

template <typename real>
vlb_status do_chan_stage(vlb_ctx* c, int k, int prev, int out, bool clb = false) {
  ChanArgs<real> a{};
  a.Fprev = static_cast<const real*>(c->F[prev]);
  a.Fl = static_cast<const real*>(c->F[c->cur]);
  a.Fout = static_cast<real*>(c->F[out]);
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cc[3] = {1.0, 0.25, 2.0 / 3.0};
  a.ca = real(ca[k - 1]);
  a.ccdt = real(cc[k - 1] * c->inst[0].dt);
  a.tables = c->d_ctab;
  if constexpr (sizeof(real) == 8) a.geo = clb ? c->d_clbcgeo : c->d_cgeo;
  else a.geo = clb ? c->d_clbcgeof : c->d_cgeof;
  a.nw = c->d_nw;
  a.err = c->d_err;
  a.nl = c->cdesc.nl;
  a.nx = c->cdesc.nx;
  a.ikn = real(1.0 / c->cdesc.kn);
  a.n_in = real(c->cdesc.n_in);
  a.n_out = real(c->cdesc.n_out);
  a.T0 = real(c->cdesc.T0);
  a.max_polls = 1ull << 26;
  a.flow = c->cdesc.flow;
  a.qflow = static_cast<const real*>(c->d_qflow);
  const ChanVariant& v = c->cvariants[c->variant];
  channel_segments(c, v, &a.seglen, &a.nseg);
  const int grid = (a.nx / v.tp) * a.nseg;
  cudaError_t e = launch_channel<real>(v, a, c->chan_kp.data(), c->nq0, c->nq1, grid, c->stream, clb);
  if (e != cudaSuccess) return cuda_fail(c, e, "channel stage kernel launch");
  c->launches += 1;
  return VLB_OK;
}

// Rebuild the channel's table block (it carries f_eq(1, 0, T0)) and upload it
// on the context stream.
vlb_status upload_channel_tables(vlb_ctx* c) {
  std::vector<unsigned char> tb;
  const bool ok = c->prec == VLB_FP64 ? channel_tables<double>(c->nq0, c->nq1, c->ax, c->margs, c->cdesc.T0, &tb)
                                      : channel_tables<float>(c->nq0, c->nq1, c->ax, c->margs, c->cdesc.T0, &tb);
  if (!ok) return fail(c, VLB_ERR_UNSUPPORTED, "no channel kernel for this velocity set");
  if (!c->d_ctab) {
    VLB_CUDA(c, cudaMalloc(&c->d_ctab, tb.size()));
    c->ctab_bytes = tb.size();
  }
  if (tb.size() != c->ctab_bytes) return fail(c, VLB_ERR_STATE, "channel table size changed");
  VLB_CUDA(c, cudaMemcpyAsync(c->d_ctab, tb.data(), tb.size(), cudaMemcpyHostToDevice, c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return VLB_OK;
}

vlb_status run_stage(vlb_ctx* c, int k) {
  // buffers: cur = F_l; stage 1 -> (cur+1); stage 2 reads (cur+1) -> (cur+2); stage 3 reads (cur+2) -> (cur+1)
  const int b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
  int prev, out;
  if (k == 1) {
    prev = c->cur, out = b1;
  } else if (k == 2) {
    prev = b1, out = b2;
  } else {
    prev = b2, out = b1;
  }
  vlb_status st;
  if (c->kind == 1 && c->clb && c->clb_march)
    st = c->prec == VLB_FP64 ? do_chan_stage<double>(c, k, prev, out, true) : do_chan_stage<float>(c, k, prev, out, true);
  else if (c->kind == 1 && c->clb)
    st = c->prec == VLB_FP64 ? do_clb_stage<double>(c, k, prev, out) : do_clb_stage<float>(c, k, prev, out);
  else if (c->kind == 1 && c->n_cvariants == 0)
    return fail(c, VLB_ERR_UNSUPPORTED, "no vielbein channel kernel for this velocity set (16x12 or 8x4 nodes): "
                                        "it runs the Cartesian split (vlb_set_formulation)");
  else if (c->kind == 1)
    st = c->prec == VLB_FP64 ? do_chan_stage<double>(c, k, prev, out) : do_chan_stage<float>(c, k, prev, out);
  else if (c->large || (c->ftilde && !c->ft_fused))
    st = c->prec == VLB_FP64 ? do_large_stage<double>(c, k, prev, out) : do_large_stage<float>(c, k, prev, out);
  else
    st = c->prec == VLB_FP64 ? do_stage<double>(c, k, prev, out) : do_stage<float>(c, k, prev, out);
  if (st != VLB_OK) return st;
  if (c->collision == 1) {  // Shakhov: the heat-flux term of F_prev, added to the BGK stage's output
    const double ccw[3] = {1.0, 0.25, 2.0 / 3.0};
    const double knf = c->kind == 1 ? c->cdesc.kn : -1.0;
    const cudaError_t e =
        c->prec == VLB_FP64
            ? launch_shakhov<double>(static_cast<double*>(c->F[out]), static_cast<const double*>(c->F[prev]),
                                     c->total_cells, c->Vp, c->margs, c->d_inst, c->n_inst, ccw[k - 1],
                                     1.0 - c->prandtl, knf, c->stream)
            : launch_shakhov<float>(static_cast<float*>(c->F[out]), static_cast<const float*>(c->F[prev]),
                                    c->total_cells, c->Vp, c->margs, c->d_inst, c->n_inst, ccw[k - 1],
                                    1.0 - c->prandtl, knf, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "Shakhov correction launch");
    c->launches += 1;
  }
  c->last = out;
  c->stage_done = k;
  if (k == 3) {
    c->cur = out;
    c->steps += 1;
  }
  return VLB_OK;
}

vlb_status check_err(vlb_ctx* c) {
  unsigned h = 0;
  VLB_CUDA(c, cudaMemcpyAsync(&h, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h & ERR_TIMEOUT) return fail(c, VLB_ERR_TIMEOUT, "a bounded device wait ran out");
  if (h & ERR_NONFINITE) return fail(c, VLB_ERR_NONFINITE, "a wall density came out non-finite");
  return VLB_OK;
}

vlb_status compute_moments(vlb_ctx* c, double* dst) {
  if (c->large) {
    cudaError_t e = c->prec == VLB_FP64
                        ? lm_moments<double>(c->lm, static_cast<const double*>(c->F[c->last]), c->total_cells, dst,
                                             c->stream)
                        : lm_moments<float>(c->lm, static_cast<const float*>(c->F[c->last]), c->total_cells, dst,
                                            c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel launch");
    return VLB_OK;
  }
  cudaError_t e = c->prec == VLB_FP64
                      ? launch_moments<double>(static_cast<const double*>(c->F[c->last]), c->total_cells, c->Vp,
                                               c->margs, dst, c->stream, c->cmap)
                      : launch_moments<float>(static_cast<const float*>(c->F[c->last]), c->total_cells, c->Vp,
                                              c->margs, dst, c->stream, c->cmap);
  if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel launch");
  return VLB_OK;
}

// Weights in single precision and the sums of the rest state R_ij = w0_i w1_j
// that the kernels add back to the deviation sums (see ModelArgs).
void fill_reference(ModelArgs& m) {
  double s0 = 0, s1 = 0, sp0 = 0, sp1 = 0, sq0 = 0, sq1 = 0, sf0 = 0, sf1 = 0, pos = 0, neg = 0;
  for (int k = 0; k < m.nq0; ++k) {
    m.w0f[k] = float(m.w0[k]);
    s0 += m.w0[k];
    sp0 += m.p0[k] * m.w0[k];
    sq0 += m.p0[k] * m.p0[k] * m.w0[k];
    sf0 += double(m.w0f[k]);
    if (m.p0[k] > 0.0) pos += m.p0[k] * m.w0[k];
    if (m.p0[k] < 0.0) neg += m.p0[k] * m.w0[k];
  }
  for (int k = 0; k < m.nq1; ++k) {
    m.w1f[k] = float(m.w1[k]);
    s1 += m.w1[k];
    sp1 += m.p1[k] * m.w1[k];
    sq1 += m.p1[k] * m.p1[k] * m.w1[k];
    sf1 += double(m.w1f[k]);
  }
  m.ref_n = s0 * s1;
  m.ref_r = sp0 * s1;
  m.ref_p = s0 * sp1;
  m.ref_e = sq0 * s1 + s0 * sq1 + s0 * s1;
  m.ref_sum_f = sf0 * sf1;
  m.ref_flux_pos = pos * s1;
  m.ref_flux_neg = neg * s1;
  m.ref_nf[0] = float(m.ref_n);
  m.ref_nf[1] = float(m.ref_n - double(m.ref_nf[0]));
  m.ref_sumf[0] = float(m.ref_sum_f);
  m.ref_sumf[1] = float(m.ref_sum_f - double(m.ref_sumf[0]));
  m.ref_rf = float(m.ref_r);
  m.ref_pf = float(m.ref_p);
  m.ref_ef = float(m.ref_e);
}

// Moment vector of the truncated equilibrium on one axis (the same recurrences as
// eq_moment_vector in the kernels), on the host in double.
void host_moment_vector(int kind, int N, double u, double T, double* m) {
  if (kind == 0) {
    m[0] = 1.0;
    if (N >= 1) m[1] = u;
    for (int l = 2; l <= N; ++l) m[l] = (u * m[l - 1] + (T - 1.0) * m[l - 2]) / double(l);
    return;
  }
  const double pi = 3.14159265358979323846;
  const double g0 = std::exp(-u * u / (2.0 * T)) / std::sqrt(2.0 * pi * T);
  m[0] = 0.5 * (1.0 + std::erf(u / std::sqrt(2.0 * T)));
  if (N >= 1) m[1] = u * m[0] + T * g0;
  for (int s = 2; s <= N; ++s) m[s] = u * m[s - 1] + double(s - 1) * T * m[s - 2];
}

// Wall equilibria f_eq(1, (0, u_w), T_w) of every Couette instance (inner, outer):
// factors per axis and incoming flux, into c->walls (host) for upload to d_wall.
void fill_walls(vlb_ctx* c, std::vector<WallEq>& out) {
  const ModelArgs& m = c->margs;
  out.assign(size_t(2) * c->n_inst, WallEq{});
  for (int i = 0; i < c->n_inst; ++i)
    for (int w = 0; w < 2; ++w) {
      WallEq& e = out[size_t(2) * i + w];
      const double uw = w == 0 ? c->inst[i].u_in : c->inst[i].u_out;
      const double Tw = w == 0 ? c->inst[i].T_in : c->inst[i].T_out;
      double mp[MAXN], mm[MAXN];
      host_moment_vector(m.kind0, m.N0, 0.0, Tw, mp);
      for (int k = 0; k < m.nq0; ++k) {
        double g = 0;
        for (int s = 0; s <= m.N0; ++s) g += m.tab0[k * MAXN + s] * mp[s];  // u = 0: both sides alike
        e.g0[k] = g;
      }
      host_moment_vector(m.kind1, m.N1, uw, Tw, mp);
      host_moment_vector(m.kind1, m.N1, -uw, Tw, mm);
      for (int k = 0; k < m.nq1; ++k) {
        const double* v = (m.kind1 == 1 && m.p1[k] < 0.0) ? mm : mp;
        double g = 0;
        for (int s = 0; s <= m.N1; ++s) g += m.tab1[k * MAXN + s] * v[s];
        e.g1[k] = g;
      }
      const double sgn = w == 0 ? 1.0 : -1.0;  // incoming half: p^R > 0 at the inner wall
      double s0 = 0, s1 = 0;
      for (int k = 0; k < m.nq0; ++k)
        if (sgn * m.p0[k] > 0.0) s0 += e.g0[k] * m.p0[k];
      for (int k = 0; k < m.nq1; ++k) s1 += e.g1[k];
      e.in_flux = s0 * s1;
    }
}

vlb_status upload_walls(vlb_ctx* c) {
  if (c->d_lwall) {  // the multi-kernel path: per (instance, wall) g0, g1, in_flux, T_w from the axis tables
    const int nq0 = c->nq0, nq1 = c->nq1, st = nq0 + nq1 + 2;
    const AxisTables &a0 = c->ax[0], &a1 = c->ax[1];
    std::vector<double> w(size_t(c->n_inst) * 2 * st);
    for (int i = 0; i < c->n_inst; ++i)
      for (int wl = 0; wl < 2; ++wl) {
        double* e = &w[(size_t(i) * 2 + wl) * st];
        const double uw = wl == 0 ? c->inst[i].u_in : c->inst[i].u_out;
        const double Tw = wl == 0 ? c->inst[i].T_in : c->inst[i].T_out;
        double mp[MAXN], mm[MAXN];
        host_moment_vector(a0.kind, a0.N, 0.0, Tw, mp);
        for (int k = 0; k < nq0; ++k) {
          double g = 0;
          for (int s2 = 0; s2 <= a0.N; ++s2) g += a0.eqtab[size_t(k) * (a0.N + 1) + s2] * mp[s2];
          e[k] = g;
        }
        host_moment_vector(a1.kind, a1.N, uw, Tw, mp);
        host_moment_vector(a1.kind, a1.N, -uw, Tw, mm);
        for (int k = 0; k < nq1; ++k) {
          const double* v = (a1.kind == 1 && a1.p[k] < 0.0) ? mm : mp;
          double g = 0;
          for (int s2 = 0; s2 <= a1.N; ++s2) g += a1.eqtab[size_t(k) * (a1.N + 1) + s2] * v[s2];
          e[nq0 + k] = g;
        }
        const double sgn = wl == 0 ? 1.0 : -1.0;
        double s0 = 0, s1 = 0;
        for (int k = 0; k < nq0; ++k)
          if (sgn * a0.p[k] > 0.0) s0 += e[k] * a0.p[k];
        for (int k = 0; k < nq1; ++k) s1 += e[nq0 + k];
        e[nq0 + nq1] = s0 * s1;
        e[nq0 + nq1 + 1] = Tw;
      }
    VLB_CUDA(c, cudaMemcpyAsync(c->d_lwall, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    VLB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->large) return VLB_OK;
  }
  std::vector<WallEq> w;
  fill_walls(c, w);
  VLB_CUDA(c, cudaMemcpyAsync(c->d_wall, w.data(), sizeof(WallEq) * w.size(), cudaMemcpyHostToDevice, c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return VLB_OK;
}

// The buffer that holds neither F_l nor the last result: free between calls.
int spare_buffer(const vlb_ctx* c) {
  for (int b = 0; b < 3; ++b)
    if (b != c->cur && b != c->last) return b;
  return -1;
}

// Caller layout F <-> device layout D = F - R (see launch_deviation).
vlb_status convert(vlb_ctx* c, const void* src, void* dst, int to_deviation) {
  if (c->large) {
    cudaError_t e = c->prec == VLB_FP64
                        ? lm_deviation<double>(c->lm, static_cast<const double*>(src), static_cast<double*>(dst),
                                               c->total_cells, to_deviation, c->stream)
                        : lm_deviation<float>(c->lm, static_cast<const float*>(src), static_cast<float*>(dst),
                                              c->total_cells, to_deviation, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "conversion kernel launch");
    return VLB_OK;
  }
  cudaError_t e = c->prec == VLB_FP64
                      ? launch_deviation<double>(static_cast<const double*>(src), static_cast<double*>(dst),
                                                 c->total_cells, c->Vp, c->margs, to_deviation, c->stream, c->cmap)
                      : launch_deviation<float>(static_cast<const float*>(src), static_cast<float*>(dst),
                                                c->total_cells, c->Vp, c->margs, to_deviation, c->stream, c->cmap);
  if (e != cudaSuccess) return cuda_fail(c, e, "conversion kernel launch");
  return VLB_OK;
}

}  // namespace

extern "C" {

vlb_status vlb_parse_model(const char* text, vlb_model* out) {
  if (!text || !out) return fail(nullptr, VLB_ERR_INVALID, "null argument");
  vlb_model m{};
  const char* s = text;
  for (int a = 0; a < 2; ++a) {
    while (*s == ' ') ++s;
    int kind;
    if (s[0] == 'H' && s[1] == 'H') {
      kind = VLB_HALF;
      s += 2;
    } else if (s[0] == 'H') {
      kind = VLB_FULL;
      s += 1;
    } else {
      return fail(nullptr, VLB_ERR_INVALID, "model component must start with H or HH");
    }
    int N, Q, used = 0;
    if (sscanf(s, "(%d;%d)%n", &N, &Q, &used) != 2 || used == 0)
      return fail(nullptr, VLB_ERR_INVALID, "expected (N;Q) after H or HH");
    s += used;
    m.kind[a] = kind;
    m.N[a] = N;
    m.Q[a] = Q;
    while (*s == ' ') ++s;
    if (a == 0) {
      if (*s == 'x' || *s == 'X') {
        ++s;
      } else if ((unsigned char)s[0] == 0xC3 && (unsigned char)s[1] == 0x97) {  // UTF-8 multiplication sign
        s += 2;
      } else {
        return fail(nullptr, VLB_ERR_INVALID, "expected 'x' between the two axes");
      }
    }
  }
  while (*s == ' ') ++s;
  if (*s) return fail(nullptr, VLB_ERR_INVALID, "trailing characters after the model");
  std::string why;
  if (!valid_model(&m, &why)) return fail(nullptr, VLB_ERR_INVALID, why);
  *out = m;
  return VLB_OK;
}

int vlb_axis_nodes(const vlb_model* m, int axis) {
  std::string why;
  if (!m || axis < 0 || axis > 1 || !valid_model(m, &why)) return VLB_ERR_INVALID;
  return axis_nodes(m, axis);
}

vlb_status vlb_axis_tables(const vlb_model* m, int axis, double* p, double* w, double* K, double* Kt) {
  std::string why;
  if (!m || axis < 0 || axis > 1) return fail(nullptr, VLB_ERR_INVALID, "bad axis");
  if (!valid_model(m, &why)) return fail(nullptr, VLB_ERR_INVALID, why);
  AxisTables t;
  if (!build_axis(m->kind[axis] == VLB_HALF ? 1 : 0, m->N[axis], m->Q[axis], &t, &why))
    return fail(nullptr, VLB_ERR_INVALID, why);
  const int nq = t.nq;
  for (int k = 0; k < nq; ++k) {
    if (p) p[k] = t.p[k];
    if (w) w[k] = t.w[k];
  }
  for (int k = 0; k < nq * nq; ++k) {
    if (K) K[k] = t.K[k];
    if (Kt) Kt[k] = t.Kt[k];
  }
  return VLB_OK;
}

vlb_status vlb_quadrature(const vlb_model* m, int axis, double* p, double* w) {
  if (!p || !w) return fail(nullptr, VLB_ERR_INVALID, "null output");
  return vlb_axis_tables(m, axis, p, w, nullptr, nullptr);
}

vlb_status vlb_create_couette(const vlb_model* model, vlb_precision prec, int n_inst,
                              const vlb_couette_grid* grids, const vlb_wall* inner, const vlb_wall* outer,
                              const double* kn, const int* tau_mode, void* cuda_stream, vlb_ctx** out) {
  if (!model || !grids || !inner || !outer || !kn || !tau_mode || !out || n_inst < 1)
    return fail(nullptr, VLB_ERR_INVALID, "null or empty argument");
  *out = nullptr;
  std::string why;
  if (!valid_model(model, &why)) return fail(nullptr, VLB_ERR_INVALID, why);
  if (prec != VLB_FP64 && prec != VLB_FP32_BULK) return fail(nullptr, VLB_ERR_INVALID, "bad precision");
  for (int i = 0; i < n_inst; ++i) {
    const vlb_couette_grid& g = grids[i];
    if (g.n_cells < 3) return fail(nullptr, VLB_ERR_INVALID, "a Couette instance needs at least 3 cells");
    if (!(g.cell_begin == 0 && g.cell_end == 0) &&
        !(g.cell_begin >= 0 && g.cell_end <= g.n_cells && g.cell_end - g.cell_begin >= 3))
      return fail(nullptr, VLB_ERR_INVALID, "a slab needs 0 <= cell_begin, cell_end <= n_cells and at least 3 cells");
    if (!(g.r_in > 0.0) || !(g.r_out > g.r_in)) return fail(nullptr, VLB_ERR_INVALID, "need 0 < r_in < r_out");
    if (!(g.stretch_A >= 0.0 && g.stretch_A < 1.0) || !(g.stretch_delta >= 0.0 && g.stretch_delta <= 1.0))
      return fail(nullptr, VLB_ERR_INVALID, "stretching needs 0 <= A < 1, 0 <= delta <= 1");
    if (!(kn[i] > 0.0)) return fail(nullptr, VLB_ERR_INVALID, "Kn must be positive");
    if (tau_mode[i] < 0 || tau_mode[i] > 2) return fail(nullptr, VLB_ERR_INVALID, "bad tau mode");
    if (!(inner[i].T > 0.0) || !(outer[i].T > 0.0)) return fail(nullptr, VLB_ERR_INVALID, "wall temperature must be > 0");
  }
  const int nq0 = axis_nodes(model, 0), nq1 = axis_nodes(model, 1);
  const bool large = nq0 > MAXQ || nq1 > MAXQ;  // beyond the fused kernels: the multi-kernel path
  if (large && (long long)nq0 * nq1 > 65536) return fail(nullptr, VLB_ERR_UNSUPPORTED, "more than 65536 velocities");
  if (large)
    for (int i = 0; i < n_inst; ++i)
      if (!(grids[i].cell_begin == 0 && grids[i].cell_end == 0) &&
          !(grids[i].cell_begin == 0 && grids[i].cell_end == grids[i].n_cells))
        return fail(nullptr, VLB_ERR_UNSUPPORTED, "slabs of large velocity sets are not built");
  if (model->N[0] + 1 > MAXN || model->N[1] + 1 > MAXN)
    return fail(nullptr, VLB_ERR_UNSUPPORTED, "expansion order above 7");

  std::unique_ptr<vlb_ctx> c(new vlb_ctx);
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(nullptr, VLB_ERR_CUDA, "cudaGetDevice failed");
  c->model = *model;
  c->prec = prec;
  c->n_inst = n_inst;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  for (int a = 0; a < 2; ++a)
    if (!build_axis(model->kind[a] == VLB_HALF ? 1 : 0, model->N[a], model->Q[a], &c->ax[a], &why))
      return fail(nullptr, VLB_ERR_INVALID, why);
  c->nq0 = nq0;
  c->nq1 = nq1;
  c->V = nq0 * nq1;
  c->Vp = (c->V + 3) / 4 * 4;
  c->esize = prec == VLB_FP64 ? 8 : 4;
  c->large = large;
  if (large) {
    c->variants[0] = StageVariant{1, 256, 0};  // one launch shape: the four kernels of vlb_large.cu
    c->n_variants = 1;
    vlb_status ls = setup_large(c.get());
    if (ls != VLB_OK) return ls;
  } else {
    StageVariant all[8];
    const int n = prec == VLB_FP64 ? stage_variants<double>(nq0, nq1, all) : stage_variants<float>(nq0, nq1, all);
    for (int i = 0; i < n; ++i) {
      const size_t smem = prec == VLB_FP64 ? stage_smem_bytes<double>(all[i], c->Vp)
                                           : stage_smem_bytes<float>(all[i], c->Vp);
      if (smem > 0 && smem <= 227 * 1024 && c->n_variants + 2 <= 16) {
        c->variants[c->n_variants++] = StageVariant{all[i].tc, all[i].nt, 0};
        c->variants[c->n_variants++] = StageVariant{all[i].tc, all[i].nt, 1};
      }
    }
    if (c->n_variants == 0) return fail(nullptr, VLB_ERR_UNSUPPORTED, "velocity set too large for one tile");
  }

  ModelArgs& m = c->margs;
  if (!large) {
  m.nq0 = nq0;
  m.nq1 = nq1;
  m.N0 = model->N[0];
  m.N1 = model->N[1];
  m.kind0 = model->kind[0] == VLB_HALF ? 1 : 0;
  m.kind1 = model->kind[1] == VLB_HALF ? 1 : 0;
  for (int k = 0; k < nq0; ++k) {
    m.p0[k] = c->ax[0].p[k];
    m.w0[k] = c->ax[0].w[k];
    m.iw0[k] = 1.0 / m.w0[k];
    m.p0f[k] = float(m.p0[k]);
    m.iw0f[k] = float(m.iw0[k]);
    for (int s = 0; s <= m.N0; ++s) {
      m.tab0[k * MAXN + s] = c->ax[0].eqtab[k * (m.N0 + 1) + s];
      m.tab0f[k * MAXN + s] = float(m.tab0[k * MAXN + s]);
    }
  }
  for (int k = 0; k < nq1; ++k) {
    m.p1[k] = c->ax[1].p[k];
    m.w1[k] = c->ax[1].w[k];
    m.iw1[k] = 1.0 / m.w1[k];
    m.p1f[k] = float(m.p1[k]);
    m.iw1f[k] = float(m.iw1[k]);
    for (int s = 0; s <= m.N1; ++s) {
      m.tab1[k * MAXN + s] = c->ax[1].eqtab[k * (m.N1 + 1) + s];
      m.tab1f[k * MAXN + s] = float(m.tab1[k * MAXN + s]);
    }
  }
  fill_reference(m);
  c->k32.reset(new KArgs<float>());
  c->k64.reset(new KArgs<double>());
  const bool split = prec == VLB_FP64 ? stage_split_tables<double>(nq0, nq1) : stage_split_tables<float>(nq0, nq1);
  if (split && !(force_reflection_symmetric(c->ax[0].p, c->ax[0].K, m.kind0, nq0, -1.0) &&
                 force_reflection_symmetric(c->ax[1].p, c->ax[1].Kt, m.kind1, nq1, 1.0)))
    return fail(nullptr, VLB_ERR_UNSUPPORTED, "force kernels are not reflection-symmetric");
  fill_force_tables(*c->k64, c->ax[0].K, c->ax[1].Kt, m.kind0, m.kind1, nq0, nq1, split);
  fill_force_tables(*c->k32, c->ax[0].K, c->ax[1].Kt, m.kind0, m.kind1, nq0, nq1, split);
  } else {
    m.nq0 = nq0, m.nq1 = nq1, m.N0 = model->N[0], m.N1 = model->N[1];
    m.kind0 = model->kind[0] == VLB_HALF ? 1 : 0;
    m.kind1 = model->kind[1] == VLB_HALF ? 1 : 0;
  }

  long long cell0 = 0;
  for (int i = 0; i < n_inst; ++i) {
    InstDesc d{};
    const vlb_couette_grid& g = grids[i];
    const bool slab = !(g.cell_begin == 0 && g.cell_end == 0);
    const int cb = slab ? g.cell_begin : 0, ce = slab ? g.cell_end : g.n_cells;
    d.cell0 = cell0;
    d.n_cells = ce - cb;
    d.halo = (cb > 0 ? 1 : 0) | (ce < g.n_cells ? 2 : 0);
    c->has_halo |= d.halo != 0;
    d.tau_mode = tau_mode[i];
    d.kn = kn[i];
    d.dt = 0.0;
    d.kn_f = float(kn[i]);
    d.dt_f = 0.0f;
    d.u_in = inner[i].u_tangential;
    d.T_in = inner[i].T;
    d.u_out = outer[i].u_tangential;
    d.T_out = outer[i].T;
    c->inst.push_back(d);
    c->grids.push_back(grids[i]);
    cell0 += d.n_cells;
  }
  c->total_cells = cell0;
  if (!large) build_tiles(c.get());
  c->geo.resize(cell0);
  for (int i = 0; i < n_inst; ++i) {  // a slab takes its cells' geometry from the whole grid
    std::vector<GeoCell> full(grids[i].n_cells);
    couette_geometry(grids[i], full.data());
    const int cb = grids[i].cell_begin == 0 && grids[i].cell_end == 0 ? 0 : grids[i].cell_begin;
    std::copy(full.begin() + cb, full.begin() + cb + c->inst[i].n_cells, c->geo.begin() + c->inst[i].cell0);
  }

  vlb_ctx* cp = c.get();
  const size_t fbytes = size_t(c->total_cells) * 2 * c->Vp * c->esize;
  for (int b = 0; b < 3; ++b) {
    VLB_CUDA(cp, cudaMalloc(&c->F[b], fbytes));
    VLB_CUDA(cp, cudaMemsetAsync(c->F[b], 0, fbytes, c->stream));
  }
  VLB_CUDA(cp, cudaMalloc(&c->d_inst, sizeof(InstDesc) * n_inst));
  // room for the tile list of any tile size (at most one tile per cell)
  c->tile_cap = size_t(c->total_cells);
  VLB_CUDA(cp, cudaMalloc(&c->d_tiles, sizeof(TileDesc) * c->tile_cap));
  VLB_CUDA(cp, cudaMalloc(&c->d_geo, sizeof(GeoCell) * c->total_cells));
  VLB_CUDA(cp, cudaMalloc(&c->d_geof, sizeof(GeoCellF) * c->total_cells));
  VLB_CUDA(cp, cudaMalloc(&c->d_nw, sizeof(double) * 2 * n_inst));
  VLB_CUDA(cp, cudaMalloc(&c->d_wall, sizeof(WallEq) * 2 * n_inst));
  VLB_CUDA(cp, cudaMalloc(&c->d_err, sizeof(unsigned)));
  VLB_CUDA(cp, cudaMalloc(&c->d_mom, sizeof(double) * 9 * c->total_cells));
  VLB_CUDA(cp, cudaMalloc(&c->d_prev, sizeof(double) * 9 * c->total_cells));
  VLB_CUDA(cp, cudaMalloc(&c->d_res, sizeof(double) * 3 * n_inst));
  VLB_CUDA(cp, cudaMalloc(&c->d_halo, size_t(n_inst) * 6 * 2 * c->Vp * c->esize));
  VLB_CUDA(cp, cudaMemsetAsync(c->d_halo, 0, size_t(n_inst) * 6 * 2 * c->Vp * c->esize, c->stream));
  VLB_CUDA(cp, cudaMemcpyAsync(c->d_inst, c->inst.data(), sizeof(InstDesc) * n_inst, cudaMemcpyHostToDevice, c->stream));
  if (large) {
    const size_t cells = size_t(c->total_cells), es = c->esize;
    VLB_CUDA(cp, cudaMalloc(&c->d_lrec, cells * (nq0 + nq1 + 2) * es));
    VLB_CUDA(cp, cudaMalloc(&c->d_lforce, lm_force_reals(c->lm, c->total_cells) * es));
    VLB_CUDA(cp, cudaMalloc(&c->d_lpart, lm_part_doubles(c->lm, c->total_cells, n_inst) * sizeof(double)));
    VLB_CUDA(cp, cudaMalloc(&c->d_lwall, size_t(n_inst) * 2 * (nq0 + nq1 + 2) * sizeof(double)));
    c->lm.err = c->d_err;
  }
  {
    vlb_status ws = upload_walls(cp);
    if (ws != VLB_OK) return ws;
  }
  VLB_CUDA(cp, cudaMemcpyAsync(c->d_tiles, c->tiles.data(), sizeof(TileDesc) * c->tiles.size(),
                               cudaMemcpyHostToDevice, c->stream));
  VLB_CUDA(cp, cudaMemcpyAsync(c->d_geo, c->geo.data(), sizeof(GeoCell) * c->total_cells, cudaMemcpyHostToDevice,
                               c->stream));
  {
    std::vector<GeoCellF> gf(c->total_cells);
    for (long long i = 0; i < c->total_cells; ++i)
      gf[i] = GeoCellF{float(c->geo[i].cp), float(c->geo[i].cm), float(c->geo[i].inv_rbar), 0.0f};
    VLB_CUDA(cp, cudaMemcpy(c->d_geof, gf.data(), sizeof(GeoCellF) * c->total_cells, cudaMemcpyHostToDevice));
  }
  VLB_CUDA(cp, cudaMemsetAsync(c->d_nw, 0, sizeof(double) * 2 * n_inst, c->stream));
  VLB_CUDA(cp, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
  VLB_CUDA(cp, cudaStreamSynchronize(c->stream));
  vlb_status st = vlb_init_equilibrium(cp, 1.0, 0.0, 0.0, 1.0);
  if (st != VLB_OK) return st;
  *out = c.release();
  return VLB_OK;
}

vlb_status vlb_create_channel(const vlb_model* model, vlb_precision prec, const vlb_channel_grid* grid, double kn,
                              double n_in, double n_out, double T0, void* cuda_stream, vlb_ctx** out) {
  if (!model || !grid || !out) return fail(nullptr, VLB_ERR_INVALID, "null argument");
  *out = nullptr;
  std::string why;
  if (!valid_model(model, &why)) return fail(nullptr, VLB_ERR_INVALID, why);
  if (prec != VLB_FP64 && prec != VLB_FP32_BULK) return fail(nullptr, VLB_ERR_INVALID, "bad precision");
  if (model->kind[0] != VLB_HALF) return fail(nullptr, VLB_ERR_INVALID, "the wall-normal axis must be half range");
  const int nl = grid->n_lambda, nx = grid->n_xi;
  if (nl < 3 || nx < 4) return fail(nullptr, VLB_ERR_INVALID, "need n_lambda >= 3 and n_xi >= 4");
  if (!(grid->xi_out > grid->xi_in) || !(grid->re_c > 0.0) || !(grid->stretch_A > 0.0 && grid->stretch_A < 1.0))
    return fail(nullptr, VLB_ERR_INVALID, "need xi_in < xi_out, re_c > 0, 0 < stretch_A < 1");
  if (!(kn > 0.0) || !(n_in > 0.0) || !(n_out > 0.0) || !(T0 > 0.0))
    return fail(nullptr, VLB_ERR_INVALID, "need Kn, reservoir densities and T0 positive");
  const int nq0 = axis_nodes(model, 0), nq1 = axis_nodes(model, 1);
  std::unique_ptr<vlb_ctx> c(new vlb_ctx);
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(nullptr, VLB_ERR_CUDA, "cudaGetDevice failed");
  c->kind = 1;
  c->model = *model;
  c->prec = prec;
  c->n_inst = 1;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail(nullptr, VLB_ERR_CUDA, "cannot query the device");
  }
  for (int a = 0; a < 2; ++a)
    if (!build_axis(model->kind[a] == VLB_HALF ? 1 : 0, model->N[a], model->Q[a], &c->ax[a], &why))
      return fail(nullptr, VLB_ERR_INVALID, why);
  c->nq0 = nq0;
  c->nq1 = nq1;
  c->V = nq0 * nq1;
  c->Vp = (c->V + 3) / 4 * 4;
  c->esize = prec == VLB_FP64 ? 8 : 4;
  {
    // launch shapes: shared memory within an SM's, whole strips of columns; the
    // single-precision CUDA-core force needs the split force block, the double-precision
    // kernel contracts on its own (its shapes are the tc = 0 ones)
    const bool kp_ok = channel_force_pairs(nq0, nq1, c->ax, &c->chan_kp);
    if (!kp_ok) c->chan_kp.assign(16384, 0);
    ChanVariant all[8];
    const int n = channel_variants(nq0, nq1, all);
    for (int i = 0; i < n; ++i) {
      const size_t sm = prec == VLB_FP64 ? channel_smem_bytes<double>(all[i], nq0, nq1)
                                         : channel_smem_bytes<float>(all[i], nq0, nq1);
      if (!(sm > 0 && sm <= 227 * 1024 && nx % all[i].tp == 0)) continue;
      if (prec == VLB_FP64 && all[i].tc) continue;
      if (prec == VLB_FP32_BULK && !all[i].tc && !kp_ok) continue;
      c->cvariants[c->n_cvariants++] = all[i];
    }
    // no vielbein kernel for this velocity set: the context can still run the Cartesian split
    if (c->n_cvariants == 0 && (nq0 > MAXQ || nq1 > MAXQ))
      return fail(nullptr, VLB_ERR_UNSUPPORTED, "more than 32 nodes on an axis of a channel velocity set");
  }
  ModelArgs& m = c->margs;
  m.nq0 = nq0, m.nq1 = nq1, m.N0 = model->N[0], m.N1 = model->N[1];
  m.kind0 = 1, m.kind1 = model->kind[1] == VLB_HALF ? 1 : 0;
  for (int ax = 0; ax < 2; ++ax) {
    const AxisTables& t = c->ax[ax];
    const int N = model->N[ax];
    for (int k = 0; k < t.nq; ++k) {
      (ax ? m.p1 : m.p0)[k] = t.p[k];
      (ax ? m.w1 : m.w0)[k] = t.w[k];
      (ax ? m.iw1 : m.iw0)[k] = 1.0 / t.w[k];
      (ax ? m.p1f : m.p0f)[k] = float(t.p[k]);
      (ax ? m.iw1f : m.iw0f)[k] = float(1.0 / t.w[k]);
      for (int s = 0; s <= N; ++s) {
        (ax ? m.tab1 : m.tab0)[k * MAXN + s] = t.eqtab[k * (N + 1) + s];
        (ax ? m.tab1f : m.tab0f)[k * MAXN + s] = float(t.eqtab[k * (N + 1) + s]);
      }
    }
  }
  fill_reference(m);
  // geometry (Sec. VII.A-B): lambda(eta) = tanh(eta) / A, eta equidistant; xi equidistant; H/2 = 1
  const double A = grid->stretch_A, ea = atanh(A), re = grid->re_c;
  auto phi = [&](double x) { return 0.5 * (tanh(2.0) - tanh(2.0 - 30.0 * x / re)); };
  auto dphi = [&](double x) { const double ch = cosh(2.0 - 30.0 * x / re); return 0.5 * (30.0 / re) / (ch * ch); };
  auto chi = [&](double x) { return (1.0 + tanh(2.0) / 2.0) * x + re / 60.0 * log(cosh(2.0 - 30.0 * x / re) / cosh(2.0)); };
  std::vector<double> lf(nl + 1), lc(nl), xf(nx + 1), xc(nx);
  for (int s = 0; s <= nl; ++s) lf[s] = tanh(double(s) / nl * ea) / A;
  lf[nl] = 1.0;
  for (int s = 0; s < nl; ++s) lc[s] = tanh((s + 0.5) / nl * ea) / A;
  const double L = grid->xi_out - grid->xi_in;
  for (int p = 0; p <= nx; ++p) xf[p] = grid->xi_in + L * p / nx;
  for (int p = 0; p < nx; ++p) xc[p] = grid->xi_in + L * (p + 0.5) / nx;
  std::vector<ChanCell<double>> gd(size_t(nl) * nx);
  std::vector<ChanCell<float>> gf(size_t(nl) * nx);
  for (int p = 0; p < nx; ++p) {
    const double ph = phi(xc[p]), dp = dphi(xc[p]);
    const double phm = phi(xf[p]), dpm = dphi(xf[p]), php = phi(xf[p + 1]), dpp = dphi(xf[p + 1]);
    const double dchi = chi(xf[p + 1]) - chi(xf[p]);
    for (int s = 0; s < nl; ++s) {
      ChanCell<double> g{};
      g.am = sqrt(1.0 + lf[s] * lf[s] * dp * dp) / (1.0 + ph);
      g.ap = sqrt(1.0 + lf[s + 1] * lf[s + 1] * dp * dp) / (1.0 + ph);
      const double rm = sqrt(1.0 + lc[s] * lc[s] * dpm * dpm), rp = sqrt(1.0 + lc[s] * lc[s] * dpp * dpp);
      g.bm = (1.0 + phm) / rm;
      g.bp = (1.0 + php) / rp;
      g.cm = lc[s] * dpm * (1.0 + phm) / rm;
      g.cp = lc[s] * dpp * (1.0 + php) / rp;
      const double dl = lf[s + 1] - lf[s];
      g.idl = 1.0 / dl;
      g.idx = 1.0 / dchi;
      g.glxl = (g.bp - g.bm) / dchi;
      g.glxx = -(g.ap - g.am) / dl + (g.cp - g.cm) / dchi;
      gd[size_t(s) * nx + p] = g;  // device cell order: s * n_xi + p
      const double* src = &g.am;
      float* dst = &gf[size_t(s) * nx + p].am;
      for (int k = 0; k < 12; ++k) dst[k] = float(src[k]);
    }
  }
  c->cmap.nl = nl;
  c->cmap.nx = nx;
  c->chan_lc = lc;
  c->chan_grid = *grid;
  c->chan_phi_end[0] = phi(xf[0]);
  c->chan_phi_end[1] = phi(xf[nx]);
  ChanDesc& cd = c->cdesc;
  cd.nl = nl, cd.nx = nx, cd.kn = kn, cd.n_in = n_in, cd.n_out = n_out, cd.T0 = T0, cd.dt = 0.0;
  cd.knf = float(kn), cd.n_inf = float(n_in), cd.n_outf = float(n_out), cd.T0f = float(T0), cd.dtf = 0.0f;
  InstDesc d{};
  d.cell0 = 0;
  d.n_cells = nl * nx;
  d.kn = kn;
  d.kn_f = float(kn);
  c->inst.push_back(d);
  c->total_cells = (long long)nl * nx;
  vlb_ctx* cp = c.get();
  const size_t fbytes = size_t(c->total_cells) * 2 * c->Vp * c->esize;
  for (int b = 0; b < 3; ++b) {
    VLB_CUDA(cp, cudaMalloc(&c->F[b], fbytes));
    VLB_CUDA(cp, cudaMemsetAsync(c->F[b], 0, fbytes, c->stream));
  }
  VLB_CUDA(cp, cudaMalloc(&c->d_inst, sizeof(InstDesc)));
  VLB_CUDA(cp, cudaMalloc(&c->d_nw, sizeof(double) * nx));
  VLB_CUDA(cp, cudaMalloc(&c->d_err, sizeof(unsigned)));
  VLB_CUDA(cp, cudaMalloc(&c->d_mom, sizeof(double) * 9 * c->total_cells));
  VLB_CUDA(cp, cudaMalloc(&c->d_cgeo, sizeof(ChanCell<double>) * gd.size()));
  VLB_CUDA(cp, cudaMalloc(&c->d_cgeof, sizeof(ChanCell<float>) * gf.size()));
  VLB_CUDA(cp, cudaMemcpy(c->d_inst, c->inst.data(), sizeof(InstDesc), cudaMemcpyHostToDevice));
  VLB_CUDA(cp, cudaMemcpy(c->d_cgeo, gd.data(), sizeof(ChanCell<double>) * gd.size(), cudaMemcpyHostToDevice));
  VLB_CUDA(cp, cudaMemcpy(c->d_cgeof, gf.data(), sizeof(ChanCell<float>) * gf.size(), cudaMemcpyHostToDevice));
  VLB_CUDA(cp, cudaMemsetAsync(c->d_nw, 0, sizeof(double) * nx, c->stream));
  VLB_CUDA(cp, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
  {  // geometry of the post-processing (vlb_channel_postprocess)
    std::vector<double> pg;
    pg.insert(pg.end(), lc.begin(), lc.end());
    pg.insert(pg.end(), lf.begin(), lf.end());
    for (int p = 0; p < nx; ++p) pg.push_back(phi(xc[p]));
    for (int p = 0; p < nx; ++p) pg.push_back(dphi(xc[p]));
    c->chan_dxi = L / nx;
    VLB_CUDA(cp, cudaMalloc(&c->d_cpost, pg.size() * sizeof(double)));
    VLB_CUDA(cp, cudaMemcpy(c->d_cpost, pg.data(), pg.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  VLB_CUDA(cp, cudaStreamSynchronize(c->stream));
  if (c->n_cvariants > 0) {
    vlb_status ts = upload_channel_tables(cp);
    if (ts != VLB_OK) return ts;
  }
  vlb_status st = vlb_init_equilibrium(cp, 1.0, 0.0, 0.0, T0);
  if (st != VLB_OK) return st;
  *out = c.release();
  return VLB_OK;
}

vlb_status vlb_sizes(const vlb_ctx* c, long long* total_cells, int* nvel, long long* f_bytes) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (total_cells) *total_cells = c->total_cells;
  if (nvel) *nvel = c->V;
  if (f_bytes) *f_bytes = c->total_cells * 2LL * c->V * (long long)c->esize;
  return VLB_OK;
}

vlb_status vlb_set_walls(vlb_ctx* c, const vlb_wall* inner, const vlb_wall* outer) {
  if (!c || !inner || !outer) return fail(c, VLB_ERR_INVALID, "null argument");
  if (c->kind != 0) return fail(c, VLB_ERR_UNSUPPORTED, "walls are set at creation for the channel");
  for (int i = 0; i < c->n_inst; ++i) {
    if (!(inner[i].T > 0.0) || !(outer[i].T > 0.0)) return fail(c, VLB_ERR_INVALID, "wall temperature must be > 0");
    c->inst[i].u_in = inner[i].u_tangential;
    c->inst[i].T_in = inner[i].T;
    c->inst[i].u_out = outer[i].u_tangential;
    c->inst[i].T_out = outer[i].T;
  }
  VLB_CUDA(c, cudaMemcpyAsync(c->d_inst, c->inst.data(), sizeof(InstDesc) * c->n_inst, cudaMemcpyHostToDevice,
                              c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return upload_walls(c);
}

// Channel launches take their descriptor (dt, Kn, reservoirs) by value, so a
// captured three-step graph holds the values of its capture: drop the graphs
// whenever one of them changes (Couette instances read theirs from device
// memory and keep their graphs).
static vlb_status drop_channel_graphs(vlb_ctx* c) {
  if (c->kind != 1) return VLB_OK;
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int b = 0; b < 3; ++b) {
    if (c->graph_exec[b]) cudaGraphExecDestroy(c->graph_exec[b]);
    c->graph_exec[b] = nullptr;
    c->graph_variant[b] = -1;
  }
  return VLB_OK;
}

vlb_status vlb_set_knudsen(vlb_ctx* c, double kn, int tau_mode) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (!(kn > 0.0) || !std::isfinite(kn)) return fail(c, VLB_ERR_INVALID, "Kn must be finite and > 0");
  if (tau_mode < VLB_TAU_KN_OVER_NT || tau_mode > VLB_TAU_KN_OVER_N)
    return fail(c, VLB_ERR_INVALID, "unknown relaxation-time convention");
  if (c->kind == 1) {
    if (tau_mode != VLB_TAU_KN_OVER_NT)
      return fail(c, VLB_ERR_UNSUPPORTED, "the channel relaxes with tau = Kn / (n T)");
    c->cdesc.kn = kn;
    c->cdesc.knf = float(kn);
    return drop_channel_graphs(c);
  }
  for (int i = 0; i < c->n_inst; ++i) {
    c->inst[i].kn = kn;
    c->inst[i].kn_f = float(kn);
    c->inst[i].tau_mode = tau_mode;
  }
  VLB_CUDA(c, cudaMemcpyAsync(c->d_inst, c->inst.data(), sizeof(InstDesc) * c->n_inst, cudaMemcpyHostToDevice,
                              c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return VLB_OK;
}

static vlb_status upload_clb_weq(vlb_ctx* c);

vlb_status vlb_set_channel_reservoirs(vlb_ctx* c, double n_in, double n_out, double T0) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->kind != 1) return fail(c, VLB_ERR_UNSUPPORTED, "reservoirs belong to channel contexts");
  if (!(n_in > 0.0) || !(n_out > 0.0) || !(T0 > 0.0) || !std::isfinite(n_in) || !std::isfinite(n_out) ||
      !std::isfinite(T0))
    return fail(c, VLB_ERR_INVALID, "reservoir densities and temperature must be finite and > 0");
  c->cdesc.n_in = n_in, c->cdesc.n_inf = float(n_in);
  c->cdesc.n_out = n_out, c->cdesc.n_outf = float(n_out);
  c->cdesc.T0 = T0, c->cdesc.T0f = float(T0);
  c->cdesc.flow = 0;
  vlb_status st = drop_channel_graphs(c);
  if (st != VLB_OK) return st;
  if (c->clb && !c->clb_march) {
    st = upload_clb_weq(c);
    if (st != VLB_OK) return st;
  }
  return c->n_cvariants > 0 ? upload_channel_tables(c) : VLB_OK;
}

// The resources of the multi-kernel Couette path (vlb_large.cu) for a context created on the
// fused path (the f~ formulation runs there for any velocity set).
static vlb_status ensure_multi_path(vlb_ctx* c) {
  if (!c->d_lm) {
    vlb_status st = setup_large(c);
    if (st != VLB_OK) return st;
  }
  const size_t cells = size_t(c->total_cells), es = c->esize;
  if (!c->d_lrec) VLB_CUDA(c, cudaMalloc(&c->d_lrec, cells * (c->nq0 + c->nq1 + 2) * es));
  if (!c->d_lforce) VLB_CUDA(c, cudaMalloc(&c->d_lforce, lm_force_reals(c->lm, c->total_cells) * es));
  if (!c->d_lpart) VLB_CUDA(c, cudaMalloc(&c->d_lpart, lm_part_doubles(c->lm, c->total_cells, c->n_inst) * sizeof(double)));
  if (!c->d_lwall) {
    VLB_CUDA(c, cudaMalloc(&c->d_lwall, size_t(c->n_inst) * 2 * (c->nq0 + c->nq1 + 2) * sizeof(double)));
    vlb_status st = upload_walls(c);
    if (st != VLB_OK) return st;
  }
  c->lm.err = c->d_err;
  return VLB_OK;
}

// the wall equilibrium factors f_eq(1, 0, T0) of the Cartesian-split channel (host tables)
static vlb_status upload_clb_weq(vlb_ctx* c) {
  const AxisTables &a0 = c->ax[0], &a1 = c->ax[1];
  std::vector<double> w(size_t(c->nq0) + c->nq1);
  double mp[MAXN];
  host_moment_vector(a0.kind, a0.N, 0.0, c->cdesc.T0, mp);
  for (int k = 0; k < c->nq0; ++k) {
    double g = 0;
    for (int s2 = 0; s2 <= a0.N; ++s2) g += a0.eqtab[size_t(k) * (a0.N + 1) + s2] * mp[s2];
    w[k] = g;
  }
  host_moment_vector(a1.kind, a1.N, 0.0, c->cdesc.T0, mp);
  for (int k = 0; k < c->nq1; ++k) {
    double g = 0;
    for (int s2 = 0; s2 <= a1.N; ++s2) g += a1.eqtab[size_t(k) * (a1.N + 1) + s2] * mp[s2];
    w[c->nq0 + k] = g;
  }
  VLB_CUDA(c, cudaMemcpy(const_cast<double*>(c->clbg.weq), w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  return VLB_OK;
}

// Channel contexts: VLB_CHI (the vielbein stage) or VLB_CARTESIAN (Sec. VII.G)
static vlb_status set_channel_formulation(vlb_ctx* c, int formulation) {
  if (formulation == 1) return fail(c, VLB_ERR_UNSUPPORTED, "the f~ formulation is built for Couette contexts");
  if (formulation == 0 && c->n_cvariants == 0)
    return fail(c, VLB_ERR_UNSUPPORTED, "no vielbein channel kernel for this velocity set (16x12 or 8x4 nodes)");
  if (formulation == 2 && c->cdesc.flow) return fail(c, VLB_ERR_STATE, "the Cartesian split runs with reservoir ends");
  vlb_status st = drop_channel_graphs(c);
  if (st != VLB_OK) return st;
  const vlb_channel_grid& cg = c->chan_grid;
  auto cphi = [&](double x) { return 0.5 * (tanh(2.0) - tanh(2.0 - 30.0 * x / cg.re_c)); };
  auto cdphi = [&](double x) {
    const double ch = cosh(2.0 - 30.0 * x / cg.re_c);
    return 0.5 * (30.0 / cg.re_c) / (ch * ch);
  };
  auto cchi = [&](double x) {
    return (1.0 + tanh(2.0) / 2.0) * x + cg.re_c / 60.0 * log(cosh(2.0 - 30.0 * x / cg.re_c) / cosh(2.0));
  };
  if (formulation == 2 && c->n_cvariants > 0 && !c->d_clbcgeo) {
    // the marching kernel's records: V^lambda = a (p^x - lambda phi' p^y) at the row faces, a = 1 / (1 + phi)
    // at the column centre; V^xi = (1 + phi) p^y at the column faces (Sec. VII.G)
    const int nl = cg.n_lambda, nx = cg.n_xi;
    const double A = cg.stretch_A, ea = atanh(A), L = cg.xi_out - cg.xi_in;
    std::vector<double> lf(nl + 1);
    for (int s2 = 0; s2 <= nl; ++s2) lf[s2] = s2 == nl ? 1.0 : tanh(double(s2) / nl * ea) / A;
    std::vector<ChanCell<double>> gd(size_t(nl) * nx);
    std::vector<ChanCell<float>> gf(size_t(nl) * nx);
    for (int p = 0; p < nx; ++p) {
      const double xc = cg.xi_in + L * (p + 0.5) / nx, xm = cg.xi_in + L * p / nx, xp = cg.xi_in + L * (p + 1) / nx;
      const double a = 1.0 / (1.0 + cphi(xc)), dph = cdphi(xc);
      for (int s2 = 0; s2 < nl; ++s2) {
        ChanCell<double> g{};
        g.am = g.ap = a;
        g.glxl = a * lf[s2] * dph;
        g.glxx = a * lf[s2 + 1] * dph;
        g.bm = 1.0 + cphi(xm);
        g.bp = 1.0 + cphi(xp);
        g.cm = g.cp = 0.0;
        g.idl = 1.0 / (lf[s2 + 1] - lf[s2]);
        g.idx = 1.0 / (cchi(xp) - cchi(xm));
        gd[size_t(s2) * nx + p] = g;
        const double* src = &g.am;
        float* dst = &gf[size_t(s2) * nx + p].am;
        for (int q = 0; q < 12; ++q) dst[q] = float(src[q]);
      }
    }
    VLB_CUDA(c, cudaMalloc(&c->d_clbcgeo, sizeof(ChanCell<double>) * gd.size()));
    VLB_CUDA(c, cudaMalloc(&c->d_clbcgeof, sizeof(ChanCell<float>) * gf.size()));
    VLB_CUDA(c, cudaMemcpy(c->d_clbcgeo, gd.data(), sizeof(ChanCell<double>) * gd.size(), cudaMemcpyHostToDevice));
    VLB_CUDA(c, cudaMemcpy(c->d_clbcgeof, gf.data(), sizeof(ChanCell<float>) * gf.size(), cudaMemcpyHostToDevice));
  }
  if (formulation == 2 && c->n_cvariants == 0 && !c->d_clbgeo) {
    if (!c->d_lm) {
      st = setup_large(c);
      if (st != VLB_OK) return st;
    }
    c->lm.err = c->d_err;
    const vlb_channel_grid& gr = c->chan_grid;
    const int nl = gr.n_lambda, nx = gr.n_xi;
    const double A = gr.stretch_A, ea = atanh(A), re = gr.re_c, L = gr.xi_out - gr.xi_in;
    auto phi = [&](double x) { return 0.5 * (tanh(2.0) - tanh(2.0 - 30.0 * x / re)); };
    auto dphi = [&](double x) { const double ch = cosh(2.0 - 30.0 * x / re); return 0.5 * (30.0 / re) / (ch * ch); };
    auto chi = [&](double x) { return (1.0 + tanh(2.0) / 2.0) * x + re / 60.0 * log(cosh(2.0 - 30.0 * x / re) / cosh(2.0)); };
    std::vector<double> d;
    const size_t o_va = d.size();
    for (int p = 0; p < nx; ++p) d.push_back(1.0 / (1.0 + phi(gr.xi_in + L * (p + 0.5) / nx)));
    const size_t o_dph = d.size();
    for (int p = 0; p < nx; ++p) d.push_back(dphi(gr.xi_in + L * (p + 0.5) / nx));
    const size_t o_lf = d.size();
    for (int s2 = 0; s2 <= nl; ++s2) d.push_back(s2 == nl ? 1.0 : tanh(double(s2) / nl * ea) / A);
    const size_t o_vx = d.size();
    for (int p = 0; p <= nx; ++p) d.push_back(1.0 + phi(gr.xi_in + L * p / nx));
    const size_t o_idl = d.size();
    for (int s2 = 0; s2 < nl; ++s2) {
      const double lo = tanh(double(s2) / nl * ea) / A, hi = s2 + 1 == nl ? 1.0 : tanh(double(s2 + 1) / nl * ea) / A;
      d.push_back(1.0 / (hi - lo));
    }
    const size_t o_idx = d.size();
    for (int p = 0; p < nx; ++p) d.push_back(1.0 / (chi(gr.xi_in + L * (p + 1) / nx) - chi(gr.xi_in + L * p / nx)));
    const size_t o_weq = d.size();
    d.resize(d.size() + c->nq0 + c->nq1, 0.0);
    std::vector<int> ib(c->nq0);
    for (int k = 0; k < c->nq0; ++k) ib[k] = refl(c->margs.kind0, c->nq0, k);
    const size_t dbytes = d.size() * sizeof(double);
    VLB_CUDA(c, cudaMalloc(&c->d_clbgeo, dbytes + ib.size() * sizeof(int)));
    VLB_CUDA(c, cudaMemcpy(c->d_clbgeo, d.data(), dbytes, cudaMemcpyHostToDevice));
    VLB_CUDA(c, cudaMemcpy(static_cast<char*>(c->d_clbgeo) + dbytes, ib.data(), ib.size() * sizeof(int),
                           cudaMemcpyHostToDevice));
    const double* D = static_cast<const double*>(c->d_clbgeo);
    ClbGeom& g = c->clbg;
    g.nl = nl, g.nx = nx;
    g.va = D + o_va, g.dph = D + o_dph, g.lf = D + o_lf, g.vx = D + o_vx, g.idl = D + o_idl, g.idx = D + o_idx;
    g.weq = D + o_weq;
    g.ibar = reinterpret_cast<const int*>(static_cast<const char*>(c->d_clbgeo) + dbytes);
    const size_t cells = size_t(nl) * nx;
    VLB_CUDA(c, cudaMalloc(&c->d_clbrec, cells * (c->nq0 + c->nq1 + 2) * c->esize));
    VLB_CUDA(c, cudaMalloc(&c->d_clbres, size_t(nl) * 2 * (c->nq0 + c->nq1) * c->esize));
  }
  if (formulation == 2 && c->n_cvariants == 0) {
    st = upload_clb_weq(c);
    if (st != VLB_OK) return st;
  }
  c->clb = formulation == 2;
  c->clb_march = formulation == 2 && c->n_cvariants > 0;
  return VLB_OK;
}

vlb_status vlb_set_formulation(vlb_ctx* c, int formulation) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (formulation < 0 || formulation > 2) return fail(c, VLB_ERR_INVALID, "unknown formulation");
  if (c->kind == 1) return set_channel_formulation(c, formulation);
  if (formulation == 2) return fail(c, VLB_ERR_UNSUPPORTED, "the Cartesian split is a channel formulation");
  if (formulation == 1 && c->has_halo) return fail(c, VLB_ERR_UNSUPPORTED, "slabs run the chi formulation");
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int b = 0; b < 3; ++b) {  // captured graphs hold the old launch sequence
    if (c->graph_exec[b]) cudaGraphExecDestroy(c->graph_exec[b]);
    c->graph_exec[b] = nullptr;
    c->graph_variant[b] = -1;
  }
  if (formulation == 1) {
    // the fused stage kernel has an f~ instance of each velocity set's first launch shape
    bool fused = !c->large;
    if (fused) {
      StageVariant first[16];
      const int nf = c->prec == VLB_FP64 ? stage_variants<double>(c->nq0, c->nq1, first)
                                         : stage_variants<float>(c->nq0, c->nq1, first);
      fused = nf > 0 && c->n_variants >= 2 && c->variants[0].tc == first[0].tc && c->variants[0].nt == first[0].nt;
    }
    if (!fused) {
      vlb_status st = ensure_multi_path(c);
      if (st != VLB_OK) return st;
    }
    if (!c->d_tgeo || (fused && !c->d_ftgeo)) {  // per cell: sqrt(g), e_{s+1/2} / (d eta sqrt(g)), e_{s-1/2} / (...), 1 / R_s; per velocity forceR
      const size_t N = size_t(c->total_cells);
      std::vector<double> t(4 * N);
      for (int i = 0; i < c->n_inst; ++i) {
        const vlb_couette_grid& g = c->grids[i];
        const int n = g.n_cells;
        const double L = g.r_out - g.r_in;
        for (int s2 = 0; s2 < n; ++s2) {
          double sg, ep, em, R;
          if (g.stretch_A == 0.0) {
            R = g.r_in + (s2 + 0.5) / n * L;
            sg = R, ep = em = 1.0;
            const double de = L / n;
            ep /= de * sg, em /= de * sg;
          } else {
            const double A = g.stretch_A, dl = g.stretch_delta, A0 = dl > 1.0 - dl ? dl : 1.0 - dl;
            const double e_in = -atanh(A * dl / A0), e_out = atanh(A * (1.0 - dl) / A0), de = (e_out - e_in) / n;
            const double ec = e_in + (s2 + 0.5) * de, em_ = e_in + s2 * de, ep_ = e_in + (s2 + 1) * de;
            R = g.r_in + L * (dl + A0 / A * tanh(ec));
            sg = A0 * L * R / (A * cosh(ec) * cosh(ec));
            ep = A * cosh(ep_) * cosh(ep_) / (A0 * L) / (de * sg);
            em = A * cosh(em_) * cosh(em_) / (A0 * L) / (de * sg);
          }
          const size_t k = size_t(c->inst[i].cell0) + s2;
          t[k] = sg, t[N + k] = ep, t[2 * N + k] = em, t[3 * N + k] = 1.0 / R;
        }
      }
      // the inertial term of the rest state R_ij = w0_i w1_j through the discrete kernels
      const AxisTables &a0 = c->ax[0], &a1 = c->ax[1];
      const int nq0 = c->nq0, nq1 = c->nq1;
      std::vector<double> k0w(nq0, 0.0), k1w(nq1, 0.0);
      for (int i = 0; i < nq0; ++i)
        for (int k = 0; k < nq0; ++k) k0w[i] += a0.K[size_t(i) * nq0 + k] * a0.w[k];
      for (int j = 0; j < nq1; ++j)
        for (int l = 0; l < nq1; ++l) k1w[j] += a1.Kt[size_t(j) * nq1 + l] * a1.w[l];
      for (int i = 0; i < nq0; ++i)
        for (int j = 0; j < nq1; ++j)
          t.push_back(a1.p[j] * a1.p[j] * k0w[i] * a1.w[j] - a0.p[i] * a0.w[i] * k1w[j]);
      if (!c->d_tgeo) {
        VLB_CUDA(c, cudaMalloc(&c->d_tgeo, t.size() * sizeof(double)));
        VLB_CUDA(c, cudaMemcpy(c->d_tgeo, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
        c->lm.sqrtg = c->d_tgeo, c->lm.advp = c->d_tgeo + N, c->lm.advm = c->d_tgeo + 2 * N, c->lm.inv_r = c->d_tgeo + 3 * N;
        c->lm.forceR = c->d_tgeo + 4 * N;
      }
      if (fused && !c->d_ftgeo) {  // the fused kernel's records and arrays, in its bulk type
        std::vector<GeoCell> gd(N);
        std::vector<GeoCellF> gf(N);
        for (size_t k = 0; k < N; ++k) {
          gd[k] = GeoCell{t[N + k], t[2 * N + k], t[3 * N + k], 0.0};
          gf[k] = GeoCellF{float(t[N + k]), float(t[2 * N + k]), float(t[3 * N + k]), 0.0f};
        }
        const size_t V = size_t(c->nq0) * c->nq1;
        VLB_CUDA(c, cudaMalloc(&c->d_ftgeo, N * sizeof(GeoCell)));
        VLB_CUDA(c, cudaMalloc(&c->d_ftgeof, N * sizeof(GeoCellF)));
        VLB_CUDA(c, cudaMemcpy(c->d_ftgeo, gd.data(), N * sizeof(GeoCell), cudaMemcpyHostToDevice));
        VLB_CUDA(c, cudaMemcpy(c->d_ftgeof, gf.data(), N * sizeof(GeoCellF), cudaMemcpyHostToDevice));
        VLB_CUDA(c, cudaMalloc(&c->d_ftsg, N * c->esize));
        VLB_CUDA(c, cudaMalloc(&c->d_ftfr, V * c->esize));
        if (c->prec == VLB_FP64) {
          VLB_CUDA(c, cudaMemcpy(c->d_ftsg, t.data(), N * sizeof(double), cudaMemcpyHostToDevice));
          VLB_CUDA(c, cudaMemcpy(c->d_ftfr, t.data() + 4 * N, V * sizeof(double), cudaMemcpyHostToDevice));
        } else {
          std::vector<float> sg(N), fr(V);
          for (size_t k = 0; k < N; ++k) sg[k] = float(t[k]);
          for (size_t k = 0; k < V; ++k) fr[k] = float(t[4 * N + k]);
          VLB_CUDA(c, cudaMemcpy(c->d_ftsg, sg.data(), N * sizeof(float), cudaMemcpyHostToDevice));
          VLB_CUDA(c, cudaMemcpy(c->d_ftfr, fr.data(), V * sizeof(float), cudaMemcpyHostToDevice));
        }
      }
    }
    c->lm.ftilde = 1;
    c->ftilde = true;
    c->ft_fused = fused;
    if (fused && c->variant > 1) {
      vlb_status st = vlb_set_variant(c, c->variants[c->variant].persist ? 1 : 0);
      if (st != VLB_OK) return st;
    } else if (fused) {
      build_tiles(c);  // the tile list of the same launch shape, rebuilt for the f~ kernel's occupancy
      VLB_CUDA(c, cudaMemcpy(c->d_tiles, c->tiles.data(), sizeof(TileDesc) * c->tiles.size(), cudaMemcpyHostToDevice));
    }
    return VLB_OK;
  }
  c->lm.ftilde = 0;
  c->ftilde = false;
  if (!c->large) {  // the chi kernel's tile list
    build_tiles(c);
    VLB_CUDA(c, cudaMemcpy(c->d_tiles, c->tiles.data(), sizeof(TileDesc) * c->tiles.size(), cudaMemcpyHostToDevice));
  }
  return VLB_OK;
}

vlb_status vlb_set_collision(vlb_ctx* c, int collision, double prandtl) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (collision != 0 && collision != 1) return fail(c, VLB_ERR_INVALID, "collision must be VLB_BGK or VLB_SHAKHOV");
  if (collision == 1 && (!(prandtl > 0.0) || !std::isfinite(prandtl)))
    return fail(c, VLB_ERR_INVALID, "the Prandtl number must be finite and > 0");
  if (collision == 1 && c->large) return fail(c, VLB_ERR_UNSUPPORTED, "the Shakhov pass is built for up to 32 nodes per axis");
  if (collision == 1 && (c->margs.N0 < 3 || c->margs.N1 < 3))
    return fail(c, VLB_ERR_UNSUPPORTED, "the Shakhov term needs expansion orders >= 3 on both axes");
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int b = 0; b < 3; ++b) {  // captured graphs hold the old launch sequence
    if (c->graph_exec[b]) cudaGraphExecDestroy(c->graph_exec[b]);
    c->graph_exec[b] = nullptr;
    c->graph_variant[b] = -1;
  }
  c->collision = collision;
  c->prandtl = collision == 1 ? prandtl : 1.0;
  return VLB_OK;
}

vlb_status vlb_set_channel_flow_rate(vlb_ctx* c, double q0) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->kind != 1) return fail(c, VLB_ERR_UNSUPPORTED, "flow-rate ends belong to channel contexts");
  if (!(q0 >= 0.0) || !std::isfinite(q0)) return fail(c, VLB_ERR_INVALID, "the flow rate must be finite and >= 0");
  if (c->clb) return fail(c, VLB_ERR_STATE, "the Cartesian split runs with reservoir ends");
  const int nl = c->cdesc.nl;
  // Eqs. (canalie_inlet, canalie_outlet), H = 2: Q_s = 3 Q0 (1 - 4 lambda_s^2 / H^2) / (H (1 + phi))
  std::vector<double> q(size_t(4) * nl);
  const double H = 2.0;
  for (int e = 0; e < 2; ++e) {
    const double ph = c->chan_phi_end[e];
    for (int r = 0; r < nl; ++r) {
      const double lam = c->chan_lc[r];
      const double Qs = 3.0 * q0 * (1.0 - 4.0 * lam * lam / (H * H)) / (H * (1.0 + ph));
      q[size_t(2 * e) * nl + r] = Qs;
      q[size_t(2 * e + 1) * nl + r] = (1.0 + ph) * Qs;
    }
  }
  if (!c->d_qflow) VLB_CUDA(c, cudaMalloc(&c->d_qflow, size_t(4) * nl * c->esize));
  if (c->prec == VLB_FP64) {
    VLB_CUDA(c, cudaMemcpy(c->d_qflow, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> qf(q.begin(), q.end());
    VLB_CUDA(c, cudaMemcpy(c->d_qflow, qf.data(), qf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  c->cdesc.flow = 1;
  c->cdesc.q0 = q0;
  return drop_channel_graphs(c);
}

vlb_status vlb_channel_postprocess(vlb_ctx* c, double* ux, double* uy, double* psi, double* omega, double* pw) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->kind != 1) return fail(c, VLB_ERR_UNSUPPORTED, "post-processing belongs to channel contexts");
  if (c->clb) return fail(c, VLB_ERR_STATE, "post-processing reads triad components (the vielbein formulation)");
  const int nl = c->cdesc.nl, nx = c->cdesc.nx;
  const size_t cells = size_t(nl) * nx, npsi = size_t(nl + 1) * nx;
  const size_t total = 3 * cells + npsi + nx;
  if (!c->d_post) VLB_CUDA(c, cudaMalloc(&c->d_post, total * sizeof(double)));
  vlb_status st = compute_moments(c, c->d_mom);
  if (st != VLB_OK) return st;
  double* d = c->d_post;
  cudaError_t e = launch_channel_post(c->d_mom, c->d_cpost, nl, nx, c->chan_dxi, d, d + cells, d + 2 * cells,
                                      d + 3 * cells, d + 3 * cells + npsi, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "post-processing kernel launch");
  double* dst[5] = {ux, uy, omega, psi, pw};
  const size_t off[5] = {0, cells, 2 * cells, 3 * cells, 3 * cells + npsi};
  const size_t cnt[5] = {cells, cells, cells, npsi, size_t(nx)};
  for (int k = 0; k < 5; ++k)
    if (dst[k])
      VLB_CUDA(c, cudaMemcpyAsync(dst[k], d + off[k], cnt[k] * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_err(c);
}

vlb_status vlb_init_equilibrium(vlb_ctx* c, double n0, double u0, double u1, double T0) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (!(n0 > 0.0) || !(T0 > 0.0)) return fail(c, VLB_ERR_INVALID, "need n0 > 0 and T0 > 0");
  cudaError_t e = c->large
                      ? (c->prec == VLB_FP64
                             ? lm_init<double>(c->lm, static_cast<double*>(c->F[c->cur]), c->total_cells, n0, u0, u1,
                                               T0, c->stream)
                             : lm_init<float>(c->lm, static_cast<float*>(c->F[c->cur]), c->total_cells, n0, u0, u1,
                                              T0, c->stream))
                  : c->prec == VLB_FP64
                      ? launch_init_equilibrium<double>(static_cast<double*>(c->F[c->cur]), c->total_cells, c->Vp,
                                                        c->margs, n0, u0, u1, T0, c->stream)
                      : launch_init_equilibrium<float>(static_cast<float*>(c->F[c->cur]), c->total_cells, c->Vp,
                                                       c->margs, n0, u0, u1, T0, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel launch");
  c->last = c->cur;
  c->stage_done = 0;
  c->have_prev = false;
  return VLB_OK;
}

vlb_status vlb_init_from_moments(vlb_ctx* c, const double* n, const double* u0, const double* u1, const double* T,
                                 const double* q0, int on_device) {
  if (!c || !n || !u0 || !u1 || !T) return fail(c, VLB_ERR_INVALID, "null argument");
  if (c->large) return fail(c, VLB_ERR_UNSUPPORTED, "seeding is built for up to 32 nodes per axis");
  const size_t N = size_t(c->total_cells);
  if (!on_device)
    for (size_t i = 0; i < N; ++i)
      if (!(n[i] > 0.0) || !(T[i] > 0.0) || !std::isfinite(u0[i]) || !std::isfinite(u1[i]) ||
          (q0 && !std::isfinite(q0[i])))
        return fail(c, VLB_ERR_INVALID, "fields must be finite with n > 0 and T > 0");
  const double* src[5] = {n, u0, u1, T, q0};
  double* dev = c->d_mom;  // 9 doubles per cell of room: five of them stage the fields
  for (int a = 0; a < 5; ++a) {
    if (!src[a]) continue;
    VLB_CUDA(c, cudaMemcpyAsync(dev + a * N, src[a], sizeof(double) * N,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  if (!on_device) VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  const double* dq = q0 ? dev + 4 * N : nullptr;
  cudaError_t e = c->prec == VLB_FP64
                      ? launch_seed<double>(static_cast<double*>(c->F[c->cur]), c->total_cells, c->Vp, c->margs, dev,
                                            dev + N, dev + 2 * N, dev + 3 * N, dq, c->stream, c->cmap)
                      : launch_seed<float>(static_cast<float*>(c->F[c->cur]), c->total_cells, c->Vp, c->margs, dev,
                                           dev + N, dev + 2 * N, dev + 3 * N, dq, c->stream, c->cmap);
  if (e != cudaSuccess) return cuda_fail(c, e, "seed kernel launch");
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->last = c->cur;
  c->stage_done = 0;
  c->have_prev = false;
  return VLB_OK;
}

vlb_status vlb_set_f(vlb_ctx* c, const void* f, int on_device) {
  if (!c || !f) return fail(c, VLB_ERR_INVALID, "null argument");
  const void* src = f;
  if (!on_device) {  // stage the host array in a buffer that holds nothing live
    void* stage = c->F[(c->cur + 1) % 3];
    VLB_CUDA(c, cudaMemcpyAsync(stage, f, size_t(c->total_cells) * 2 * c->V * c->esize, cudaMemcpyHostToDevice,
                                c->stream));
    src = stage;
  }
  vlb_status st = convert(c, src, c->F[c->cur], 1);
  if (st != VLB_OK) return st;
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->last = c->cur;
  c->stage_done = 0;
  c->have_prev = false;
  return VLB_OK;
}

vlb_status vlb_read_f(vlb_ctx* c, void* f, int on_device) {
  if (!c || !f) return fail(c, VLB_ERR_INVALID, "null argument");
  if (on_device) {
    vlb_status st = convert(c, c->F[c->last], f, 0);
    if (st != VLB_OK) return st;
  } else {
    void* stage = c->F[spare_buffer(c)];
    vlb_status st = convert(c, c->F[c->last], stage, 0);
    if (st != VLB_OK) return st;
    VLB_CUDA(c, cudaMemcpyAsync(f, stage, size_t(c->total_cells) * 2 * c->V * c->esize, cudaMemcpyDeviceToHost,
                                c->stream));
  }
  return check_err(c);
}

vlb_status vlb_set_dt(vlb_ctx* c, const double* dt) {
  if (!c || !dt) return fail(c, VLB_ERR_INVALID, "null argument");
  for (int i = 0; i < c->n_inst; ++i)
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(c, VLB_ERR_INVALID, "time steps must be finite and positive");
  for (int i = 0; i < c->n_inst; ++i) {
    c->inst[i].dt = dt[i];
    c->inst[i].dt_f = float(dt[i]);
  }
  VLB_CUDA(c, cudaMemcpyAsync(c->d_inst, c->inst.data(), sizeof(InstDesc) * c->n_inst, cudaMemcpyHostToDevice,
                              c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return drop_channel_graphs(c);
}

static vlb_status apply_dt(vlb_ctx* c, double dt) {
  if (dt < 0.0 || !std::isfinite(dt)) return fail(c, VLB_ERR_INVALID, "dt must be finite and >= 0");
  if (dt > 0.0) {
    bool change = false;
    for (int i = 0; i < c->n_inst; ++i) change |= c->inst[i].dt != dt;
    if (change) {
      std::vector<double> v(c->n_inst, dt);
      return vlb_set_dt(c, v.data());
    }
    return VLB_OK;
  }
  for (int i = 0; i < c->n_inst; ++i)
    if (!(c->inst[i].dt > 0.0)) return fail(c, VLB_ERR_STATE, "dt = 0 needs per-instance steps from vlb_set_dt");
  return VLB_OK;
}

vlb_status vlb_stage(vlb_ctx* c, double dt, int k) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (k < 1 || k > 3) return fail(c, VLB_ERR_INVALID, "stage must be 1, 2 or 3");
  if (k != c->stage_done % 3 + 1) return fail(c, VLB_ERR_STATE, "stages must run in the order 1, 2, 3");
  vlb_status st = apply_dt(c, dt);
  if (st != VLB_OK) return st;
  c->launches = 0;
  return run_stage(c, k);
}

vlb_status vlb_step(vlb_ctx* c, double dt, long long nsteps) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->has_halo) return fail(c, VLB_ERR_STATE, "a slab steps one stage at a time (vlb_stage), halos written before each");
  if (nsteps < 0) return fail(c, VLB_ERR_INVALID, "nsteps must be >= 0");
  if (c->stage_done % 3 != 0) return fail(c, VLB_ERR_STATE, "a partial RK3 step is pending");
  vlb_status st = apply_dt(c, dt);
  if (st != VLB_OK) return st;
  c->launches = 0;
  for (long long s = 0; s < nsteps; ++s)
    for (int k = 1; k <= 3; ++k) {
      st = run_stage(c, k);
      if (st != VLB_OK) return st;
    }
  return VLB_OK;
}

vlb_status vlb_read_moments(vlb_ctx* c, double* n, double* u0, double* u1, double* T, double* Tab, double* q,
                            int on_device) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  vlb_status st = compute_moments(c, c->d_mom);
  if (st != VLB_OK) return st;
  std::vector<double> h(size_t(9) * c->total_cells);
  VLB_CUDA(c, cudaMemcpyAsync(h.data(), c->d_mom, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  st = check_err(c);
  if (st != VLB_OK) return st;
  const long long N = c->total_cells;
  std::vector<double> tmp[6];
  double* dst[6] = {n, u0, u1, T, Tab, q};
  bool bad = false;
  for (long long i = 0; i < N; ++i) {
    const double* o = &h[size_t(9) * i];
    for (int k = 0; k < 9; ++k) bad |= !std::isfinite(o[k]);
  }
  if (on_device) {
    for (int a = 0; a < 6; ++a) {
      if (!dst[a]) continue;
      const int width = a == 4 ? 3 : a == 5 ? 2 : 1;
      tmp[a].resize(size_t(N) * width);
      for (long long i = 0; i < N; ++i)
        for (int k = 0; k < width; ++k) {
          const int src = a < 4 ? a : (a == 4 ? 4 + k : 7 + k);
          tmp[a][size_t(i) * width + k] = h[size_t(9) * i + src];
        }
      VLB_CUDA(c, cudaMemcpyAsync(dst[a], tmp[a].data(), tmp[a].size() * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
    }
    VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  } else {
    for (long long i = 0; i < N; ++i) {
      const double* o = &h[size_t(9) * i];
      if (n) n[i] = o[0];
      if (u0) u0[i] = o[1];
      if (u1) u1[i] = o[2];
      if (T) T[i] = o[3];
      if (Tab) Tab[3 * i] = o[4], Tab[3 * i + 1] = o[5], Tab[3 * i + 2] = o[6];
      if (q) q[2 * i] = o[7], q[2 * i + 1] = o[8];
    }
  }
  if (bad) return fail(c, VLB_ERR_NONFINITE, "a moment is NaN or Inf");
  return VLB_OK;
}

vlb_status vlb_wall_density(vlb_ctx* c, double* nw) {
  if (!c || !nw) return fail(c, VLB_ERR_INVALID, "null argument");
  const size_t cnt = c->kind == 1 ? size_t(c->cdesc.nx) : size_t(2) * c->n_inst;
  VLB_CUDA(c, cudaMemcpyAsync(nw, c->d_nw, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  return check_err(c);
}

// the weighted sums of squares of Eq. (msites_steady) per instance (zeros on the first call)
static vlb_status residual_sums(vlb_ctx* c, std::vector<double>& res) {
  if (c->kind != 0) return fail(c, VLB_ERR_UNSUPPORTED, "steady-state norms are defined for Couette contexts");
  vlb_status st = compute_moments(c, c->d_mom);
  if (st != VLB_OK) return st;
  res.assign(3 * size_t(c->n_inst), 0.0);
  if (c->have_prev) {
    cudaError_t e = launch_residual(c->d_mom, c->d_prev, c->d_inst, c->d_geo, c->n_inst, c->d_res, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "residual kernel launch");
    VLB_CUDA(c, cudaMemcpyAsync(res.data(), c->d_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  VLB_CUDA(c, cudaMemcpyAsync(c->d_prev, c->d_mom, sizeof(double) * 9 * c->total_cells, cudaMemcpyDeviceToDevice,
                              c->stream));
  st = check_err(c);
  if (st != VLB_OK) return st;
  c->have_prev = true;
  return VLB_OK;
}

vlb_status vlb_residual(vlb_ctx* c, double* l2u, double* l2n, double* l2T) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  std::vector<double> res;
  vlb_status st = residual_sums(c, res);
  if (st != VLB_OK) return st;
  for (int i = 0; i < c->n_inst; ++i) {
    if (l2u) l2u[i] = std::sqrt(res[3 * i]);
    if (l2n) l2n[i] = std::sqrt(res[3 * i + 1]);
    if (l2T) l2T[i] = std::sqrt(res[3 * i + 2]);
  }
  return VLB_OK;
}

vlb_status vlb_residual_sums(vlb_ctx* c, double* su, double* sn, double* sT) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  std::vector<double> res;
  vlb_status st = residual_sums(c, res);
  if (st != VLB_OK) return st;
  for (int i = 0; i < c->n_inst; ++i) {
    if (su) su[i] = res[3 * i];
    if (sn) sn[i] = res[3 * i + 1];
    if (sT) sT[i] = res[3 * i + 2];
  }
  return VLB_OK;
}

long long vlb_halo_bytes(const vlb_ctx* c) {
  if (!c) return VLB_ERR_INVALID;
  return 3ll * 2 * c->Vp * (long long)c->esize;
}

// the buffer the next stage reads as F_prev (see run_stage)
static int next_stage_input(const vlb_ctx* c) {
  const int k = c->stage_done % 3 + 1;
  return k == 1 ? c->cur : (k == 2 ? (c->cur + 1) % 3 : (c->cur + 2) % 3);
}

vlb_status vlb_read_edge(vlb_ctx* c, int inst, int end, void* rows, int on_device) {
  if (!c || !rows) return fail(c, VLB_ERR_INVALID, "null argument");
  if (c->kind != 0) return fail(c, VLB_ERR_UNSUPPORTED, "slabs are Couette instances");
  if (inst < 0 || inst >= c->n_inst || (end != 0 && end != 1)) return fail(c, VLB_ERR_INVALID, "bad instance or end");
  const InstDesc& d = c->inst[inst];
  const size_t rowb = size_t(2) * c->Vp * c->esize;
  const long long first = d.cell0 + (end == 0 ? 0 : d.n_cells - 3);
  const char* src = static_cast<const char*>(c->F[next_stage_input(c)]) + size_t(first) * rowb;
  VLB_CUDA(c, cudaMemcpyAsync(rows, src, 3 * rowb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return VLB_OK;
}

vlb_status vlb_write_halo(vlb_ctx* c, int inst, int end, const void* rows, int on_device) {
  if (!c || !rows) return fail(c, VLB_ERR_INVALID, "null argument");
  if (c->kind != 0) return fail(c, VLB_ERR_UNSUPPORTED, "slabs are Couette instances");
  if (inst < 0 || inst >= c->n_inst || (end != 0 && end != 1)) return fail(c, VLB_ERR_INVALID, "bad instance or end");
  if (!(c->inst[inst].halo & (1 << end))) return fail(c, VLB_ERR_STATE, "that end is a wall, not a slab halo");
  const size_t rowb = size_t(2) * c->Vp * c->esize;
  char* dst = static_cast<char*>(c->d_halo) + (size_t(inst) * 2 + end) * 3 * rowb;
  VLB_CUDA(c, cudaMemcpyAsync(dst, rows, 3 * rowb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return VLB_OK;
}

struct SaveHeader {
  char magic[8];
  int model[6];
  int prec, n_inst, V, pad;
  long long total_cells, steps;
};

vlb_status vlb_save(vlb_ctx* c, const char* path) {
  if (!c || !path) return fail(c, VLB_ERR_INVALID, "null argument");
  if (c->stage_done % 3 != 0) return fail(c, VLB_ERR_STATE, "save between full steps only");
  SaveHeader h{};
  memcpy(h.magic, "VLBSAVE3", 8);
  for (int a = 0; a < 2; ++a) {
    h.model[3 * a] = c->model.kind[a];
    h.model[3 * a + 1] = c->model.N[a];
    h.model[3 * a + 2] = c->model.Q[a];
  }
  h.prec = c->prec;
  h.n_inst = c->n_inst;
  h.V = c->V;
  h.total_cells = c->total_cells;
  h.steps = c->steps;
  // the device buffer as stored (the deviation from the rest state), so that a run
  // continued from the file is bitwise the run that wrote it
  std::vector<char> buf(size_t(c->total_cells) * 2 * c->Vp * c->esize);
  VLB_CUDA(c, cudaMemcpyAsync(buf.data(), c->F[c->last], buf.size(), cudaMemcpyDeviceToHost, c->stream));
  vlb_status st = check_err(c);
  if (st != VLB_OK) return st;
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(c, VLB_ERR_INVALID, std::string("cannot open ") + path);
  bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
  for (int i = 0; i < c->n_inst && ok; ++i) ok = fwrite(&c->inst[i].n_cells, sizeof(int), 1, fp) == 1;
  ok = ok && fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  ok = (fclose(fp) == 0) && ok;
  if (!ok) return fail(c, VLB_ERR_INVALID, "write failed");
  return VLB_OK;
}

vlb_status vlb_load(vlb_ctx* c, const char* path) {
  if (!c || !path) return fail(c, VLB_ERR_INVALID, "null argument");
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(c, VLB_ERR_INVALID, std::string("cannot open ") + path);
  SaveHeader h{};
  bool ok = fread(&h, sizeof(h), 1, fp) == 1 && memcmp(h.magic, "VLBSAVE3", 8) == 0;
  for (int a = 0; a < 2 && ok; ++a)
    ok = h.model[3 * a] == c->model.kind[a] && h.model[3 * a + 1] == c->model.N[a] &&
         h.model[3 * a + 2] == c->model.Q[a];
  ok = ok && h.prec == c->prec && h.n_inst == c->n_inst && h.V == c->V && h.total_cells == c->total_cells;
  for (int i = 0; i < c->n_inst && ok; ++i) {
    int nc = 0;
    ok = fread(&nc, sizeof(int), 1, fp) == 1 && nc == c->inst[i].n_cells;
  }
  std::vector<char> buf(size_t(c->total_cells) * 2 * c->Vp * c->esize);
  ok = ok && fread(buf.data(), 1, buf.size(), fp) == buf.size();
  fclose(fp);
  if (!ok) return fail(c, VLB_ERR_INVALID, "file does not match this context");
  VLB_CUDA(c, cudaMemcpyAsync(c->F[c->cur], buf.data(), buf.size(), cudaMemcpyHostToDevice, c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->last = c->cur;
  c->stage_done = 0;
  c->have_prev = false;
  c->steps = h.steps;
  return VLB_OK;
}

int vlb_channel_variants(const vlb_ctx* c, int* ts, int* tp, int* nt, int max) {
  if (!c) return VLB_ERR_INVALID;
  if (c->kind != 1) return 0;
  for (int v = 0; v < c->n_cvariants && v < max; ++v) {
    int L = 0, n = 0;
    channel_segments(c, c->cvariants[v], &L, &n);
    if (ts) ts[v] = L;
    if (tp) tp[v] = c->cvariants[v].tp;
    if (nt) nt[v] = c->cvariants[v].nt;
  }
  return c->n_cvariants;
}

int vlb_channel_variant_tensor_cores(const vlb_ctx* c, int v) {
  if (!c || c->kind != 1 || v < 0 || v >= c->n_cvariants) return VLB_ERR_INVALID;
  return c->cvariants[v].tc;
}

int vlb_variants(const vlb_ctx* c, int* tc, int* nt, int* persistent, int max) {
  if (!c) return VLB_ERR_INVALID;
  if (c->kind == 1) {
    for (int v = 0; v < c->n_cvariants && v < max; ++v) {
      int L = 0, n = 0;
      channel_segments(c, c->cvariants[v], &L, &n);
      if (tc) tc[v] = L * c->cvariants[v].tp;
      if (nt) nt[v] = c->cvariants[v].nt;
      if (persistent) persistent[v] = 0;
    }
    return c->n_cvariants;
  }
  for (int v = 0; v < c->n_variants && v < max; ++v) {
    if (tc) tc[v] = c->variants[v].tc;
    if (nt) nt[v] = c->variants[v].nt;
    if (persistent) persistent[v] = c->variants[v].persist;
  }
  return c->n_variants;
}

vlb_status vlb_set_variant(vlb_ctx* c, int v) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->kind == 1 && c->n_cvariants == 0 && v == 0) return VLB_OK;  // a Cartesian-split-only channel
  if (v < 0 || v >= (c->kind == 1 ? c->n_cvariants : c->n_variants)) return fail(c, VLB_ERR_INVALID, "no such launch shape");
  if (c->kind == 0 && c->ftilde && c->ft_fused && v > 1)
    return fail(c, VLB_ERR_INVALID, "the f~ formulation runs launch shape 0 (variants 0 and 1)");
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->variant = v;
  if (c->kind == 1 || c->large) return VLB_OK;
  build_tiles(c);
  VLB_CUDA(c, cudaMemcpyAsync(c->d_tiles, c->tiles.data(), sizeof(TileDesc) * c->tiles.size(),
                              cudaMemcpyHostToDevice, c->stream));
  VLB_CUDA(c, cudaStreamSynchronize(c->stream));
  return VLB_OK;
}

vlb_status vlb_autotune(vlb_ctx* c, double dt, int reps, int* chosen, double* best_ms) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (reps < 1) return fail(c, VLB_ERR_INVALID, "reps must be >= 1");
  if (c->stage_done % 3 != 0) return fail(c, VLB_ERR_STATE, "a partial RK3 step is pending");
  vlb_status st = apply_dt(c, dt);
  if (st != VLB_OK) return st;
  cudaEvent_t e0, e1;
  VLB_CUDA(c, cudaEventCreate(&e0));
  VLB_CUDA(c, cudaEventCreate(&e1));
  int best = 0;
  float best_t = 1e30f;
  const int keep_last = c->last;
  const int nvar = c->kind == 1 ? std::max(1, c->n_cvariants) : (c->ftilde && c->ft_fused ? 2 : c->n_variants);
  for (int v = 0; v < nvar; ++v) {
    st = vlb_set_variant(c, v);
    if (st != VLB_OK) break;
    // stage 1 only reads F_l and writes the scratch buffer F^(1): the state is unchanged
    for (int w = 0; w < 2 && st == VLB_OK; ++w) st = run_stage(c, 1);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && st == VLB_OK; ++r) st = run_stage(c, 1);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best_t) best_t = ms, best = v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->stage_done = 0;
  c->last = keep_last;
  if (st != VLB_OK) return st;
  st = vlb_set_variant(c, best);
  if (st != VLB_OK) return st;
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  return VLB_OK;
}

vlb_status vlb_step_graph(vlb_ctx* c, double dt, long long nsteps) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->has_halo) return fail(c, VLB_ERR_STATE, "a slab steps one stage at a time (vlb_stage), halos written before each");
  if (nsteps < 0) return fail(c, VLB_ERR_INVALID, "nsteps must be >= 0");
  if (c->stage_done % 3 != 0) return fail(c, VLB_ERR_STATE, "a partial RK3 step is pending");
  vlb_status st = apply_dt(c, dt);
  if (st != VLB_OK) return st;
  c->launches = 0;
  const long long groups = nsteps / 3;
  // the graph bakes in the buffer roles of the three steps, which depend on
  // the buffer F_l starts in: one graph per starting buffer
  const int gc = c->cur;
  if (groups > 0 && (!c->graph_exec[gc] || c->graph_variant[gc] != c->variant)) {
    // capture three steps: the buffer rotation returns to the same F_l after three steps
    if (c->graph_exec[gc]) {
      cudaGraphExecDestroy(c->graph_exec[gc]);
      c->graph_exec[gc] = nullptr;
    }
    cudaStream_t s = c->stream;
    if (!s) {
      if (!c->capture_stream) VLB_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
      s = c->capture_stream;
    }
    const int keep_cur = c->cur, keep_last = c->last, keep_done = c->stage_done;
    const long long keep_steps = c->steps;
    cudaStream_t keep_stream = c->stream;
    c->stream = s;
    VLB_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    vlb_status cst = VLB_OK;
    for (int r = 0; r < 3 && cst == VLB_OK; ++r)
      for (int k = 1; k <= 3 && cst == VLB_OK; ++k) cst = run_stage(c, k);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    c->stream = keep_stream;
    c->cur = keep_cur, c->last = keep_last, c->stage_done = keep_done, c->steps = keep_steps;
    if (cst != VLB_OK) {
      if (g) cudaGraphDestroy(g);
      return cst;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph_exec[gc], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graph_variant[gc] = c->variant;
  }
  for (long long r = 0; r < groups; ++r) {
    VLB_CUDA(c, cudaGraphLaunch(c->graph_exec[gc], c->stream));
    c->steps += 3;
  }
  c->launches = groups * 9;
  if (groups > 0) c->last = c->cur;  // three steps bring F_l back to the same buffer
  for (long long s = 0; s < nsteps - 3 * groups; ++s)
    for (int k = 1; k <= 3; ++k) {
      st = run_stage(c, k);
      if (st != VLB_OK) return st;
    }
  return VLB_OK;
}

vlb_status vlb_run_to_steady(vlb_ctx* c, double dt, long long check_steps, double threshold, long long max_steps,
                             long long* steps_taken, double* residual, long long* converged_step) {
  if (!c) return fail(nullptr, VLB_ERR_INVALID, "null context");
  if (c->kind != 0) return fail(c, VLB_ERR_UNSUPPORTED, "steady-state norms are defined for Couette contexts");
  if (c->has_halo) return fail(c, VLB_ERR_STATE, "a slab steps one stage at a time (vlb_stage), halos written before each");
  if (check_steps < 1 || !(threshold > 0.0) || max_steps < check_steps)
    return fail(c, VLB_ERR_INVALID, "need check_steps >= 1, threshold > 0, max_steps >= check_steps");
  const int ni = c->n_inst;
  std::vector<double> l2u(ni), l2n(ni), l2T(ni);
  std::vector<long long> conv(ni, -1);
  c->have_prev = false;
  vlb_status st = vlb_residual(c, nullptr, nullptr, nullptr);  // stores the starting moments
  if (st != VLB_OK) return st;
  long long done = 0;
  int left = ni;
  while (done < max_steps && left > 0) {
    st = vlb_step_graph(c, dt, check_steps);
    if (st != VLB_OK) return st;
    done += check_steps;
    st = vlb_residual(c, l2u.data(), l2n.data(), l2T.data());
    if (st != VLB_OK) return st;
    for (int i = 0; i < ni; ++i) {
      const double r = std::max(l2u[i], std::max(l2n[i], l2T[i]));
      if (residual) residual[i] = r;
      if (conv[i] < 0 && r < threshold) {
        conv[i] = done;
        --left;
      }
    }
  }
  if (steps_taken) *steps_taken = done;
  for (int i = 0; i < ni; ++i)
    if (converged_step) converged_step[i] = conv[i];
  return VLB_OK;
}

long long vlb_kernel_launches(const vlb_ctx* c) { return c ? c->launches : 0; }

const char* vlb_last_error(const vlb_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

void vlb_destroy(vlb_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int b = 0; b < 3; ++b) cudaFree(c->F[b]);
  cudaFree(c->d_inst);
  cudaFree(c->d_tiles);
  cudaFree(c->d_geo);
  cudaFree(c->d_geof);
  cudaFree(c->d_cgeo);
  cudaFree(c->d_cgeof);
  cudaFree(c->d_ctab);
  for (int b = 0; b < 3; ++b)
    if (c->graph_exec[b]) cudaGraphExecDestroy(c->graph_exec[b]);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  cudaFree(c->d_nw);
  cudaFree(c->d_wall);
  cudaFree(c->d_err);
  cudaFree(c->d_mom);
  cudaFree(c->d_prev);
  cudaFree(c->d_res);
  cudaFree(c->d_halo);
  cudaFree(c->d_qflow);
  cudaFree(c->d_cpost);
  cudaFree(c->d_post);
  cudaFree(c->d_lm);
  cudaFree(c->d_lwall);
  cudaFree(c->d_lrec);
  cudaFree(c->d_lforce);
  cudaFree(c->d_lpart);
  cudaFree(c->d_tgeo);
  cudaFree(c->d_ftgeo);
  cudaFree(c->d_ftgeof);
  cudaFree(c->d_ftsg);
  cudaFree(c->d_ftfr);
  cudaFree(c->d_clbgeo);
  cudaFree(c->d_clbcgeo);
  cudaFree(c->d_clbcgeof);
  cudaFree(c->d_clbrec);
  cudaFree(c->d_clbres);
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------- residual kernel
namespace vlb {

// One block per instance: squared L2 norms of Eq. (msites_steady) with the weights R dR
// (equidistant grid) or the rectangle rule in eta (stretched grid).
__global__ void residual_kernel(const double* mom, const double* prev, const InstDesc* inst, const GeoCell* geo,
                                double* res) {
  __shared__ double red[3][32];
  const InstDesc in = inst[blockIdx.x];
  const double uw = in.u_in != 0.0 ? fabs(in.u_in) : 1.0;
  double su = 0, sn = 0, sT = 0;
  for (int s = threadIdx.x; s < in.n_cells; s += blockDim.x) {
    const long long c = in.cell0 + s;
    const double w = geo[c].wres;
    const double* a = mom + 9 * c;
    const double* b = prev + 9 * c;
    const double du = (a[2] - b[2]) / uw, dn = a[0] / b[0] - 1.0, dT = a[3] / b[3] - 1.0;
    su += w * du * du;
    sn += w * dn * dn;
    sT += w * dT * dT;
  }
  su = warp_sum<double>(su);
  sn = warp_sum<double>(sn);
  sT = warp_sum<double>(sT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[0][warp] = su, red[1][warp] = sn, red[2][warp] = sT;
  __syncthreads();
  if (threadIdx.x < 3) {  // the sums of squares; the host takes the square root
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    res[3 * blockIdx.x + threadIdx.x] = t;
  }
}

cudaError_t launch_residual(const double* mom, const double* prev, const InstDesc* inst, const GeoCell* geo,
                            int n_inst, double* res, cudaStream_t s) {
  residual_kernel<<<n_inst, 256, 0, s>>>(mom, prev, inst, geo, res);
  return cudaGetLastError();
}

// Channel post-processing (Sec. VII.D-F), one thread per xi column p, moments mom in the
// caller's cell order p * nl + s (n, u^lambda-hat, u^xi-hat, T first):
//  - Cartesian velocity (Eq. canalie_u): u^x = (u^l + a u^x-hat) / r, u^y = (u^x-hat - a u^l) / r,
//    a = lambda_s phi'(xi_p), r = sqrt(1 + a^2);
//  - stream function at the row interfaces (Eq. canalie_psi_sol), zero on the centreline:
//    psi_{s+1/2} = psi_{s-1/2} - n u^y (lambda_{s+1/2} - lambda_{s-1/2}) (1 + phi_p);
//  - vorticity (Eq. canalie_vorti): -d u^x / d xi + [d u^y / d lambda + a d u^x / d lambda] / (1 + phi),
//    xi derivatives centred (second-order one-sided at the first and last column), lambda
//    derivatives by the three-point formulas on the non-equidistant rows (bulk, first, last node);
//  - wall pressure: P = n T extrapolated linearly from the last two rows to lambda = 1.
// tab: lambda_c (nl), lambda_f (nl + 1), phi (nx), phi' (nx) of the column centres.
__global__ void channel_post_kernel(const double* mom, const double* tab, int nl, int nx, double dxi, double* ux,
                                    double* uy, double* omega, double* psi, double* pw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx) return;
  const double* lc = tab;
  const double* lf = lc + nl;
  const double* ph = lf + nl + 1;
  const double* dph = ph + nx;
  auto cart = [&](int q, int s, double& x, double& y) {
    const double* m = mom + 9 * (size_t(q) * nl + s);
    const double a = lc[s] * dph[q], r = sqrt(1.0 + a * a);
    x = (m[1] + a * m[2]) / r;
    y = (m[2] - a * m[1]) / r;
  };
  auto cx = [&](int q, int s) { double x, y; cart(q, s, x, y); return x; };
  auto cy = [&](int q, int s) { double x, y; cart(q, s, x, y); return y; };
  // three-point d/d lambda of g(row) at row s
  auto dl = [&](auto g, int s) {
    if (s == 0) {
      const double l1 = lc[0], l2 = lc[1], l3 = lc[2];
      return -(l2 + l3 - 2 * l1) * g(0) / ((l2 - l1) * (l3 - l1)) + (l3 - l1) * g(1) / ((l2 - l1) * (l3 - l2)) -
             (l2 - l1) * g(2) / ((l3 - l1) * (l3 - l2));
    }
    if (s == nl - 1) {
      const double lN = lc[nl - 1], lN1 = lc[nl - 2], lN2 = lc[nl - 3];
      return (2 * lN - lN1 - lN2) * g(nl - 1) / ((lN - lN1) * (lN - lN2)) -
             (lN - lN2) * g(nl - 2) / ((lN - lN1) * (lN1 - lN2)) + (lN - lN1) * g(nl - 3) / ((lN - lN2) * (lN1 - lN2));
    }
    const double lm = lc[s - 1], l0 = lc[s], lp = lc[s + 1];
    return (l0 - lm) * g(s + 1) / ((lp - l0) * (lp - lm)) + (lp - 2 * l0 + lm) * g(s) / ((lp - l0) * (l0 - lm)) -
           (lp - l0) * g(s - 1) / ((lp - lm) * (l0 - lm));
  };
  double ps = 0.0;
  psi[size_t(p) * (nl + 1)] = 0.0;
  for (int s = 0; s < nl; ++s) {
    double x, y;
    cart(p, s, x, y);
    const size_t k = size_t(p) * nl + s;
    ux[k] = x;
    uy[k] = y;
    ps = ps - mom[9 * k] * y * (lf[s + 1] - lf[s]) * (1.0 + ph[p]);
    psi[size_t(p) * (nl + 1) + s + 1] = ps;
    double dxux;
    if (p == 0) dxux = (-3.0 * x + 4.0 * cx(1, s) - cx(2, s)) / (2.0 * dxi);
    else if (p == nx - 1) dxux = (3.0 * x - 4.0 * cx(nx - 2, s) + cx(nx - 3, s)) / (2.0 * dxi);
    else dxux = (cx(p + 1, s) - cx(p - 1, s)) / (2.0 * dxi);
    const double dly = dl([&](int r) { return cy(p, r); }, s);
    const double dlx = dl([&](int r) { return cx(p, r); }, s);
    omega[k] = -dxux + (dly + lc[s] * dph[p] * dlx) / (1.0 + ph[p]);
  }
  const double* mN = mom + 9 * (size_t(p) * nl + nl - 1);
  const double* mN1 = mom + 9 * (size_t(p) * nl + nl - 2);
  const double PN = mN[0] * mN[3], PN1 = mN1[0] * mN1[3];
  const double lw = lf[nl], l1 = lc[nl - 1], l2 = lc[nl - 2];
  pw[p] = ((lw - l2) * PN - (lw - l1) * PN1) / (l1 - l2);
}

cudaError_t launch_channel_post(const double* mom, const double* tab, int nl, int nx, double dxi, double* ux,
                                double* uy, double* omega, double* psi, double* pw, cudaStream_t s) {
  channel_post_kernel<<<(nx + 127) / 128, 128, 0, s>>>(mom, tab, nl, nx, dxi, ux, uy, omega, psi, pw);
  return cudaGetLastError();
}

}  // namespace vlb
