// One TVD-RK3 stage of the gradually expanding channel in the vielbein frame
// (Sec. VII.A-C, Eq. canalie_boltz), as a marching kernel: each CTA owns a
// strip of TP adjacent xi-columns and walks up a segment of lambda rows
// (wall-normal, the contiguous direction of the cell index p * n_lambda + s).
// For every row s it
//
//   - pushes row s+3 into a per-thread six-row register window (f', f'') of
//     its (column, velocity), so the lambda-WENO-5 interface value s+1/2
//     comes from registers and every lambda interface is reconstructed once;
//   - reduces the moments of row s+3; two dedicated equilibrium warps turn
//     them into the row's truncated equilibrium (Sec. IV.D) asynchronously,
//     handing rows over through mbarrier rings, two or three rows ahead of use;
//   - reconstructs the xi interfaces of row s from a shared-memory ring that
//     bulk copies (cp.async.bulk, mbarrier completion) fill PD rows ahead;
//   - contracts the momentum-space force matrices of Eq. (canalie_boltz)
//     over the row's cells: in single precision either on the CUDA cores
//     (packed FP32x2 fmas on the reflection-split matrices, run by two extra
//     warps) or on the tensor cores (mma.sync m16n8k8 TF32 with a hi/lo split
//     of both operands, three products per tile), one template instance each,
//     chosen per context by timing; in double precision on the CUDA cores;
//   - combines advection, force, BGK relaxation and the RK3 weights and
//     stores the cell's updated populations straight to global memory.
//
// The march is software-pipelined: step s combines row s-1 while it builds row
// s's interface values and force (double-buffered by row parity), so all warp
// roles work between the one barrier a step takes, and each column warp waits
// for its own bulk copies.
//
// Boundaries: the centreline mirror (Sec. VII.C.3) fills the window at the
// bottom of the march, the diffuse wall (Sec. VII.C.4) at its top with n_w per
// column from the zero-mass-flux balance, and the inlet/outlet reservoirs give
// the xi-halo values past the first and last strip, evaluated by each thread
// whose stencil reaches them.
//
// Distribution buffers hold the deviation D = F - R from the rest state
// (ModelArgs), with (f', f'') interleaved per velocity: a cell row is
// 2 Q0 Q1 reals, element (i, j, d) at 2 (i Q1 + j) + d.
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
static_assert(sizeof(ChanCell<float>) == 48 && sizeof(ChanCell<double>) == 96, "bulk-copied geometry rows");

// Tile counts of the force contractions of one cell on m16n8k8 tensor-core tiles.
// lambda: D = [K0; Kt0] F, rows of the A operand interleaved per m-tile t as
//   (K0 rows 8t..8t+7, Kt0 rows 8t..8t+7), F as the B operand [i'][2 j + d];
// xi: D = F [K1^T | Kt1^T], F as the A operand with rows (i, d) of m-tile t =
//   (8t + r/2, r & 1), the B operand [j'][2 j + e] (e = 0: K1, e = 1: Kt1), j' >= Q1 zero.
template <int Q0, int Q1>
struct ChanShape {
  static constexpr int V = Q0 * Q1;
  static constexpr int ROW = 2 * V;         // reals per cell row
  static constexpr int NWC = V / 32;        // warps per column (one velocity per thread)
  static constexpr int MT = Q0 / 8;         // m-tiles (both contractions)
  static constexpr int KKL = Q0 / 8;        // k-steps of the lambda contraction
  static constexpr int NN = Q1 / 4;         // n-tiles (both contractions)
  static constexpr int KKX = (Q1 + 7) / 8;  // k-steps of the xi contraction
  static constexpr int S = 2 * NN;          // force subtasks per cell (one n-tile each)
  static constexpr int EQW = Q0 + Q1 + 4;   // per-cell equilibrium record: n g0, g1, T, 1/tau, u^xi, pad
  static_assert(V % 32 == 0 && Q0 % 8 == 0 && Q1 % 4 == 0, "velocity set shape of the channel kernel");
  static_assert(Q0 + Q1 <= 32, "one lane per equilibrium factor");
};

// Model tables of a channel context, in device memory, bulk-copied into each
// CTA's shared memory.  gw0/gw1 are the factors of f_eq(1, 0, T0), the wall and
// reservoir equilibrium at rest (they change with T0).
template <typename real, int Q0, int Q1>
struct alignas(16) ChanTables {
  using S = ChanShape<Q0, Q1>;
  uint32_t fl[S::MT][S::KKL][2][32][4];  // lambda A fragments, [hi|lo] TF32 bit patterns
  uint32_t fx[S::KKX][S::NN][2][32][2];  // xi B fragments, [hi|lo]
  real K0[Q0 * Q0], Kt0[Q0 * Q0];        // d/dp^lambda, d/dp^lambda (p^lambda .)
  real K1[Q1 * Q1], Kt1[Q1 * Q1];        // d/dp^xi, d/dp^xi (p^xi .)
  real p0[Q0], p1[Q1], iw0[Q0], iw1[Q1], w0[Q0], w1[Q1];
  real tab0[Q0 * MAXN], tab1[Q1 * MAXN];  // equilibrium tables [k][s]
  real gw0[Q0], gw1[Q1];
  double wall_den;  // sum over p^lambda < 0 of gw0 p^lambda times sum of gw1: incoming flux of f_eq(1, 0, T0)
  double ref_flux_pos;  // sum over p^lambda > 0 of p^lambda R (ModelArgs)
  // sums of R (ModelArgs: n, rho u0, rho u1, energy) as (hi, lo) in the bulk type (lo = 0 in double)
  real ref_hi[4], ref_lo[4];
  int N0, N1, kind0, kind1;
};

// Host-side description of a channel context: grid size, Kn, time step, reservoirs,
// and the flow-rate ends (flow = 1: the parabolic profiles of Q0 replace the reservoirs).
struct ChanDesc {
  int nl, nx;
  double kn, dt, n_in, n_out, T0;
  float knf, dtf, n_inf, n_outf, T0f;
  int flow;
  double q0;
};

template <typename real>
struct ChanArgs {
  const real* Fprev;  // distribution L acts on
  const real* Fl;     // F_l of the step (read when ca != 0)
  real* Fout;
  const void* tables;  // ChanTables of the context's shape
  const ChanCell<real>* geo;
  double* nw;  // per column
  unsigned* err;
  int nl, nx;
  int seglen;  // rows per lambda segment (the last one may be shorter, >= 3 rows)
  int nseg;
  // Fout = F_prev + ca (F_l - F_prev) + ccdt L[F_prev] (see StageArgs)
  real ca, ccdt;
  real ikn, n_in, n_out, T0;  // 1/Kn, reservoir densities, wall and reservoir temperature
  unsigned long long max_polls;
  // flow-rate ends (Sec. VII.C.1-2), when flow != 0: per end e and row s,
  // qflow[(2 e) nl + s] = Q_s (the inflow equilibrium's u^xi) and
  // qflow[(2 e + 1) nl + s] = (1 + phi) Q_s (the particle flux through the end interface)
  const real* qflow;
  int flow;
};

// Shared-memory carve-up of a CTA, identical on host and device.  The ring holds
// rows s-1 .. s+3+PD of the strip, each with its xi-halo (TP + 6 cells): row s-1
// for the geometry of the combine, row s for the xi reconstruction and the force,
// s+3 for the window, and PD rows in flight (bulk copies issued PD steps ahead).
// The xi interface values and the force results are double-buffered by row parity:
// step s writes row s's while it combines row s-1 from the other half.
template <typename real, int Q0, int Q1, int TP>
struct ChanSmem {
  using S = ChanShape<Q0, Q1>;
  using Tab = ChanTables<real, Q0, Q1>;
  static constexpr bool F32 = sizeof(real) == 4;
  static constexpr int NSYNC = (TP + 1) * S::V;  // TP column groups and one extra group, in step
  static constexpr int NT = NSYNC + 64;          // and two equilibrium warps running ahead of them
  static constexpr int NPR = 4;                  // moment-partial ring (rows r .. r+3)
  // prefetch distance in rows: double precision copies each row in the step that needs it,
  // which keeps its larger ring within an SM's shared memory
  static constexpr int PD = F32 ? 2 : 0;
  static constexpr int NRING = 5 + PD;        // ring rows
  static constexpr int NB = PD + 1;           // mbarriers of the step groups (one more for the prologue)
  static constexpr int NEQ = 8;               // equilibrium records (rows s-1 .. s+3 in use), a power of 2
  static constexpr int RC = TP + 6;           // cells of a ring row
  static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t rowb = size_t(S::ROW) * sizeof(real);
  // mbarriers: NB step groups, the prologue, NPR partials-ready, NEQ equilibrium-ready
  static constexpr size_t bar_off = 0;
  static constexpr int NBAR = NB + 1 + NPR + NEQ;
  static constexpr size_t tab_off = 128;
  static constexpr size_t ring_off = al(tab_off + sizeof(Tab));
  static constexpr size_t geo_off = ring_off + size_t(NRING) * RC * rowb;
  static constexpr size_t xif_off = al(geo_off + size_t(NRING) * TP * sizeof(ChanCell<real>));
  static constexpr size_t lbl_off = xif_off + size_t(2) * (TP + 1) * S::V * 2 * sizeof(real);
  static constexpr size_t lbuf_rows = F32 ? 2 * TP : 0;  // force results of two rows (single precision only)
  static constexpr size_t lbx_off = lbl_off + lbuf_rows * rowb;
  static constexpr size_t eq_off = lbx_off + lbuf_rows * rowb;
  static constexpr size_t res_off = al(eq_off + size_t(NEQ) * TP * S::EQW * sizeof(real));
  static constexpr size_t resn_off = al(res_off + size_t(NEQ) * 2 * Q1 * sizeof(real));
  static constexpr size_t mvs_off = al(resn_off + size_t(NEQ) * 2 * sizeof(real));
  static constexpr size_t red_off = al(mvs_off + size_t(TP + 2) * 4 * MAXN * sizeof(real));
  static constexpr size_t wred_off = al(red_off + size_t(NPR) * TP * S::NWC * 4 * sizeof(real));
  static constexpr size_t nwv_off = al(wred_off + size_t(2) * TP * S::NWC * sizeof(real));  // two wall sums
  static constexpr size_t bytes = al(nwv_off + size_t(TP) * sizeof(double));
  static_assert(sizeof(Tab) % 16 == 0, "tables are one bulk copy");
  static_assert(rowb % 16 == 0 && (TP * sizeof(ChanCell<real>)) % 16 == 0, "rows are bulk copies");
  static_assert(ring_off % 16 == 0 && geo_off % 16 == 0, "bulk destinations are 16-byte aligned");
  static_assert(xif_off % 16 == 0 && lbl_off % 16 == 0 && lbx_off % 16 == 0, "pair arrays are aligned");
  static_assert(bar_off + NBAR * sizeof(uint64_t) <= tab_off, "mbarriers fit before the tables");
  static_assert((NEQ & (NEQ - 1)) == 0, "record slots by mask");
  static_assert(TP >= 3, "only the end strips' stencils reach past the inlet / outlet");
  static_assert(NT <= 1024, "one thread per (column, velocity) and an extra group");
};

// Moment vector of the truncated equilibrium on one axis (the recurrences of
// eq_moment_vector) with the loop unrolled to MAXN terms, the 1/l factors as
// constants and one reciprocal of T: no division on the per-cell path.
template <typename R>
__device__ __forceinline__ void eq_moments_fast(int kind, int N, R u, R T, R* m) {
  if (kind == 0) {
    R a = R(1), b = u;
    m[0] = a;
    m[1] = b;
#pragma unroll
    for (int l = 2; l < MAXN; ++l) {
      const R x = (u * b + (T - R(1)) * a) * R(1.0 / l);
      if (l <= N) m[l] = x;
      a = b;
      b = x;
    }
  } else {
    const R iT = rcp_rn(T);
    const R is2T = rsqrt_t(R(2) * T);
    const R g0 = exp_t(-R(0.5) * u * u * iT) * is2T * R(0.56418958354775628695);  // N(0; u, T) = e^.. / sqrt(2 pi T)
    R a = R(0.5) * (R(1) + erf_t<R>(u * is2T));
    R b = u * a + T * g0;
    m[0] = a;
    m[1] = b;
#pragma unroll
    for (int l = 2; l < MAXN; ++l) {
      const R x = u * b + R(l - 1) * T * a;
      if (l <= N) m[l] = x;
      a = b;
      b = x;
    }
  }
}

// Force matrices of the channel split by the reflection of each axis (see
// KArgs): with J the node permutation p -> -p, K0 J = -J K0 and K1 J = -J K1
// (derivatives), Kt0 J = J Kt0 and Kt1 J = J Kt1 (derivatives of p f).  On the
// even and odd parts e_k = f_k + f_Jk, o_k = f_k - f_Jk (k over the first half):
//   P[i][k] = (K[i][k] + K[i][Jk]) / 2,  M[i][k] = (K[i][k] - K[i][Jk]) / 2,
//   odd K:  (K f)_i = P e + M o,  (K f)_Ji = M o - P e;
//   even K: (K f)_i = P e + M o,  (K f)_Ji = P e - M o.
// Every coefficient is duplicated into a pair, the operand of a packed fma over
// (f', f''); the block travels as a kernel parameter, so the coefficients are
// uniform constant-bank operands.
template <int Q0, int Q1>
struct ChanKP {
  static constexpr int H0 = Q0 / 2, H1 = Q1 / 2;
  float2 P0[H0 * H0], M0[H0 * H0], Pt0[H0 * H0], Mt0[H0 * H0];  // K0, Kt0: [i][k]
  float2 P1[H1 * H1], M1[H1 * H1], Pt1[H1 * H1], Mt1[H1 * H1];  // K1, Kt1: [j][k]
};

// lambda force task of column j of one cell on the CUDA cores: out[(i, j)] =
// G_lxx (p^xi_j)^2 (K0 f)_i + G_lxl p^xi_j (Kt0 f)_i for both fields.
template <int Q0, int Q1>
__device__ __forceinline__ void force_lambda_cc(const ChanKP<Q0, Q1>& kp, const float* F, int j, float wa, float wb,
                                                float* out) {
  constexpr int H = Q0 / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 f = p_load(F + 2 * (k * Q1 + j)), g = p_load(F + 2 * ((k + H) * Q1 + j));
    e[k] = p_add(f, g);
    o[k] = p_sub(f, g);
  }
  const float2 WA = p_set(wa), WB = p_set(wb);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float2 A = p_mul(kp.P0[i * H], e[0]), B = p_mul(kp.M0[i * H], o[0]);
    float2 C = p_mul(kp.Pt0[i * H], e[0]), D = p_mul(kp.Mt0[i * H], o[0]);
#pragma unroll
    for (int k = 1; k < H; ++k) {
      A = p_fma(kp.P0[i * H + k], e[k], A);
      B = p_fma(kp.M0[i * H + k], o[k], B);
      C = p_fma(kp.Pt0[i * H + k], e[k], C);
      D = p_fma(kp.Mt0[i * H + k], o[k], D);
    }
    // row i: wa (A + B) + wb (C + D); row Ji: wa (B - A) + wb (C - D)
    p_store(out + 2 * (i * Q1 + j), p_fma(WA, p_add(A, B), p_mul(WB, p_add(C, D))));
    p_store(out + 2 * ((i + H) * Q1 + j), p_fma(WA, p_sub(B, A), p_mul(WB, p_sub(C, D))));
  }
}

// xi force task of row i of one cell on the CUDA cores: out[(i, j)] =
// -G_lxx p^lambda_i (Kt1 f)_j - G_lxl (p^lambda_i)^2 (K1 f)_j for both fields
// (wa = -G_lxx p^lambda_i, wb = -G_lxl (p^lambda_i)^2).
template <int Q0, int Q1>
__device__ __forceinline__ void force_xi_cc(const ChanKP<Q0, Q1>& kp, const float* F, int i, float wa, float wb,
                                            float* out) {
  constexpr int H = Q1 / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 f = p_load(F + 2 * (i * Q1 + k)), g = p_load(F + 2 * (i * Q1 + Q1 - 1 - k));
    e[k] = p_add(f, g);
    o[k] = p_sub(f, g);
  }
  const float2 WA = p_set(wa), WB = p_set(wb);
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float2 A = p_mul(kp.P1[j * H], e[0]), B = p_mul(kp.M1[j * H], o[0]);
    float2 C = p_mul(kp.Pt1[j * H], e[0]), D = p_mul(kp.Mt1[j * H], o[0]);
#pragma unroll
    for (int k = 1; k < H; ++k) {
      A = p_fma(kp.P1[j * H + k], e[k], A);
      B = p_fma(kp.M1[j * H + k], o[k], B);
      C = p_fma(kp.Pt1[j * H + k], e[k], C);
      D = p_fma(kp.Mt1[j * H + k], o[k], D);
    }
    // K1 odd: (K1 f)_j = A + B, (K1 f)_Jj = B - A; Kt1 even: (Kt1 f)_j = C + D, (Kt1 f)_Jj = C - D
    p_store(out + 2 * (i * Q1 + j), p_fma(WA, p_add(C, D), p_mul(WB, p_add(A, B))));
    p_store(out + 2 * (i * Q1 + Q1 - 1 - j), p_fma(WA, p_sub(C, D), p_mul(WB, p_sub(B, A))));
  }
}

// ------------------------------------------------------------------ tensor-core helpers
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo with hi, lo TF32 (hi carries the top 11 significand bits, lo the next 11)
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(__fsub_rn(x, __uint_as_float(hi)));
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Force subtask of one cell on the tensor cores (single precision): n-tile nn of
// the lambda contraction (k < NN) or of the xi contraction (k >= NN), written to
// fl_out (lambda part, pairs) or fx_out (xi part, scalars):
//   lambda: G_lxx (p^xi)^2 K0 f + G_lxl p^xi Kt0 f,
//   xi:    -G_lxx p^lambda Kt1 f - G_lxl (p^lambda)^2 K1 f    (Eq. canalie_boltz).
template <int Q0, int Q1>
__device__ __forceinline__ void force_subtask_tc(const ChanTables<float, Q0, Q1>& tb, const float* F, float glxx,
                                                 float glxl, int k, int lane, float* fl_out, float* fx_out) {
  using S = ChanShape<Q0, Q1>;
  const int g = lane >> 2, tq = lane & 3;
  float acc[S::MT][4];
#pragma unroll
  for (int t = 0; t < S::MT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
  if (k < S::NN) {
    const int nn = k;
#pragma unroll
    for (int kk = 0; kk < S::KKL; ++kk) {
      uint32_t bh0, bl0, bh1, bl1;
      tf32_split(F[(8 * kk + tq) * (2 * Q1) + 8 * nn + g], bh0, bl0);
      tf32_split(F[(8 * kk + tq + 4) * (2 * Q1) + 8 * nn + g], bh1, bl1);
#pragma unroll
      for (int t = 0; t < S::MT; ++t) {
        const uint4 h4 = *reinterpret_cast<const uint4*>(tb.fl[t][kk][0][lane]);
        const uint4 l4 = *reinterpret_cast<const uint4*>(tb.fl[t][kk][1][lane]);
        const uint32_t ah[4] = {h4.x, h4.y, h4.z, h4.w}, alo[4] = {l4.x, l4.y, l4.z, l4.w};
        mma_tf32(acc[t], alo, bh0, bh1);
        mma_tf32(acc[t], ah, bl0, bl1);
        mma_tf32(acc[t], ah, bh0, bh1);
      }
    }
    const int j = 4 * nn + tq;
    const float px = tb.p1[j];
    const float wa = glxx * px * px, wb = glxl * px;
#pragma unroll
    for (int t = 0; t < S::MT; ++t) {
      const int i = 8 * t + g;
      float2 o;
      o.x = fmaf(wa, acc[t][0], wb * acc[t][2]);
      o.y = fmaf(wa, acc[t][1], wb * acc[t][3]);
      *reinterpret_cast<float2*>(fl_out + 2 * (i * Q1 + j)) = o;
    }
  } else {
    const int nn = k - S::NN;
    const int d = g & 1;
#pragma unroll
    for (int kk = 0; kk < S::KKX; ++kk) {
      const uint2 bh = *reinterpret_cast<const uint2*>(tb.fx[kk][nn][0][lane]);
      const uint2 bl = *reinterpret_cast<const uint2*>(tb.fx[kk][nn][1][lane]);
      const int ja = 8 * kk + tq, jb = ja + 4;
#pragma unroll
      for (int t = 0; t < S::MT; ++t) {
        const int ia = 8 * t + (g >> 1), ib = ia + 4;
        const float x0 = ja < Q1 ? F[ia * (2 * Q1) + 2 * ja + d] : 0.0f;
        const float x1 = ja < Q1 ? F[ib * (2 * Q1) + 2 * ja + d] : 0.0f;
        const float x2 = jb < Q1 ? F[ia * (2 * Q1) + 2 * jb + d] : 0.0f;
        const float x3 = jb < Q1 ? F[ib * (2 * Q1) + 2 * jb + d] : 0.0f;
        uint32_t ah[4], alo[4];
        tf32_split(x0, ah[0], alo[0]);
        tf32_split(x1, ah[1], alo[1]);
        tf32_split(x2, ah[2], alo[2]);
        tf32_split(x3, ah[3], alo[3]);
        mma_tf32(acc[t], alo, bh.x, bh.y);
        mma_tf32(acc[t], ah, bl.x, bl.y);
        mma_tf32(acc[t], ah, bh.x, bh.y);
      }
    }
    const int j = 4 * nn + tq;
#pragma unroll
    for (int t = 0; t < S::MT; ++t) {
      const int ia = 8 * t + (g >> 1), ib = ia + 4;
      const float pa = tb.p0[ia], pb = tb.p0[ib];
      fx_out[2 * (ia * Q1 + j) + d] = -fmaf(glxx * pa, acc[t][1], glxl * pa * pa * acc[t][0]);
      fx_out[2 * (ib * Q1 + j) + d] = -fmaf(glxx * pb, acc[t][3], glxl * pb * pb * acc[t][2]);
    }
  }
}

// Geometry of one cell into registers with vector loads (12 reals).
template <typename real>
__device__ __forceinline__ void load_geo(const ChanCell<real>* g, real* o) {
  if constexpr (sizeof(real) == 4) {
    const float4* q = reinterpret_cast<const float4*>(g);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 x = q[k];
      o[4 * k] = x.x, o[4 * k + 1] = x.y, o[4 * k + 2] = x.z, o[4 * k + 3] = x.w;
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(g);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double2 x = q[k];
      o[2 * k] = x.x, o[2 * k + 1] = x.y;
    }
  }
}
enum { G_AM = 0, G_AP, G_BM, G_BP, G_CM, G_CP, G_IDL, G_IDX, G_GLXL, G_GLXX };

// ------------------------------------------------------------------ the stage kernel
// Device cell (s, p) of the channel is s * n_xi + p (xi fastest), so the cells of a
// strip's row and its xi-halo are one contiguous bulk copy.
//
// TC selects the single-precision force contraction: true, the tensor cores
// (mma.sync TF32, three products per tile) on the column-group warps; false,
// packed FP32x2 fmas with the split matrices of kp on the extra warps.  The
// double-precision kernel contracts in FP64 on the column-group threads.
//
// CLB runs the Cartesian-split formulation (Sec. VII.G, Eq. canalie_coord_beq_cons) on the
// same march: momenta (p^x, p^y) on the model's axes, no force term, fluxes of F = D + R, and
// the geometry record read as V^lambda = am p^x - glxl p^y at s - 1/2 and ap p^x - glxx p^y at
// s + 1/2 (a = 1 / (1 + phi), glxl / glxx = a lambda phi' at the interfaces), V^xi = b p^y
// (c = 0).  The lambda upwind side and the wall's incoming half-plane (Eq. canalie_coord_nw)
// then depend on the column and the interface.
template <typename real, int Q0, int Q1, int TP, bool TC, bool CLB = false>
__global__ void __launch_bounds__(ChanSmem<real, Q0, Q1, TP>::NT, 1)
    channel_stage_kernel(const __grid_constant__ ChanArgs<real> a, const __grid_constant__ ChanKP<Q0, Q1> kp) {
  using S = ChanShape<Q0, Q1>;
  using L = ChanSmem<real, Q0, Q1, TP>;
  using Tab = ChanTables<real, Q0, Q1>;
  using P = pair_t<real>;
  constexpr int V = S::V, ROW = S::ROW, NWC = S::NWC, EQW = S::EQW;
  constexpr int NMAIN = TP * V;    // threads of the column groups
  constexpr int NMW = NMAIN / 32;  // their warps
  constexpr int PD = L::PD, NRING = L::NRING, NB = L::NB, RC = L::RC;
  constexpr bool F32 = L::F32;
  extern __shared__ __align__(128) unsigned char smem[];

  constexpr int NSYNC = L::NSYNC;  // threads of the named barrier the step phases use
  const int tid = threadIdx.x, lane = tid & 31;
  const bool is_main = tid < NMAIN;
  const bool is_eqw = tid >= NSYNC;       // the two equilibrium warps
  const int qw = is_eqw ? (tid - NSYNC) >> 5 : -1;
  const int c = is_main ? tid / V : TP;  // column of a main thread; TP marks the extra group
  const int v = is_main ? tid - c * V : (is_eqw ? lane : tid - NMAIN);
  const int i = v / Q1, j = v - i * Q1;
  const int wc = v >> 5;                             // warp within the group
  const int mw = is_main ? tid >> 5 : -1;            // main warp index
  const int ew = is_main ? -1 : (tid - NMAIN) >> 5;  // extra warp index

  const int nl = a.nl, nx = a.nx;
  const int nstrips = nx / TP;
  const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
  const int p0 = strip * TP;
  const int sA = seg * a.seglen, sB = min(sA + a.seglen, nl);
  const bool inlet = p0 == 0, outlet = p0 + TP == nx;
  const bool top = sB == nl;
  const bool need_fl = a.ca != real(0);
  const int rlast = min(sB + 2, nl - 1);  // last row a segment reads
  const int pa = max(p0 - 3, 0), pb = min(p0 + TP + 3, nx);  // xi cells of a ring row in memory

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar_off);  // NB step groups, then the prologue
  uint64_t* pready = bar + NB + 1;     // [NPR] moment partials of row r in slot r % NPR written
  uint64_t* eready = pready + L::NPR;  // [NEQ] equilibrium record of row r in slot r % NEQ written
  const Tab& tb = *reinterpret_cast<const Tab*>(smem + L::tab_off);
  real* ring = reinterpret_cast<real*>(smem + L::ring_off);                      // [NRING][RC][ROW]
  ChanCell<real>* gring = reinterpret_cast<ChanCell<real>*>(smem + L::geo_off);  // [NRING][TP]
  P* xif = reinterpret_cast<P*>(smem + L::xif_off);                              // [TP+1][V]
  real* lbl = reinterpret_cast<real*>(smem + L::lbl_off);                        // [TP][ROW] (single precision)
  real* lbx = reinterpret_cast<real*>(smem + L::lbx_off);                        // [TP][ROW]
  real* eqr = reinterpret_cast<real*>(smem + L::eq_off);                         // [4][TP][EQW]
  real* resr = reinterpret_cast<real*>(smem + L::res_off);                       // [4][2][Q1]
  real* resn = reinterpret_cast<real*>(smem + L::resn_off);                      // [4][2] inflow densities
  real* mvs = reinterpret_cast<real*>(smem + L::mvs_off);                        // [TP+2][4][MAXN]
  real* red = reinterpret_cast<real*>(smem + L::red_off);                        // [NPR][TP][NWC][4]
  real* wred = reinterpret_cast<real*>(smem + L::wred_off);                      // [TP][NWC]
  double* nwv = reinterpret_cast<double*>(smem + L::nwv_off);                    // [TP]

  auto dcell = [&](int s, int p) -> size_t { return size_t(s) * nx + p; };
  // cell cc in [-3, TP + 3) of the ring row in slot k
  auto krow = [&](int k, int cc) -> real* { return ring + size_t(k * RC + cc + 3) * ROW; };
  auto row_bytes = [&]() -> unsigned { return unsigned((pb - pa) * L::rowb + TP * sizeof(ChanCell<real>)); };
  auto row_issue = [&](int r, uint64_t* b) {  // row r with its halo, and its geometry
    const int k = r % NRING;
    bulk_g2s(krow(k, pa - p0), a.Fprev + dcell(r, pa) * ROW, unsigned((pb - pa) * L::rowb), b);
    bulk_g2s(gring + k * TP, a.geo + dcell(r, p0), unsigned(TP * sizeof(ChanCell<real>)), b);
  };

  // ---- prologue: tables and rows sA .. sA+2+PD
  if (tid == 0) {
    for (int b = 0; b <= NB; ++b) mbar_init(bar + b, 1);
    for (int k = 0; k < L::NPR; ++k) mbar_init(pready + k, NMW);
    for (int k = 0; k < L::NEQ; ++k) mbar_init(eready + k, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int rtop = min(sA + 2 + PD, rlast);
  if (tid == NMAIN) {  // one arrival with every byte of the prologue, then the copies
    const unsigned total = unsigned(sizeof(Tab)) + unsigned(rtop - sA + 1) * row_bytes();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar + NB, total);
    bulk_g2s(smem + L::tab_off, a.tables, unsigned(sizeof(Tab)), bar + NB);
    for (int r = sA; r <= rtop; ++r) row_issue(r, bar + NB);
  }
  P W0, W1, W2, W3, W4, W5;  // F(s-3 .. s+2) before the push of step s
  W0 = W1 = W2 = p_set(real(0));
  if (is_main && sA > 0) {  // window rows below the segment (each thread its own populations)
    const real* base = a.Fprev + 2 * v;
    W0 = p_load(base + dcell(sA - 3, p0 + c) * ROW);
    W1 = p_load(base + dcell(sA - 2, p0 + c) * ROW);
    W2 = p_load(base + dcell(sA - 1, p0 + c) * ROW);
  }
  {
    bool ok = true;
    if (tid == 0) ok = mbar_wait(bar + NB, 0, a.max_polls);
    ok = __syncthreads_and(ok);
    if (!ok) {
      if (tid == 0) {
        atomicOr(a.err, ERR_TIMEOUT);
        mbar_wait(bar + NB, 0, a.max_polls);
      }
      __syncthreads();
      return;
    }
  }
  // per-thread constants
  const real pl = tb.p0[i], px = tb.p1[j];
  const real sc = tb.iw0[i] * tb.iw1[j];
  const real Rij = tb.w0[i] * tb.w1[j];
  const bool lpos = pl >= real(0);
  const real T0 = a.T0;

  // moments of row r (main threads): per-warp partial sums of the deviation
  auto moment_partials = [&](P f, int r) {
    const real f1 = f.x, f2 = f.y;
    const real sn = f1, srr = pl * f1, spp = px * f1, se = (pl * pl + px * px) * f1 + f2;
    const bool h16 = lane & 16, h8 = lane & 8;
    real k0 = h16 ? spp : sn, k1 = h16 ? se : srr;
    const real t0 = h16 ? sn : spp, t1 = h16 ? srr : se;
    k0 += __shfl_xor_sync(0xffffffffu, t0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, t1, 16);
    real kq = h8 ? k1 : k0;
    kq += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    kq += __shfl_xor_sync(0xffffffffu, kq, 4);
    kq += __shfl_xor_sync(0xffffffffu, kq, 2);
    kq += __shfl_xor_sync(0xffffffffu, kq, 1);
    // lanes 0, 8, 16, 24: n, rho u0, rho u1, energy
    if ((lane & 7) == 0) red[(((r % L::NPR) * TP + c) * NWC + wc) * 4 + (lane >> 3)] = kq;
  };

  // equilibrium record of cell cc of row r (one extra warp): n, u, T, tau and the
  // factors n g0_i, g1_j normalised so that sum_ij n g0_i g1_j = n (reading 18)
  auto eq_job = [&](int r, int cc) {
    real* mv = mvs + cc * 4 * MAXN;
    const real* rp = red + ((r % L::NPR) * TP + cc) * NWC * 4;
    // cross-warp sums of the partials plus the sums of R; n compensated (float-float)
    // on the single-precision path
    real q[4], nlo = real(0);
    {
      real sn = real(0), e = real(0);
#pragma unroll
      for (int w = 0; w < NWC; ++w) {
        const real x = rp[w * 4];
        if constexpr (F32) {
          float t, er;
          two_sum(sn, x, t, er);
          sn = t;
          e += er;
        } else {
          sn += x;
        }
      }
      if constexpr (F32) {
        float t, er;
        two_sum(sn, tb.ref_hi[0], t, er);
        q[0] = t;
        nlo = er + e + tb.ref_lo[0];
      } else {
        q[0] = sn + tb.ref_hi[0];
      }
    }
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      real sk = real(0);
#pragma unroll
      for (int w = 0; w < NWC; ++w) sk += rp[w * 4 + k];
      q[k] = sk + (tb.ref_hi[k] + tb.ref_lo[k]);
    }
    const real nn = q[0] + nlo;
    const real inn = rcp_rn(nn);
    const real u0 = q[1] * inn, u1 = q[2] * inn;
    const real T = (q[3] * inn - (u0 * u0 + u1 * u1)) * (real(1) / real(3));
    if (lane < 4) {
      const int ax = lane >> 1, side = lane & 1;
      const real u = (ax ? u1 : u0) * (side ? real(-1) : real(1));
      eq_moments_fast<real>(ax ? tb.kind1 : tb.kind0, ax ? tb.N1 : tb.N0, u, T, mv + lane * MAXN);
    }
    __syncwarp();
    real g = real(0);
    if (lane < Q0) {
      const real* m = mv + ((tb.kind0 == 1 && tb.p0[lane] < real(0)) ? 1 : 0) * MAXN;
      for (int s = 0; s <= tb.N0; ++s) g += tb.tab0[lane * MAXN + s] * m[s];
      g *= nn;
    } else if (lane < Q0 + Q1) {
      const int jj = lane - Q0;
      const real* m = mv + (2 + ((tb.kind1 == 1 && tb.p1[jj] < real(0)) ? 1 : 0)) * MAXN;
      for (int s = 0; s <= tb.N1; ++s) g += tb.tab1[jj * MAXN + s] * m[s];
    }
    real s0 = lane < Q0 ? g : real(0), s1 = (lane >= Q0 && lane < Q0 + Q1) ? g : real(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    // scale = n / (s0 s1), n in float-float on the single-precision path
    const real iden = rcp_rn(s0 * s1);
    const real scl = q[0] * iden + nlo * iden;
    real val = g;
    if (lane < Q0) val = g * scl;
    else if (lane == Q0 + Q1) val = T;
    else if (lane == Q0 + Q1 + 1) val = nn * T * a.ikn;  // 1/tau, tau = Kn / (n T) (Eq. canalie_tau)
    else if (lane == Q0 + Q1 + 2) val = u1;
    if (lane < EQW) eqr[((r & (L::NEQ - 1)) * TP + cc) * EQW + lane] = val;
    __syncwarp();
  };

  // inflow factors g_xi(u^xi, T0) of row r at one end: reservoirs, u^xi of the adjacent
  // cell from its moment partials; flow-rate ends, u^xi = Q_s and the density n_s of
  // Eq. (canalie_inlet_s)
  auto res_job = [&](int r, int end) {
    const int cc = end == 0 ? 0 : TP - 1;
    real ures;
    if (a.flow) {
      ures = a.qflow[(2 * end) * nl + r];
    } else {
      const real* rp = red + ((r % L::NPR) * TP + cc) * NWC * 4;
      real sn = real(0), sp = real(0);
#pragma unroll
      for (int w = 0; w < NWC; ++w) sn += rp[w * 4], sp += rp[w * 4 + 2];
      ures = (sp + (tb.ref_hi[2] + tb.ref_lo[2])) * rcp_rn(sn + (tb.ref_hi[0] + tb.ref_lo[0]));
    }
    real* mv = mvs + (TP + end) * 4 * MAXN;
    if (lane < 2) eq_moments_fast<real>(tb.kind1, tb.N1, lane ? -ures : ures, T0, mv + lane * MAXN);
    __syncwarp();
    if (lane < Q1) {
      const real* m = mv + ((tb.kind1 == 1 && tb.p1[lane] < real(0)) ? 1 : 0) * MAXN;
      real g = real(0);
      for (int s = 0; s <= tb.N1; ++s) g += tb.tab1[lane * MAXN + s] * m[s];
      resr[((r & (L::NEQ - 1)) * 2 + end) * Q1 + lane] = g;
    }
    __syncwarp();
    if (a.flow) {
      // n_s sum_{entering} V f'_eq(1, (0, Q_s), T0) + sum_{leaving} V f'_adjacent = (1 + phi) Q_s,
      // V = b p^xi - c p^lambda of the end interface (the decision of end_ghost);
      // the adjacent cell is row r of the ring (its slot is refilled only after this row's
      // record is waited for), FP64 sums as for n_w
      const int k = r % NRING;
      const ChanCell<real>& gk = gring[k * TP + cc];
      const real bb = end == 0 ? gk.bm : gk.bp, cq = end == 0 ? gk.cm : gk.cp;
      const real* Fa = krow(k, cc);
      const real* gr = resr + ((r & (L::NEQ - 1)) * 2 + end) * Q1;
      double lv = 0.0, en = 0.0;
      for (int vv = lane; vv < V; vv += 32) {
        const int ii = vv / Q1, jj = vv - ii * Q1;
        const real Vx = bb * tb.p1[jj] - cq * tb.p0[ii];
        const bool into = end == 0 ? (Vx > real(0)) : (Vx < real(0));
        if (into) en += double(Vx) * double(tb.gw0[ii] * gr[jj]);
        else lv += double(Vx) * (double(Fa[2 * vv]) + double(tb.w0[ii]) * double(tb.w1[jj]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lv += __shfl_xor_sync(0xffffffffu, lv, o);
        en += __shfl_xor_sync(0xffffffffu, en, o);
      }
      if (lane == 0) resn[(r & (L::NEQ - 1)) * 2 + end] = real((double(a.qflow[(2 * end + 1) * nl + r]) - lv) / en);
      __syncwarp();
    }
  };
  auto res_jobs = [&](int r) {  // equilibrium warps: both ends where the strip has one
    for (int end = 0; end < 2; ++end)
      if ((end == 0 ? inlet : outlet) && qw == end) res_job(r, end);
  };

  // xi-halo value of velocity (ii, jj) of row r beyond strip end `end` (the inlet / outlet
  // reservoirs): populations entering the domain see f_eq(n_res, (0, u^xi), T0) - R, the
  // others the adjacent cell (zeroth order).  Every thread whose stencil reaches past an
  // end evaluates it itself; the bulk copy leaves those cells out.
  auto end_ghost = [&](int r, int end, int ii, int jj) -> P {
    const int k = r % NRING, ce = end == 0 ? 0 : TP - 1;
    real gm[12];
    load_geo(gring + k * TP + ce, gm);
    const real pli = tb.p0[ii], pxj = tb.p1[jj];
    const real Vx = end == 0 ? gm[G_BM] * pxj - gm[G_CM] * pli : gm[G_BP] * pxj - gm[G_CP] * pli;
    const bool inflow = end == 0 ? (Vx > real(0)) : (Vx < real(0));
    if (inflow) {
      const int e8 = (r & (L::NEQ - 1)) * 2 + end;
      const real nres = a.flow ? resn[e8] : (end == 0 ? a.n_in : a.n_out);
      const real e = nres * tb.gw0[ii] * resr[e8 * Q1 + jj];
      const real R = tb.w0[ii] * tb.w1[jj];
      return p_make(e - R, e * T0 - R);
    }
    return p_load(krow(k, ce) + 2 * (ii * Q1 + jj));
  };
  // the upwind-ordered five-cell stencil of xi interface cl - 1/2 of ring slot k (cells
  // cl-3 .. cl+1 when up, cl+2 .. cl-2 otherwise), with the reservoir ghosts at the ends
  auto xi_stencil = [&](int r, int k, int cl, bool up, int vv, P* h) {
    const int ii = vv / Q1, jj = vv - ii * Q1;
    const int c0 = up ? cl - 3 : cl + 2, sd = up ? 1 : -1;
    if (!((inlet && cl < 3) || (outlet && cl > TP - 3))) {  // no end within reach (warp-uniform)
#pragma unroll
      for (int q = 0; q < 5; ++q) h[q] = p_load(krow(k, c0 + q * sd) + 2 * vv);
      return;
    }
    const P gin = inlet ? end_ghost(r, 0, ii, jj) : p_set(real(0));
    const P gout = outlet ? end_ghost(r, 1, ii, jj) : p_set(real(0));
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int cc = c0 + q * sd;
      h[q] = (inlet && cc < 0) ? gin : (outlet && cc >= TP) ? gout : p_load(krow(k, cc) + 2 * vv);
    }
  };

  // xi interface TP - 1/2 of row s (the right edge of the strip) for the 32 velocities of chunk ch
  auto edge_weno = [&](int r, int k, int ch, P* xo) {
    const int vv = 32 * ch + lane, ii = vv / Q1, jj = vv - ii * Q1;
    const real pli = tb.p0[ii], pxj = tb.p1[jj];
    real gm[12];
    load_geo(gring + k * TP + TP - 1, gm);
    const bool up = gm[G_BP] * pxj - gm[G_CP] * pli >= real(0);
    P h[5];
    xi_stencil(r, k, TP, up, vv, h);
    xo[TP * V + vv] = weno5p<real>(h[0], h[1], h[2], h[3], h[4], tb.iw0[ii] * tb.iw1[jj]);
  };

  // window rows from the ring (the centreline mirror below row 0: ghost 1-k of
  // cell k, p^lambda -> -p^lambda, Sec. VII.C.3)
  if (is_main) {
    if (sA == 0) {
      const int ib = refl(1, Q0, i);
      W0 = p_load(krow(2 % NRING, c) + 2 * (ib * Q1 + j));
      W1 = p_load(krow(1 % NRING, c) + 2 * (ib * Q1 + j));
      W2 = p_load(krow(0, c) + 2 * (ib * Q1 + j));
    }
    W3 = p_load(krow(sA % NRING, c) + 2 * v);
    W4 = p_load(krow((sA + 1) % NRING, c) + 2 * v);
    W5 = p_load(krow((sA + 2) % NRING, c) + 2 * v);
  }
  // moments of rows sA .. sA+2, equilibria and reservoir factors of rows sA, sA+1
  // (row sA+2's come in the first step)
  for (int r = sA; r < min(sA + 3, sB); ++r) {
    if (is_main) moment_partials(p_load(krow(r % NRING, c) + 2 * v), r);
    __syncthreads();
    if (is_eqw && r < sA + 2) {
      for (int job = qw; job < TP; job += 2) eq_job(r, job);
      res_jobs(r);
    }
    __syncthreads();
  }
  // row sA+2's partials are the first the equilibrium warps take from the ring
  if (is_main && sA + 2 < min(nl, sB) && lane == 0) mbar_arrive(pready + (sA + 2) % L::NPR);
  // lambda interface r - 1/2 from the window W0 .. W5 = F(r-3 .. r+2), upwind by V^lambda: the sign
  // of p^lambda (vielbein), or of V^lambda = am p^x - glxl p^y of row r's record (Cartesian split)
  auto lam_face = [&](const ChanCell<real>& g, bool lower) -> P {
    if constexpr (CLB) {
      const bool up = (lower ? g.am * pl - g.glxl * px : g.ap * pl - g.glxx * px) >= real(0);
      return weno5p<real>(up ? W0 : W5, up ? W1 : W4, up ? W2 : W3, up ? W3 : W2, up ? W4 : W1, sc);
    } else {
      (void)g, (void)lower;
      return lpos ? weno5p<real>(W0, W1, W2, W3, W4, sc) : weno5p<real>(W5, W4, W3, W2, W1, sc);
    }
  };
  P fm = p_set(real(0));
  if (is_main) fm = lam_face(gring[(sA % NRING) * TP + c], true);
  P gh0 = p_set(real(0)), gh1 = p_set(real(0));  // wall ghosts of rows nl, nl+1 (and nl+2)
  bool wout = false;                              // this velocity leaves through the wall
  __syncthreads();

  // ---- the equilibrium warps: rows sA+2 .. in order, each as soon as the column warps have
  // reduced its moments, two or three rows ahead of the step that uses it; they take part in
  // no step barrier (the step phases synchronise on named barrier 1 of the other NSYNC threads)
  const int rend = min(nl, sB);
  if (is_eqw) {
    unsigned pph = 0;
    for (int r = sA + 2; r < rend; ++r) {
      const int k = r % L::NPR;
      bool ok = true;
      if (lane == 0) ok = mbar_wait(pready + k, (pph >> k) & 1u, a.max_polls);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      pph ^= 1u << k;
      if (!ok) {  // the column warps stopped (their own wait ran out): leave
        if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
        return;
      }
      __syncwarp();
      for (int job = qw; job < TP; job += 2) eq_job(r, job);
      res_jobs(r);
      __syncwarp();
      if (lane == 0) mbar_arrive(eready + (r & (L::NEQ - 1)));
    }
    return;
  }
  unsigned eph = 0;          // thread 0: parity of the next wait, per equilibrium-ready slot
  int eq_waited = sA + 1;    // rows up to this one have their records (the prologue made sA, sA+1)
  unsigned phase_bits = 0;   // main threads: parity of the next wait, per step mbarrier
  bool good = true;          // every wait of this thread so far ended in time
  P flr = p_set(real(0));    // F_l of the row being finished, prefetched one step ahead
  if (is_main && need_fl) flr = p_load(a.Fl + dcell(sA, p0 + c) * ROW + 2 * v);
  P fp = p_set(real(0));     // lambda interface s + 1/2 of the row whose interfaces were built last
  P frc = p_set(real(0));    // force of that row (double-precision path)
  auto sync_all = [&]() { named_bar(1, NSYNC); };
  auto sync_and = [&](bool v) { return named_bar_and(1, NSYNC, v); };

  // combine of cell (r, c) (main threads), once row r's interface values and force are
  // written (the step barrier after row r's step): F(r) = W2, lambda interfaces r -/+ 1/2 in
  // fm / fp, xi interfaces and force from the row-parity half of the buffers
  auto combine = [&](int r) {
    real gm[12];
    load_geo(gring + (r % NRING) * TP + c, gm);
    const P* xb = xif + (r & 1) * (TP + 1) * V;
    const P FL = xb[c * V + v], FR = xb[(c + 1) * V + v];
    const real Vm = gm[G_BM] * px - gm[G_CM] * pl, Vp = gm[G_BP] * px - gm[G_CP] * pl;
    P adv;
    if constexpr (CLB) {
      // Eq. (canalie_coord_beq_cons): fluxes of F = D + R, V^lambda per interface (no force term
      // balances the rest state's advection here)
      const P R2 = p_set(Rij);
      const real Vlm = gm[G_AM] * pl - gm[G_GLXL] * px, Vlp = gm[G_AP] * pl - gm[G_GLXX] * px;
      adv = p_mul(p_set(gm[G_IDL]), p_sub(p_mul(p_set(Vlp), p_add(fp, R2)), p_mul(p_set(Vlm), p_add(fm, R2))));
      adv = p_fma(p_set(gm[G_IDX]), p_sub(p_mul(p_set(Vp), p_add(FR, R2)), p_mul(p_set(Vm), p_add(FL, R2))), adv);
    } else {
      // chi flux differences (Sec. VII.B)
      adv = p_mul(p_set(pl * gm[G_IDL]), p_sub(p_mul(p_set(gm[G_AP]), fp), p_mul(p_set(gm[G_AM]), fm)));
      adv = p_fma(p_set(gm[G_IDX]), p_sub(p_mul(p_set(Vp), FR), p_mul(p_set(Vm), FL)), adv);
    }
    if constexpr (F32 && !CLB) {
      const real* lb = lbl + (r & 1) * TP * ROW;
      const real* lx = lbx + (r & 1) * TP * ROW;
      frc = p_add(p_load(lb + c * ROW + 2 * v), p_load(lx + c * ROW + 2 * v));
    }
    const real* rec = eqr + ((r & (L::NEQ - 1)) * TP + c) * EQW;
    const real geq = rec[i] * rec[Q0 + j];
    const P deq = p_make(geq - Rij, geq * rec[Q0 + Q1] - Rij);
    const real itau = rec[Q0 + Q1 + 1];
    const P F = W2;  // F(r)
    // L = -advection + force - (F - f_eq) / tau
    const P Lv = p_sub(p_sub(frc, adv), p_mul(p_set(itau), p_sub(F, deq)));
    P o = p_fma(p_set(a.ccdt), Lv, F);
    if (need_fl) o = p_fma(p_set(a.ca), p_sub(flr, F), o);
    p_store(a.Fout + dcell(r, p0 + c) * ROW + 2 * v, o);
    if (need_fl && r + 1 < sB) flr = p_load(a.Fl + dcell(r + 1, p0 + c) * ROW + 2 * v);
  };

  // ---- the march: step s finishes row s-1 (the combine) while it builds row s's interface
  // values and force; one barrier per step, after which row s's outputs are complete.  The
  // last pass (s = sB) only finishes row sB-1.
  for (int s = sA; s <= sB; ++s) {
    const bool build = s < sB;
    const int k0 = s % NRING, k3 = (s + 3) % NRING;
    if (build && is_main && s - PD >= sA && s + 3 <= rlast) {  // the group issued PD steps ago brought row s+3
      const int b = (s - PD) % NB;
      good = mbar_wait(bar + b, (phase_bits >> b) & 1u, a.max_polls) && good;
      phase_bits ^= 1u << b;
    }
    if (build && tid == NMAIN && s + 3 + PD <= rlast) {  // row s+3+PD into the slot row s-2 left
      uint64_t* b = bar + s % NB;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(b, row_bytes());
      row_issue(s + 3 + PD, b);
    }
    // the wall (Sec. VII.C.4): at the first row whose window reaches it, n_w per
    // column from the zero-mass-flux balance and the ghosts of rows nl .. nl+2
    if (build && top && s == nl - 3) {
      if (is_main) {
        // W3 .. W5 = F(nl-3 .. nl-1); outgoing populations: quadratic extrapolation (Eq. extrapol)
        const P G0 = p_add(p_sub(p_mul(p_set(real(3)), W5), p_mul(p_set(real(3)), W4)), W3);
        const P G1 = p_add(p_sub(p_mul(p_set(real(6)), W5), p_mul(p_set(real(8)), W4)), p_mul(p_set(real(3)), W3));
        real fl = real(0), fd = real(0);
        if constexpr (CLB) {
          // V^lambda at the wall interface (row nl-1's upper face); the outgoing flux is of F = D + R,
          // the incoming one of f_eq(1, 0, T0), both over this column's half-planes (Eq. canalie_coord_nw)
          const ChanCell<real>& gw = gring[((nl - 1) % NRING) * TP + c];
          const real Vw = gw.ap * pl - gw.glxx * px;
          if (Vw > real(0)) fl = (weno5p<real>(W3, W4, W5, G0, G1, sc).x + Rij) * Vw;
          else fd = tb.gw0[i] * tb.gw1[j] * Vw;
          wout = Vw > real(0);
        } else {
          if (pl > real(0)) fl = weno5p<real>(W3, W4, W5, G0, G1, sc).x * pl;
          wout = pl > real(0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fl += __shfl_xor_sync(0xffffffffu, fl, o);
          if constexpr (CLB) fd += __shfl_xor_sync(0xffffffffu, fd, o);
        }
        if (lane == 0) wred[c * NWC + wc] = fl, wred[(TP + c) * NWC + wc] = fd;
        gh0 = G0;
        gh1 = G1;
      }
      sync_all();
      if (!is_main && lane == 0)
        for (int cc = ew; cc < TP; cc += NWC) {
          double num = CLB ? 0.0 : tb.ref_flux_pos;  // vielbein: the outgoing flux of R, then of D
          double den = CLB ? 0.0 : tb.wall_den;
          for (int w = 0; w < NWC; ++w) {
            num += double(wred[cc * NWC + w]);
            if (CLB) den += double(wred[(TP + cc) * NWC + w]);
          }
          const double nwc = -num / den;  // Eq. (nw) / (canalie_coord_nw)
          nwv[cc] = nwc;
          a.nw[p0 + cc] = nwc;
          if (!isfinite(nwc)) atomicOr(a.err, ERR_NONFINITE);
        }
      sync_all();
      if (is_main && !wout) {  // incoming: f_eq(n_w, 0, T0) - R (Eq. weno_populate)
        const real e = real(nwv[c]) * tb.gw0[i] * tb.gw1[j];
        gh0 = gh1 = p_make(e - Rij, e * T0 - Rij);
      }
    }
    if (is_main && s > sA) {
      combine(s - 1);
      fm = fp;
    }
    if (!build) break;

    // ==== row s: interface values and force, into the row-parity half of the buffers
    P* xo = xif + (s & 1) * (TP + 1) * V;
    real* lo = lbl + (s & 1) * TP * ROW;
    real* xo2 = lbx + (s & 1) * TP * ROW;
    if (is_main) {
      const int rn = s + 3;
      const P fnew = rn < nl ? p_load(krow(k3, c) + 2 * v) : (rn == nl ? gh0 : gh1);
      if (rn < rend) {
        moment_partials(fnew, rn);
        __syncwarp();
        if (lane == 0) mbar_arrive(pready + rn % L::NPR);  // the equilibrium warps take row rn from here
      }
      W0 = W1, W1 = W2, W2 = W3, W3 = W4, W4 = W5, W5 = fnew;  // W = F(s-2 .. s+3)
      real gm[12];
      load_geo(gring + k0 * TP + c, gm);
      // xi interface c - 1/2: upwind by V^xi = b p^xi - c p^lambda (Eq. canalie_V)
      const bool up = gm[G_BM] * px - gm[G_CM] * pl >= real(0);
      P h[5];
      xi_stencil(s, k0, c, up, v, h);
      const P FL = weno5p<real>(h[0], h[1], h[2], h[3], h[4], sc);
      // lambda interface s + 1/2 from the window, upwind by p^lambda (a > 0): independent of
      // the xi one, so the two interleave
      fp = lam_face(gring[k0 * TP + c], false);
      xo[c * V + v] = FL;
      if constexpr (CLB) {
        // no force term
      } else if constexpr (F32 && TC) {
        // force subtasks of the row's cells on the tensor cores (mma.sync needs the
        // warp converged after the data-dependent WENO branches)
        __syncwarp();
        for (int t = mw; t < TP * S::S; t += NMW) {
          const int cc = t / S::S, kt = t - cc * S::S;
          const ChanCell<real>& gk = gring[k0 * TP + cc];
          force_subtask_tc<Q0, Q1>(tb, krow(k0, cc), gk.glxx, gk.glxl, kt, lane, lo + cc * ROW, xo2 + cc * ROW);
        }
      } else if constexpr (!F32) {
        const real* F = krow(k0, c);
        P s0 = p_set(real(0)), s1 = p_set(real(0)), s2 = p_set(real(0)), s3 = p_set(real(0));
        for (int ip = 0; ip < Q0; ++ip) {
          const P f = p_load(F + 2 * (ip * Q1 + j));
          s0 = p_fma(p_set(tb.K0[i * Q0 + ip]), f, s0);
          s1 = p_fma(p_set(tb.Kt0[i * Q0 + ip]), f, s1);
        }
        for (int jp = 0; jp < Q1; ++jp) {
          const P f = p_load(F + 2 * (i * Q1 + jp));
          s2 = p_fma(p_set(tb.K1[j * Q1 + jp]), f, s2);
          s3 = p_fma(p_set(tb.Kt1[j * Q1 + jp]), f, s3);
        }
        // G_lxx [(p^xi)^2 K0 f - p^lambda Kt1 f] - G_lxl [(p^lambda)^2 K1 f - p^xi Kt0 f]
        const P A = p_fma(p_set(px * px), s0, p_mul(p_set(-pl), s3));
        const P B = p_fma(p_set(pl * pl), s2, p_mul(p_set(-px), s1));
        frc = p_fma(p_set(gm[G_GLXX]), A, p_mul(p_set(-gm[G_GLXL]), B));
      }
    } else if constexpr (F32 && !TC && !CLB) {
      // force tasks of the row's cells on the CUDA cores (lambda: one per (cell, column
      // j); xi: one per (cell, row i)) in units of 32 (one warp), then the strip's
      // right-edge xi interface, over the extra warps
      constexpr int NTL = TP * Q1, NTX = TP * Q0;
      constexpr int NWL = (NTL + 31) / 32, NWX = (NTX + 31) / 32;
      for (int u = ew; u < NWL + NWX + NWC; u += NWC) {
        if (u < NWL) {
          const int t = 32 * u + lane;
          if (t < NTL) {
            const int cc = t / Q1, jj = t - cc * Q1;
            const ChanCell<real>& gk = gring[k0 * TP + cc];
            const float pxj = tb.p1[jj];
            force_lambda_cc<Q0, Q1>(kp, krow(k0, cc), jj, gk.glxx * pxj * pxj, gk.glxl * pxj, lo + cc * ROW);
          }
        } else if (u < NWL + NWX) {
          const int t = 32 * (u - NWL) + lane;
          if (t < NTX) {
            const int cc = t / Q0, ii = t - cc * Q0;
            const ChanCell<real>& gk = gring[k0 * TP + cc];
            const float pli = tb.p0[ii];
            force_xi_cc<Q0, Q1>(kp, krow(k0, cc), ii, -gk.glxx * pli, -gk.glxl * pli * pli, xo2 + cc * ROW);
          }
        } else {
          edge_weno(s, k0, u - NWL - NWX, xo);
        }
      }
    } else {
      // the strip's right-edge xi interface of row s, 32 velocities per extra warp
      for (int ch = ew; ch < NWC; ch += NWC) edge_weno(s, k0, ch, xo);
    }
    // the step barrier; before it, the records of rows s (the next combine) and s+1 (the
    // reservoir ghosts of the next step) must be written
    {
      const int want = min(s + 1, rend - 1);
      if (tid == 0)
        while (eq_waited < want) {
          const int r = ++eq_waited, k = r & (L::NEQ - 1);
          good = mbar_wait(eready + k, (eph >> k) & 1u, a.max_polls) && good;
          eph ^= 1u << k;
        }
      if (!sync_and(good)) {
        // a wait ran out: wait (bounded) for the bulk copies still in flight -- the groups
        // issued at steps s-PD .. s (the one waited for this step may be the late one) --
        // then leave together
        if (tid == 0) {
          atomicOr(a.err, ERR_TIMEOUT);
          for (int g = s - PD; g <= s; ++g)
            if (g >= sA && g + 3 + PD <= rlast) {
              const int b = g % NB;
              mbar_wait(bar + b, g == s - PD ? ((phase_bits >> b) & 1u) ^ 1u : (phase_bits >> b) & 1u, a.max_polls);
            }
        }
        sync_all();
        return;
      }
    }
  }
}

}  // namespace vlb
