// Device-side building blocks shared by the libvlb kernels: descriptors,
// WENO-5 interface values, equilibrium moment vectors, bounded mbarrier waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vlb {

constexpr int MAXQ = 32;  // nodes per momentum axis
constexpr int MAXN = 8;   // equilibrium expansion order + 1

// Error bits set by kernels in a device word the host reads back.
enum : unsigned { ERR_TIMEOUT = 1u, ERR_NONFINITE = 2u };

struct InstDesc {
  long long cell0;  // first global cell of the instance
  int n_cells;
  int tau_mode;     // vlb_tau_mode
  double kn, dt;
  double u_in, T_in, u_out, T_out;  // walls: tangential speed, temperature
  float kn_f, dt_f;                 // single-precision copies
  int halo;                         // bit e set: end e (0 inner, 1 outer) is a slab halo, not a wall
  int pad;
};

// Diffuse-wall equilibrium f_eq(1, (0, u_w), T_w) of one wall (Eq. weno_populate):
// its factors per axis and its incoming particle flux, sum over the incoming
// half of g0_i p_i times sum_j g1_j.  They depend on the wall only, so the host
// computes them when the walls are set.
struct WallEq {
  double g0[MAXQ], g1[MAXQ];
  double in_flux;
  double pad;
};

struct TileDesc {
  int inst;
  int c0;  // first cell (within the instance) owned by the tile
  int nc;  // cells owned (1 .. the kernel's TC)
};

// (f', f'') pair of one velocity in the bulk type (see the pair operations below).
template <typename real>
struct PairOf;
template <>
struct PairOf<float> {
  using type = float2;
};
template <>
struct PairOf<double> {
  using type = double2;
};
template <typename real>
using pair_t = typename PairOf<real>::type;

// Per-cell chi-formulation factors (Eqs. flux_kom_R, flux_kom_eta):
//   advection = p^R (cp * Flux_{s+1/2} - cm * Flux_{s-1/2}),
//   cp = 2 R_{s+1/2} / (R_{s+1/2}^2 - R_{s-1/2}^2), cm = 2 R_{s-1/2} / (...),
//   inv_rbar = 2 / (R_{s+1/2} + R_{s-1/2}) multiplies the inertial force.
struct GeoCell {
  double cp, cm, inv_rbar, wres;
};

// Single-precision copy of the advection and force factors (cp, cm, inv_rbar, unused).
struct GeoCellF {
  float cp, cm, inv_rbar, pad;
};

// Momentum-space tables of the model (copied into shared memory by each CTA).
struct ModelArgs {
  int nq0, nq1, N0, N1, kind0, kind1;
  double p0[MAXQ], p1[MAXQ];
  double w0[MAXQ], w1[MAXQ];  // quadrature weights
  double tab0[MAXQ * MAXN], tab1[MAXQ * MAXN];  // [k][s] with stride MAXN
  float tab0f[MAXQ * MAXN], tab1f[MAXQ * MAXN];  // single-precision copies for the FP32-bulk path
  float p0f[MAXQ], p1f[MAXQ], iw0f[MAXQ], iw1f[MAXQ];  // nodes and inverse weights, single precision
  double iw0[MAXQ], iw1[MAXQ];                         // inverse weights, double precision
  float w0f[MAXQ], w1f[MAXQ];                          // weights, single precision
  // Device distributions hold the deviation D = F - R from the rest state
  // R_ij = w0_i w1_j (f_eq(1, 0, 1), the same for f' and f'').  R is a steady
  // state of the discrete equations (advection and force cancel on it, BGK
  // vanishes) and WENO-5 is unchanged by adding a constant, so the stage
  // operator applied to D is the operator applied to F; storing D keeps the
  // rounding of each update relative to |F - R| instead of |F|.  Sums of R:
  double ref_n, ref_r, ref_p, ref_e;  // sum R, sum p0 R, sum p1 R, sum (p0^2 + p1^2) R + sum R
  double ref_sum_f;                   // sum of the single-precision products float(w0_i) float(w1_j)
  double ref_flux_pos, ref_flux_neg;  // sum over p0 > 0 (p0 < 0) of p0 R
  // single-precision copies: ref_n and ref_sum_f as (hi, lo) float pairs, the others rounded
  float ref_nf[2], ref_sumf[2];
  float ref_rf, ref_pf, ref_ef;
};

// Momentum-space kernels of the inertial force (Eq. boltz_couette_kom): K0 =
// d/dp^0 on axis 0 and Kt1 = d/dp^1 (p^1 .) on axis 1.  The generic kernels read
// the full matrices; the fixed-shape kernels read the split blocks below (as
// duplicated pairs in single precision).  The split uses that each commutes with the
// reflection of its axis, up to sign: with J the node permutation p_k -> -p_k
// (see refl), K0 J = -J K0 and Kt1 J = J Kt1.  Each then splits into two
// half-size blocks acting on the even and odd parts e_k = f_k + f_Jk,
// o_k = f_k - f_Jk (k over the first half of the nodes):
//   P[i][k] = (K[i][k] + K[i][Jk]) / 2,   M[i][k] = (K[i][k] - K[i][Jk]) / 2,
//   axis 0: (K0 f)_i = P e + M o,  (K0 f)_Ji = M o - P e;
//   axis 1: (Kt1 f)_j = P e + M o, (Kt1 f)_Jj = P e - M o.
template <typename real>
struct KArgs {
  static constexpr int HQ = MAXQ / 2;
  struct Full {
    real K0[MAXQ * MAXQ];   // [i][i'] stride MAXQ
    real Kt1[MAXQ * MAXQ];  // [j][j'] stride MAXQ
  };
  struct Split {
    real P0[HQ * HQ], M0[HQ * HQ];  // [i][k] stride HQ
    real P1[HQ * HQ], M1[HQ * HQ];  // [j][k] stride HQ
  };
  struct SplitPairs {  // the same blocks with every coefficient duplicated, for packed
    pair_t<real> P0[HQ * HQ], M0[HQ * HQ];  // contraction of both fields of a velocity
    pair_t<real> P1[HQ * HQ], M1[HQ * HQ];
  };
  union {
    Full full;
    Split split;
    SplitPairs pairs;
  };
};

// Index of the node at -p_k on an axis of nq nodes: half-range axes list the
// positive nodes first and their mirror images after them (kind 1); full-range
// axes are symmetric about their middle (kind 0).
__host__ __device__ __forceinline__ int refl(int kind, int nq, int k) {
  return kind == 1 ? (k < nq / 2 ? k + nq / 2 : k - nq / 2) : nq - 1 - k;
}

// Type-exact helpers: float arguments must not be promoted to double (the
// FP64 pipe of GB300 runs at a small fraction of the FP32 rate).
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
// 1 / x correctly rounded (single precision: the reciprocal intrinsic, cheaper than a division).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return 1.0 / x; }
// x / y; single precision uses the fast divide (2 ulp), valid for |y| < 2^126.
__device__ __forceinline__ float vdiv(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double vdiv(double x, double y) { return x / y; }

// ---------------------------------------------------------------- WENO-5
// Interface value from the upwind-ordered stencil (a, b, c, d, e) =
// (F_{s-2}, F_{s-1}, F_s, F_{s+1}, F_{s+2}) (Eqs. weno5_flux, weno5_omega,
// weno_sigma) with the epsilon-free weights delta_q / sigma_q^2.
//
// The normalised weights do not change when the stencil is multiplied by a
// constant, so the indicators are computed on the stencil times sc (callers
// pass 1 / (w_i w_j), which brings the weighted populations of every velocity
// to order one and keeps sigma_q inside the single-precision range).  The
// weights are evaluated as delta_q prod_{r != q} sigma_r^2 over their sum,
// with the indicators scaled by their maximum; this form is exact for one
// vanishing indicator (Table IV: that stencil gets weight one).  When the
// products all vanish or are not finite -- two or three zero indicators
// (Table IV), or products below the single-precision range -- a slow path
// uses Table IV for exact zeros and delta_q (sigma_min / sigma_q)^2 otherwise.
template <typename real>
__device__ __noinline__ void weno5_weights_slow(real s1, real s2, real s3, real* w) {
  const real d1 = real(0.1), d2 = real(0.6), d3 = real(0.3);
  if (s1 == real(0) || s2 == real(0) || s3 == real(0)) {
    w[0] = s1 == real(0) ? d1 : real(0);
    w[1] = s2 == real(0) ? d2 : real(0);
    w[2] = s3 == real(0) ? d3 : real(0);
  } else {  // IEEE division: the indicators here may be subnormal or beyond 2^126
    const real mn = vmin(s1, vmin(s2, s3));
    const real r1 = mn / s1, r2 = mn / s2, r3 = mn / s3;
    w[0] = d1 * r1 * r1;
    w[1] = d2 * r2 * r2;
    w[2] = d3 * r3 * r3;
  }
}

template <typename real>
__device__ __forceinline__ real weno5(real a, real b, real c, real d, real e, real sc) {
  const real k1312 = real(13) / real(12), q = real(0.25);
  const real d1 = real(0.1), d2 = real(0.6), d3 = real(0.3);
  const real F1 = a * (real(1) / real(3)) - b * (real(7) / real(6)) + c * (real(11) / real(6));
  const real F2 = -b * (real(1) / real(6)) + c * (real(5) / real(6)) + d * (real(1) / real(3));
  const real F3 = c * (real(1) / real(3)) + d * (real(5) / real(6)) - e * (real(1) / real(6));
  const real A = a * sc, B = b * sc, Cc = c * sc, D = d * sc, E = e * sc;
  real t = A - real(2) * B + Cc;
  real u = A - real(4) * B + real(3) * Cc;
  real s1 = k1312 * t * t + q * u * u;
  t = B - real(2) * Cc + D;
  u = B - D;
  real s2 = k1312 * t * t + q * u * u;
  t = Cc - real(2) * D + E;
  u = real(3) * Cc - real(4) * D + E;
  real s3 = k1312 * t * t + q * u * u;
  const real r = vdiv(real(1), vmax(s1, vmax(s2, s3)));
  const real x1 = s1 * r, x2 = s2 * r, x3 = s3 * r;
  const real P = x1 * x1, Qv = x2 * x2, R = x3 * x3;
  real w1 = d1 * (Qv * R), w2 = d2 * (P * R), w3 = d3 * (P * Qv);
  real den = w1 + w2 + w3;
  if (!(den > real(0)) || !(den < real(1e30))) {
    real w[3];
    weno5_weights_slow<real>(s1, s2, s3, w);
    w1 = w[0], w2 = w[1], w3 = w[2];
    den = w1 + w2 + w3;
  }
  return vdiv(w1 * F1 + w2 * F2 + w3 * F3, den);
}

// ---------------------------------------------------------------- pairs (f', f'') of one velocity
// Device rows interleave the two reduced distributions of Sec. II: element
// (field d, velocity v) of a cell row sits at 2 v + d, so one 8- or 16-byte
// access moves both fields of a velocity.  The WENO-5 reconstruction, the
// BGK relaxation and the RK3 combine treat f' and f'' alike, and run on the
// pair: single precision through the packed FP32x2 add / multiply / fma of
// sm_100 and later (each lane rounds as the scalar instruction does), double
// precision as two scalar operations.  p_add and p_mul are never contracted
// into an fma (the packed intrinsics round per lane like __fadd_rn and
// __fmul_rn), so an expression of them rounds the same wherever it is inlined.

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_set(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 p_make(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 p_add(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) {
  return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 p_set(double s) { return make_double2(s, s); }
__device__ __forceinline__ double2 p_make(double x, double y) { return make_double2(x, y); }

// a - b on the pair (packed FP32x2 subtract; rounded, never contracted)
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ double2 p_sub(double2 a, double2 b) {
  return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}

template <typename real>
__device__ __forceinline__ pair_t<real> p_load(const real* p) {
  return *reinterpret_cast<const pair_t<real>*>(p);
}
template <typename real>
__device__ __forceinline__ void p_store(real* p, pair_t<real> v) {
  *reinterpret_cast<pair_t<real>*>(p) = v;
}
template <typename P>
__device__ __forceinline__ P p_sel(bool c, P a, P b) {
  return c ? a : b;
}

// Rounded multiply and add that the compiler may not fuse: the weights below are
// inlined at every cell position of an unrolled loop, and a cell must get the
// same bits whichever position (tile shape) it falls at.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// weno5 on a pair of fields: the candidate reconstructions, the indicators
// (times 4, which the normalisation removes) and the weights run on the pair;
// only the maxima, the reciprocals and the test for the slow path are per
// field.  The weighted sum is normalised once at the end.  The weights are
// products and sums of p_mul / p_add, so a cell gets the same bits at every
// position of an unrolled walk and the result does not depend on the tile shape.
// The reconstruction of both fields from their indicators and candidates, as the
// fast path of weno5p computes it, with the Table IV weights of weno5_weights_slow
// for each field whose fast-path denominator den is out of range (fast holds the
// fast-path result, kept for the other field).
template <typename real>
__device__ __noinline__ pair_t<real> weno5p_slow(pair_t<real> s1, pair_t<real> s2, pair_t<real> s3, pair_t<real> F1,
                                                 pair_t<real> F2, pair_t<real> F3, pair_t<real> den,
                                                 pair_t<real> fast) {
  real r[2] = {fast.x, fast.y};
  const real S1[2] = {s1.x, s1.y}, S2[2] = {s2.x, s2.y}, S3[2] = {s3.x, s3.y};
  const real G1[2] = {F1.x, F1.y}, G2[2] = {F2.x, F2.y}, G3[2] = {F3.x, F3.y}, Dn[2] = {den.x, den.y};
  for (int c = 0; c < 2; ++c) {
    if (Dn[c] > real(1e-30) && Dn[c] < real(1e30)) continue;
    real w[3];
    weno5_weights_slow<real>(S1[c], S2[c], S3[c], w);
    const real iden = vdiv(real(1), radd(radd(w[0], w[1]), w[2]));
    r[c] = rmul(rfma(w[0], G1[c], rfma(w[1], G2[c], rmul(w[2], G3[c]))), iden);
  }
  return p_make(r[0], r[1]);
}

template <typename real>
__device__ __forceinline__ pair_t<real> weno5p(pair_t<real> a, pair_t<real> b, pair_t<real> c, pair_t<real> d,
                                               pair_t<real> e, real sc) {
  using P = pair_t<real>;
  const P F1 = p_fma(a, p_set(real(1) / real(3)), p_fma(b, p_set(real(-7) / real(6)), p_mul(c, p_set(real(11) / real(6)))));
  const P F2 = p_fma(b, p_set(real(-1) / real(6)), p_fma(c, p_set(real(5) / real(6)), p_mul(d, p_set(real(1) / real(3)))));
  const P F3 = p_fma(c, p_set(real(1) / real(3)), p_fma(d, p_set(real(5) / real(6)), p_mul(e, p_set(real(-1) / real(6)))));
  const P S = p_set(sc);
  const P A = p_mul(a, S), B = p_mul(b, S), C = p_mul(c, S), D = p_mul(d, S), E = p_mul(e, S);
  const P k = p_set(real(13) / real(3));  // 4 * 13/12: sigma_q times 4
  const P t1 = p_fma(B, p_set(real(-2)), p_add(A, C));
  const P u1 = p_fma(B, p_set(real(-4)), p_fma(C, p_set(real(3)), A));
  const P t2 = p_fma(C, p_set(real(-2)), p_add(B, D));
  const P u2 = p_fma(D, p_set(real(-1)), B);
  const P t3 = p_fma(D, p_set(real(-2)), p_add(C, E));
  const P u3 = p_fma(D, p_set(real(-4)), p_fma(C, p_set(real(3)), E));
  const P s1 = p_fma(p_mul(t1, k), t1, p_mul(u1, u1));
  const P s2 = p_fma(p_mul(t2, k), t2, p_mul(u2, u2));
  const P s3 = p_fma(p_mul(t3, k), t3, p_mul(u3, u3));
  // delta_q prod_{r != q} x_r^2 with x = sigma / max sigma (exact for one vanishing indicator)
  const P r = p_make(vdiv(real(1), vmax(s1.x, vmax(s2.x, s3.x))), vdiv(real(1), vmax(s1.y, vmax(s2.y, s3.y))));
  const P x1 = p_mul(s1, r), x2 = p_mul(s2, r), x3 = p_mul(s3, r);
  const P q1 = p_mul(x1, x1), q2 = p_mul(x2, x2), q3 = p_mul(x3, x3);
  P w1 = p_mul(p_set(real(0.1)), p_mul(q2, q3));
  P w2 = p_mul(p_set(real(0.6)), p_mul(q1, q3));
  P w3 = p_mul(p_set(real(0.3)), p_mul(q1, q2));
  const P den = p_add(p_add(w1, w2), w3);
  const P iden = p_make(vdiv(real(1), den.x), vdiv(real(1), den.y));
  const P res = p_mul(p_fma(w1, F1, p_fma(w2, F2, p_mul(w3, F3))), iden);
  // the fast path needs a normal-range denominator (the reciprocals are
  // single-precision fast divides); anything else -- vanishing or non-finite
  // products, indicators out of range -- takes the slow path of Table IV for
  // that field: one test for both fields and one rarely taken branch
  const bool ok = (den.x > real(1e-30)) & (den.x < real(1e30)) & (den.y > real(1e-30)) & (den.y < real(1e30));
  if (__builtin_expect(!ok, 0)) return weno5p_slow<real>(s1, s2, s3, F1, F2, F3, den, res);
  return res;
}

// ---------------------------------------------------------------- equilibrium
// Moment vector m_s of the truncated equilibrium factor g_{a,k} = sum_s tab[k][s] m_s
// (Sec. IV.D).  Full range (Eq. eq_gak_H): m_l = E[He_l(X)] / l!, X ~ N(u, T),
// from l m_l = u m_{l-1} + (T - 1) m_{l-2} (generating function
// exp(t u + t^2 (T - 1) / 2)).  Half range (Eq. eq_gak_hh): m_s are the
// half-line moments int_0^inf x^s N(x; u, T) dx, from
// M_0 = (1 + erf(u / sqrt(2T))) / 2, M_1 = u M_0 + T N(0; u, T),
// M_s = u M_{s-1} + (s - 1) T M_{s-2} (integration by parts); the negative
// semi-axis uses u -> -u.
template <typename T_>
__device__ __forceinline__ T_ erf_t(T_ x);
template <>
__device__ __forceinline__ float erf_t<float>(float x) { return erff(x); }
template <>
__device__ __forceinline__ double erf_t<double>(double x) { return erf(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ void eq_moment_vector(int kind, int N, R u, R T, R* m) {
  if (kind == 0) {
    m[0] = R(1);
    if (N >= 1) m[1] = u;
    for (int l = 2; l <= N; ++l) m[l] = (u * m[l - 1] + (T - R(1)) * m[l - 2]) * (R(1) / R(l));
  } else {
    const R g0 = exp_t(-u * u / (R(2) * T)) * rsqrt_t(R(2) * R(3.14159265358979323846) * T);
    m[0] = R(0.5) * (R(1) + erf_t<R>(u * rsqrt_t(R(2) * T)));
    if (N >= 1) m[1] = u * m[0] + T * g0;
    for (int s = 2; s <= N; ++s) m[s] = u * m[s - 1] + R(s - 1) * T * m[s - 2];
  }
}

// Rescale the axis-0 equilibrium factor (which carries n) so that the stored
// factors reproduce the cell density exactly: sum_i gn_i sum_j g1_j = n.  In
// exact arithmetic the truncated equilibrium already has this sum (Sec. IV.D);
// in single precision the table contraction misses it by some 1e-7, and the
// BGK term would turn that into a mass source of (dt / tau) 1e-7 n every step.
// The sums are taken in double.
template <typename R>
__device__ __forceinline__ void normalise_equilibrium(R* gn, const R* g1, int nq0, int nq1, double n) {
  double s0 = 0.0, s1 = 0.0;
  for (int k = 0; k < nq0; ++k) s0 += double(gn[k]);
  for (int k = 0; k < nq1; ++k) s1 += double(g1[k]);
  const R sc = R(n / (s0 * s1));
  for (int k = 0; k < nq0; ++k) gn[k] *= sc;
}

template <typename R>
__device__ __forceinline__ R relaxation_time(int mode, R kn, R n, R T) {
  if (mode == 0) return kn / (n * T);
  if (mode == 1) return R(0.62665706865775012560) * kn / n;  // sqrt(pi / 8)
  return kn / n;
}

// ---------------------------------------------------------------- bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (one of the counted arrivals of the current phase).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named CTA barrier `id` over `count` threads (a multiple of 32), and its AND reduction.
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool named_bar_and(int id, int count, bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(unsigned(v)), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// One-dimensional bulk copy global -> shared completing on the mbarrier (16-byte
// aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One-dimensional bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}

// Commit the issued bulk stores and wait until their shared-memory sources have been read.
__device__ __forceinline__ void bulk_commit_and_wait_read() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// The same in parts: commit the issued bulk stores as a group; wait until every
// committed group of this thread has read its shared-memory source; wait until
// every committed group has completed.
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long max_polls) {
  uint32_t done = 0;
  for (unsigned long long it = 0; it < max_polls; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Knuth's TwoSum: s = fl(a + b) and the exact rounding error err = a + b - s.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Compensated butterfly sum over each half-warp (lanes 0-15 and 16-31
// separately) in single precision.  Each step adds the partner's value with
// TwoSum, and the errors accumulate in e.  On return every lane of a half holds
// the same (s, e), whose sum s + e carries about twice the float precision, so a
// reduction that would otherwise need the 1/64-rate FP64 pipe stays on FP32.
__device__ __forceinline__ void half_sum_comp(float& s, float& e) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), e2 = __shfl_xor_sync(0xffffffffu, e, o);
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    s = t;
    e = __fadd_rn(__fadd_rn(e, e2), err);
  }
}

// Plain double sum over each half-warp.
__device__ __forceinline__ double half_sum(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename real>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace vlb
