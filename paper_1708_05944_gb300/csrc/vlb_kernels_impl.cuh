// Kernels and launchers instantiated once per precision by vlb_f32.cu / vlb_f64.cu.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include "vlb_launch.h"
#include "vlb_stage.cuh"
#include "vlb_channel.cuh"

namespace vlb {

// ---------------------------------------------------------------- stage dispatch
// Launch shapes ("variants") of the stage kernel: cells per tile TC and threads
// per CTA NT.  Exact instantiations exist for the node counts of the
// configured models; anything else takes the generic kernel.  The autotuner
// (vlb_autotune) times the variants of a context's shape and keeps the best.
// Tile buffers and resident CTAs per SM of a launch shape: one buffer for a launch
// with one CTA per tile; a persistent launch takes two (staging its next tile while
// it computes one) when that leaves as many CTAs resident as one buffer does.
template <typename real, int TC, int NT, int Q0, int Q1, bool EXACT, bool FT = false>
static cudaError_t stage_buffers(int Vp, int persist, int* nbuf, int* per_sm) {
  using L = StageSmem<real, TC, NT>;
  auto kern = couette_stage_kernel<real, TC, Q0, Q1, NT, EXACT, FT>;
  const size_t limit = 227 * 1024;
  const int top = persist && L::bytes(Vp, 2) <= limit ? 2 : 1;
  // the kernel's shared-memory limit is process-wide and shared by contexts of other row
  // lengths (the generic kernels), so it is only ever raised
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (size_t(fa.maxDynamicSharedSizeBytes) < L::bytes(Vp, top)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L::bytes(Vp, top)));
    if (e != cudaSuccess) return e;
  }
  *nbuf = 1, *per_sm = 0;
  for (int nb = 1; nb <= top; ++nb) {
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, L::bytes(Vp, nb))) != cudaSuccess) return e;
    if (nb == 1 || (occ > 0 && occ >= *per_sm)) *nbuf = nb, *per_sm = occ;
  }
  return cudaSuccess;
}

template <typename real, int TC, int NT, int Q0, int Q1, bool EXACT, bool FT = false>
static cudaError_t go_stage(const StageArgs<real>& a, const ModelArgs& m, const KArgs<real>& k, int grid,
                            cudaStream_t s) {
  couette_stage_kernel<real, TC, Q0, Q1, NT, EXACT, FT>
      <<<grid, NT, StageSmem<real, TC, NT>::bytes(a.Vp, a.nbuf), s>>>(a, m, k);
  return cudaGetLastError();
}

enum Shape { SH_16x20 = 0, SH_16x12 = 1, SH_8x4 = 2, SH_SMALL = 3, SH_GENERIC = 4 };

static int shape_of(int nq0, int nq1) {
  if (nq0 == 16 && nq1 == 20) return SH_16x20;
  if (nq0 == 16 && nq1 == 12) return SH_16x12;
  if (nq0 == 8 && nq1 == 4) return SH_8x4;
  if (nq0 * nq1 <= 64) return SH_SMALL;
  return SH_GENERIC;
}

// variant tables per precision and shape: {TC, NT}
template <typename real>
struct VariantTable;
template <>
struct VariantTable<float> {
  static constexpr StageVariant v16x20[] = {{4, 256, 0},  {8, 256, 0},  {4, 320, 0}, {8, 320, 0},
                                            {16, 320, 0}, {10, 320, 0}, {9, 320, 0}};
  static constexpr StageVariant v16x12[] = {{16, 256, 0}, {8, 256, 0}, {16, 384, 0}};
  static constexpr StageVariant v8x4[] = {{16, 64, 0}, {8, 64, 0}};
  static constexpr StageVariant vsmall[] = {{16, 64, 0}};
  static constexpr StageVariant vgen[] = {{16, 256, 0}};
};
template <>
struct VariantTable<double> {
  static constexpr StageVariant v16x20[] = {{4, 256, 0}, {8, 256, 0}, {4, 128, 0}, {8, 128, 0}};
  static constexpr StageVariant v16x12[] = {{8, 256, 0}, {4, 256, 0}, {8, 384, 0}};
  static constexpr StageVariant v8x4[] = {{8, 64, 0}, {16, 64, 0}};
  static constexpr StageVariant vsmall[] = {{8, 64, 0}};
  static constexpr StageVariant vgen[] = {{8, 256, 0}};
};

template <typename real>
int stage_variants(int nq0, int nq1, StageVariant* out) {
  using T = VariantTable<real>;
  const StageVariant* v;
  int n;
  switch (shape_of(nq0, nq1)) {
    case SH_16x20: v = T::v16x20, n = int(sizeof(T::v16x20) / sizeof(StageVariant)); break;
    case SH_16x12: v = T::v16x12, n = int(sizeof(T::v16x12) / sizeof(StageVariant)); break;
    case SH_8x4: v = T::v8x4, n = int(sizeof(T::v8x4) / sizeof(StageVariant)); break;
    case SH_SMALL: v = T::vsmall, n = 1; break;
    default: v = T::vgen, n = 1; break;
  }
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

template <typename real>
bool stage_split_tables(int nq0, int nq1) {
  const int sh = shape_of(nq0, nq1);
  return sh == SH_16x20 || sh == SH_16x12 || sh == SH_8x4;
}

template <typename real>
size_t stage_smem_bytes(StageVariant v, int Vp) {
#define VLB_SMEM_CASE(TC_, NT_) \
  if (v.tc == TC_ && v.nt == NT_) return StageSmem<real, TC_, NT_>::bytes(Vp, 1);
  VLB_SMEM_CASE(16, 256) VLB_SMEM_CASE(8, 256) VLB_SMEM_CASE(16, 512) VLB_SMEM_CASE(8, 128)
  VLB_SMEM_CASE(16, 384) VLB_SMEM_CASE(16, 64) VLB_SMEM_CASE(8, 64) VLB_SMEM_CASE(4, 256)
  VLB_SMEM_CASE(4, 128) VLB_SMEM_CASE(8, 384) VLB_SMEM_CASE(4, 320) VLB_SMEM_CASE(8, 320)
  VLB_SMEM_CASE(16, 320) VLB_SMEM_CASE(10, 320) VLB_SMEM_CASE(9, 320)
#undef VLB_SMEM_CASE
  return 0;
}

template <typename real>
cudaError_t launch_stage(StageVariant v, const StageArgs<real>& a, const ModelArgs& m, const KArgs<real>& k, int grid,
                         cudaStream_t s, bool ft) {
  const int sh = shape_of(m.nq0, m.nq1);
  if (ft) {  // the f~ kernels: the first launch shape of each shape's table
#define VLB_FT(SH, TC_, NT_, q0, q1, ex) \
  if (sh == SH && v.tc == TC_ && v.nt == NT_) return go_stage<real, TC_, NT_, q0, q1, ex, true>(a, m, k, grid, s);
    if constexpr (sizeof(real) == 4) {
      VLB_FT(SH_16x20, 4, 256, 16, 20, true) VLB_FT(SH_16x12, 16, 256, 16, 12, true)
      VLB_FT(SH_8x4, 16, 64, 8, 4, true) VLB_FT(SH_SMALL, 16, 64, MAXQ, MAXQ, false)
      VLB_FT(SH_GENERIC, 16, 256, MAXQ, MAXQ, false)
    } else {
      VLB_FT(SH_16x20, 4, 256, 16, 20, true) VLB_FT(SH_16x12, 8, 256, 16, 12, true)
      VLB_FT(SH_8x4, 8, 64, 8, 4, true) VLB_FT(SH_SMALL, 8, 64, MAXQ, MAXQ, false)
      VLB_FT(SH_GENERIC, 8, 256, MAXQ, MAXQ, false)
    }
#undef VLB_FT
    return cudaErrorInvalidValue;
  }
#define VLB_CASE(SH, TC_, NT_, q0, q1, ex) \
  if (sh == SH && v.tc == TC_ && v.nt == NT_) return go_stage<real, TC_, NT_, q0, q1, ex>(a, m, k, grid, s);
  if constexpr (sizeof(real) == 4) {
    VLB_CASE(SH_16x20, 4, 256, 16, 20, true) VLB_CASE(SH_16x20, 8, 256, 16, 20, true)
    VLB_CASE(SH_16x20, 4, 320, 16, 20, true) VLB_CASE(SH_16x20, 8, 320, 16, 20, true)
    VLB_CASE(SH_16x20, 16, 320, 16, 20, true) VLB_CASE(SH_16x20, 10, 320, 16, 20, true)
    VLB_CASE(SH_16x20, 9, 320, 16, 20, true)
    VLB_CASE(SH_16x12, 16, 256, 16, 12, true) VLB_CASE(SH_16x12, 8, 256, 16, 12, true)
    VLB_CASE(SH_16x12, 16, 384, 16, 12, true)
    VLB_CASE(SH_8x4, 16, 64, 8, 4, true) VLB_CASE(SH_8x4, 8, 64, 8, 4, true)
    VLB_CASE(SH_SMALL, 16, 64, MAXQ, MAXQ, false)
    VLB_CASE(SH_GENERIC, 16, 256, MAXQ, MAXQ, false)
  } else {
    VLB_CASE(SH_16x20, 4, 256, 16, 20, true) VLB_CASE(SH_16x20, 8, 256, 16, 20, true)
    VLB_CASE(SH_16x20, 4, 128, 16, 20, true) VLB_CASE(SH_16x20, 8, 128, 16, 20, true)
    VLB_CASE(SH_16x12, 8, 256, 16, 12, true) VLB_CASE(SH_16x12, 4, 256, 16, 12, true)
    VLB_CASE(SH_16x12, 8, 384, 16, 12, true)
    VLB_CASE(SH_8x4, 8, 64, 8, 4, true) VLB_CASE(SH_8x4, 16, 64, 8, 4, true)
    VLB_CASE(SH_SMALL, 8, 64, MAXQ, MAXQ, false)
    VLB_CASE(SH_GENERIC, 8, 256, MAXQ, MAXQ, false)
  }
#undef VLB_CASE
  return cudaErrorInvalidValue;
}

template <typename real>
cudaError_t stage_config(StageVariant v, const ModelArgs& m, int Vp, int* nbuf, int* per_sm, bool ft) {
  const int sh = shape_of(m.nq0, m.nq1);
  if (ft) {
#define VLB_FT(SH, TC_, NT_, q0, q1, ex) \
  if (sh == SH && v.tc == TC_ && v.nt == NT_) return stage_buffers<real, TC_, NT_, q0, q1, ex, true>(Vp, v.persist, nbuf, per_sm);
    if constexpr (sizeof(real) == 4) {
      VLB_FT(SH_16x20, 4, 256, 16, 20, true) VLB_FT(SH_16x12, 16, 256, 16, 12, true)
      VLB_FT(SH_8x4, 16, 64, 8, 4, true) VLB_FT(SH_SMALL, 16, 64, MAXQ, MAXQ, false)
      VLB_FT(SH_GENERIC, 16, 256, MAXQ, MAXQ, false)
    } else {
      VLB_FT(SH_16x20, 4, 256, 16, 20, true) VLB_FT(SH_16x12, 8, 256, 16, 12, true)
      VLB_FT(SH_8x4, 8, 64, 8, 4, true) VLB_FT(SH_SMALL, 8, 64, MAXQ, MAXQ, false)
      VLB_FT(SH_GENERIC, 8, 256, MAXQ, MAXQ, false)
    }
#undef VLB_FT
    return cudaErrorInvalidValue;
  }
#define VLB_CASE(SH, TC_, NT_, q0, q1, ex) \
  if (sh == SH && v.tc == TC_ && v.nt == NT_)      \
    return stage_buffers<real, TC_, NT_, q0, q1, ex>(Vp, v.persist, nbuf, per_sm);
  if constexpr (sizeof(real) == 4) {
    VLB_CASE(SH_16x20, 4, 256, 16, 20, true) VLB_CASE(SH_16x20, 8, 256, 16, 20, true)
    VLB_CASE(SH_16x20, 4, 320, 16, 20, true) VLB_CASE(SH_16x20, 8, 320, 16, 20, true)
    VLB_CASE(SH_16x20, 16, 320, 16, 20, true) VLB_CASE(SH_16x20, 10, 320, 16, 20, true)
    VLB_CASE(SH_16x20, 9, 320, 16, 20, true)
    VLB_CASE(SH_16x12, 16, 256, 16, 12, true) VLB_CASE(SH_16x12, 8, 256, 16, 12, true)
    VLB_CASE(SH_16x12, 16, 384, 16, 12, true)
    VLB_CASE(SH_8x4, 16, 64, 8, 4, true) VLB_CASE(SH_8x4, 8, 64, 8, 4, true)
    VLB_CASE(SH_SMALL, 16, 64, MAXQ, MAXQ, false)
    VLB_CASE(SH_GENERIC, 16, 256, MAXQ, MAXQ, false)
  } else {
    VLB_CASE(SH_16x20, 4, 256, 16, 20, true) VLB_CASE(SH_16x20, 8, 256, 16, 20, true)
    VLB_CASE(SH_16x20, 4, 128, 16, 20, true) VLB_CASE(SH_16x20, 8, 128, 16, 20, true)
    VLB_CASE(SH_16x12, 8, 256, 16, 12, true) VLB_CASE(SH_16x12, 4, 256, 16, 12, true)
    VLB_CASE(SH_16x12, 8, 384, 16, 12, true)
    VLB_CASE(SH_8x4, 8, 64, 8, 4, true) VLB_CASE(SH_8x4, 16, 64, 8, 4, true)
    VLB_CASE(SH_SMALL, 8, 64, MAXQ, MAXQ, false)
    VLB_CASE(SH_GENERIC, 8, 256, MAXQ, MAXQ, false)
  }
#undef VLB_CASE
  *nbuf = 1, *per_sm = 0;
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- channel dispatch
template <typename real, int Q0, int Q1, int TP, bool TC, bool CLB = false>
static cudaError_t go_channel(const ChanArgs<real>& a, const void* kpb, int grid, cudaStream_t s) {
  using L = ChanSmem<real, Q0, Q1, TP>;
  auto kern = channel_stage_kernel<real, Q0, Q1, TP, TC, CLB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L::bytes));
  if (e != cudaSuccess) return e;
  ChanKP<Q0, Q1> kp;
  memcpy(&kp, kpb, sizeof(kp));
  kern<<<grid, L::NT, L::bytes, s>>>(a, kp);
  return cudaGetLastError();
}

#ifdef VLB_DEFINE_SHARED
// {rows per segment (0: host's choice, 1 << 20: one segment), columns per strip, threads, tensor-core force}
static const ChanVariant kChan16x12[] = {{0, 4, 1024, 0}, {0, 4, 1024, 1}, {1 << 20, 4, 1024, 0}, {64, 4, 1024, 0}};
static const ChanVariant kChan8x4[] = {{0, 4, 224, 0}, {0, 8, 352, 0}, {0, 4, 224, 1}, {1 << 20, 4, 224, 0}};

int channel_variants(int nq0, int nq1, ChanVariant* out) {
  const ChanVariant* v = nullptr;
  int n = 0;
  if (nq0 == 16 && nq1 == 12) v = kChan16x12, n = int(sizeof(kChan16x12) / sizeof(ChanVariant));
  if (nq0 == 8 && nq1 == 4) v = kChan8x4, n = int(sizeof(kChan8x4) / sizeof(ChanVariant));
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

template <int Q0, int Q1>
static bool fill_force_pairs(const AxisTables* ax, std::vector<unsigned char>* out) {
  using KP = ChanKP<Q0, Q1>;
  out->assign(sizeof(KP), 0);
  KP& kp = *reinterpret_cast<KP*>(out->data());
  // each axis: nodes mirror each other under J, K J = -J K and Kt J = J Kt, to rounding
  for (int a = 0; a < 2; ++a) {
    const AxisTables& t = ax[a];
    const int nq = t.nq;
    double kmax = 0.0, tmax = 0.0, pmax = 0.0;
    for (int k = 0; k < nq * nq; ++k) kmax = std::max(kmax, std::fabs(t.K[k])), tmax = std::max(tmax, std::fabs(t.Kt[k]));
    for (int k = 0; k < nq; ++k) pmax = std::max(pmax, std::fabs(t.p[k]));
    for (int r = 0; r < nq; ++r) {
      if (std::fabs(t.p[refl(t.kind, nq, r)] + t.p[r]) > 1e-13 * pmax) return false;
      for (int q = 0; q < nq; ++q) {
        const int rr = refl(t.kind, nq, r), qq = refl(t.kind, nq, q);
        if (std::fabs(t.K[rr * nq + qq] + t.K[r * nq + q]) > 1e-12 * kmax) return false;
        if (std::fabs(t.Kt[rr * nq + qq] - t.Kt[r * nq + q]) > 1e-12 * tmax) return false;
      }
    }
  }
  // the kernels take the mirror of k as k + H on the half-range lambda axis and Q1 - 1 - k
  // on the full-range xi axis
  if (ax[0].kind != 1 || ax[1].kind != 0) return false;
  auto put = [](float2* P, float2* M, const std::vector<double>& K, int nq, int kind) {
    const int H = nq / 2;
    for (int r = 0; r < H; ++r)
      for (int q = 0; q < H; ++q) {
        const double x = K[r * nq + q], y = K[r * nq + refl(kind, nq, q)];
        const float pv = float(0.5 * (x + y)), mv = float(0.5 * (x - y));
        P[r * H + q] = make_float2(pv, pv);
        M[r * H + q] = make_float2(mv, mv);
      }
  };
  put(kp.P0, kp.M0, ax[0].K, Q0, 1);
  put(kp.Pt0, kp.Mt0, ax[0].Kt, Q0, 1);
  put(kp.P1, kp.M1, ax[1].K, Q1, 0);
  put(kp.Pt1, kp.Mt1, ax[1].Kt, Q1, 0);
  return true;
}

bool channel_force_pairs(int nq0, int nq1, const AxisTables* ax, std::vector<unsigned char>* out) {
  if (nq0 == 16 && nq1 == 12) return fill_force_pairs<16, 12>(ax, out);
  if (nq0 == 8 && nq1 == 4) return fill_force_pairs<8, 4>(ax, out);
  return false;
}
#endif

template <typename real>
size_t channel_smem_bytes(ChanVariant v, int nq0, int nq1) {
  if (nq0 == 16 && nq1 == 12 && v.tp == 4) return ChanSmem<real, 16, 12, 4>::bytes;
  if (nq0 == 8 && nq1 == 4 && v.tp == 4) return ChanSmem<real, 8, 4, 4>::bytes;
  if (nq0 == 8 && nq1 == 4 && v.tp == 8) return ChanSmem<real, 8, 4, 8>::bytes;
  return 0;
}

// TF32 part of x rounded to nearest, ties away from zero (the rounding of
// cvt.rna.tf32.f32): the low 13 significand bits cleared.
static inline uint32_t host_tf32(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return u;
  return (u + 0x1000u) & 0xffffe000u;
}
static inline void host_tf32_split(double x, uint32_t* hi, uint32_t* lo) {
  const float f = float(x);
  *hi = host_tf32(f);
  float h;
  memcpy(&h, hi, 4);
  *lo = host_tf32(f - h);
}

// Axis moment vector of the truncated equilibrium at rest (u = 0), in double.
static void rest_moment_vector(int kind, int N, double T, double* m) {
  if (kind == 0) {
    m[0] = 1.0;
    if (N >= 1) m[1] = 0.0;
    for (int l = 2; l <= N; ++l) m[l] = (T - 1.0) * m[l - 2] / double(l);
    return;
  }
  m[0] = 0.5;
  if (N >= 1) m[1] = T / std::sqrt(2.0 * 3.14159265358979323846 * T);
  for (int s = 2; s <= N; ++s) m[s] = double(s - 1) * T * m[s - 2];
}

template <typename real, int Q0, int Q1>
static void fill_chan_tables(const AxisTables* ax, const ModelArgs& m, double T0, std::vector<unsigned char>* out) {
  using Tab = ChanTables<real, Q0, Q1>;
  using S = ChanShape<Q0, Q1>;
  out->assign(sizeof(Tab), 0);
  Tab& t = *reinterpret_cast<Tab*>(out->data());
  const std::vector<double>&K0 = ax[0].K, &Kt0 = ax[0].Kt, &K1 = ax[1].K, &Kt1 = ax[1].Kt;
  for (int k = 0; k < Q0 * Q0; ++k) t.K0[k] = real(K0[k]), t.Kt0[k] = real(Kt0[k]);
  for (int k = 0; k < Q1 * Q1; ++k) t.K1[k] = real(K1[k]), t.Kt1[k] = real(Kt1[k]);
  // lambda A fragments: a0 = K0[8t+g][8kk+tq], a1 = Kt0[..][8kk+tq], a2 = K0[..][8kk+tq+4], a3 = Kt0[..][8kk+tq+4]
  for (int mt = 0; mt < S::MT; ++mt)
    for (int kk = 0; kk < S::KKL; ++kk)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, tq = lane & 3, r = 8 * mt + g;
        const double v4[4] = {K0[r * Q0 + 8 * kk + tq], Kt0[r * Q0 + 8 * kk + tq], K0[r * Q0 + 8 * kk + tq + 4],
                              Kt0[r * Q0 + 8 * kk + tq + 4]};
        for (int q = 0; q < 4; ++q) host_tf32_split(v4[q], &t.fl[mt][kk][0][lane][q], &t.fl[mt][kk][1][lane][q]);
      }
  // xi B fragments: b0 = B[8kk+tq][8nn+g], b1 = B[8kk+tq+4][8nn+g], B[j'][2j+e] = (e ? Kt1 : K1)[j][j']
  for (int kk = 0; kk < S::KKX; ++kk)
    for (int nn = 0; nn < S::NN; ++nn)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, tq = lane & 3;
        const int jj = 4 * nn + (g >> 1), e = g & 1;
        const std::vector<double>& M = e ? Kt1 : K1;
        for (int q = 0; q < 2; ++q) {
          const int jp = 8 * kk + tq + 4 * q;
          const double x = jp < Q1 ? M[jj * Q1 + jp] : 0.0;
          host_tf32_split(x, &t.fx[kk][nn][0][lane][q], &t.fx[kk][nn][1][lane][q]);
        }
      }
  for (int k = 0; k < Q0; ++k) {
    t.p0[k] = real(m.p0[k]);
    t.iw0[k] = real(m.iw0[k]);
    t.w0[k] = real(m.w0[k]);
    for (int s = 0; s < MAXN; ++s) t.tab0[k * MAXN + s] = real(m.tab0[k * MAXN + s]);
  }
  for (int k = 0; k < Q1; ++k) {
    t.p1[k] = real(m.p1[k]);
    t.iw1[k] = real(m.iw1[k]);
    t.w1[k] = real(m.w1[k]);
    for (int s = 0; s < MAXN; ++s) t.tab1[k * MAXN + s] = real(m.tab1[k * MAXN + s]);
  }
  // f_eq(1, 0, T0): factors and the incoming wall flux (the denominator of Eq. nw)
  double mv0[MAXN], mv1[MAXN], g0[Q0], g1[Q1];
  rest_moment_vector(m.kind0, m.N0, T0, mv0);
  rest_moment_vector(m.kind1, m.N1, T0, mv1);
  double den0 = 0.0, den1 = 0.0;
  for (int k = 0; k < Q0; ++k) {
    g0[k] = 0.0;
    for (int s = 0; s <= m.N0; ++s) g0[k] += m.tab0[k * MAXN + s] * mv0[s];
    t.gw0[k] = real(g0[k]);
    if (m.p0[k] < 0.0) den0 += g0[k] * m.p0[k];
  }
  for (int k = 0; k < Q1; ++k) {
    g1[k] = 0.0;
    for (int s = 0; s <= m.N1; ++s) g1[k] += m.tab1[k * MAXN + s] * mv1[s];
    t.gw1[k] = real(g1[k]);
    den1 += g1[k];
  }
  t.wall_den = den0 * den1;
  t.ref_flux_pos = m.ref_flux_pos;
  const double refs[4] = {m.ref_n, m.ref_r, m.ref_p, m.ref_e};
  for (int k = 0; k < 4; ++k) {
    t.ref_hi[k] = real(refs[k]);
    t.ref_lo[k] = real(refs[k] - double(t.ref_hi[k]));
  }
  t.N0 = m.N0, t.N1 = m.N1, t.kind0 = m.kind0, t.kind1 = m.kind1;
}

template <typename real>
bool channel_tables(int nq0, int nq1, const AxisTables* ax, const ModelArgs& m, double T0,
                    std::vector<unsigned char>* out) {
  if (nq0 == 16 && nq1 == 12) return fill_chan_tables<real, 16, 12>(ax, m, T0, out), true;
  if (nq0 == 8 && nq1 == 4) return fill_chan_tables<real, 8, 4>(ax, m, T0, out), true;
  return false;
}

template <typename real>
cudaError_t launch_channel(ChanVariant v, const ChanArgs<real>& a, const void* kp, int nq0, int nq1, int grid,
                           cudaStream_t s, bool clb) {
#define VLB_CH(q0, q1, TP_)                                                                  \
  if (nq0 == q0 && nq1 == q1 && v.tp == TP_)                                                 \
    return clb ? go_channel<real, q0, q1, TP_, false, true>(a, kp, grid, s)                  \
               : (sizeof(real) == 4 && v.tc) ? go_channel<real, q0, q1, TP_, sizeof(real) == 4>(a, kp, grid, s) \
                                             : go_channel<real, q0, q1, TP_, false>(a, kp, grid, s);
  VLB_CH(16, 12, 4) VLB_CH(8, 4, 4) VLB_CH(8, 4, 8)
#undef VLB_CH
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- equilibrium fill
template <typename real>
__global__ void init_equilibrium_kernel(real* F, long long cells, int Vp, const __grid_constant__ ModelArgs m,
                                        double n0, double u0, double u1, double T0) {
  __shared__ double g0[MAXQ], g1[MAXQ];
  if (threadIdx.x < 2) {
    const int ax = threadIdx.x;
    double mp[MAXN], mm[MAXN];
    const int kind = ax ? m.kind1 : m.kind0, N = ax ? m.N1 : m.N0, nq = ax ? m.nq1 : m.nq0;
    const double u = ax ? u1 : u0;
    eq_moment_vector<double>(kind, N, u, T0, mp);
    eq_moment_vector<double>(kind, N, -u, T0, mm);
    for (int k = 0; k < nq; ++k) {
      const double pk = ax ? m.p1[k] : m.p0[k];
      const double* mv = (kind == 1 && pk < 0.0) ? mm : mp;
      double g = 0;
      for (int s = 0; s <= N; ++s) g += (ax ? m.tab1 : m.tab0)[k * MAXN + s] * mv[s];
      (ax ? g1 : g0)[k] = g;
    }
  }
  __syncthreads();
  const int V = m.nq0 * m.nq1;
  const long long total = cells * 2 * Vp;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const int e = int(x % (2 * Vp));  // (velocity, field) pairs interleaved
    const int v = e >> 1, d = e & 1;
    real val = real(0);
    if (v < V) {
      const int i = v / m.nq1, j = v - i * m.nq1;
      val = real(n0 * g0[i] * g1[j] * (d ? T0 : 1.0) - m.w0[i] * m.w1[j]);  // stored as the deviation from R
    }
    F[x] = val;
  }
}

template <typename real>
cudaError_t launch_init_equilibrium(real* F, long long cells, int Vp, const ModelArgs& m, double n0, double u0,
                                    double u1, double T0, cudaStream_t s) {
  const long long total = cells * 2 * Vp;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  init_equilibrium_kernel<real><<<int(blocks), 256, 0, s>>>(F, cells, Vp, m, n0, u0, u1, T0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- seeding from moments, one CTA per cell
// Table input vector of the one-axis function xi^k g(p) (xi = p - u, g the
// unit-mass Gaussian of mean u and variance T) for k <= 3, on the semi-axis of
// sign `side` (half range) or the whole line (full range, side ignored).
// Full range: the table takes E[He_l h] / l!, and (p - u) acts on that sequence
// as a_l -> (l + 1) a_{l+1} + a_{l-1} - u a_l (from p He_l = He_{l+1} + l He_{l-1}).
// Half range: the table takes the raw moments int_0^inf p^s h(side p) dp; with
// h(-p) = (-1)^k (p + u)^k g_{-u}(p) both sides are the binomial expansion of
// (p - v)^k, v = side u, over the raw moments of g_v on [0, inf).
__device__ inline void xi_power_vector(int kind, int N, double u, double T, int k, int side, double* out) {
  double m[MAXN + 3];
  if (kind == 0) {
    eq_moment_vector<double>(0, N + k, u, T, m);
    for (int it = 0; it < k; ++it) {
      const int top = N + k - it - 1;  // entries 0..top stay valid after this application
      double prev = 0.0;                // old m[l - 1]
      for (int l = 0; l <= top; ++l) {
        const double cur = m[l];
        m[l] = double(l + 1) * m[l + 1] + prev - u * cur;
        prev = cur;
      }
    }
    for (int l = 0; l <= N; ++l) out[l] = m[l];
    return;
  }
  const double v = side > 0 ? u : -u;
  eq_moment_vector<double>(1, N + k, v, T, m);
  // binomial coefficients C(k, i) (-v)^(k - i)
  double c[4] = {1, 0, 0, 0};
  for (int it = 0; it < k; ++it)
    for (int i = it + 1; i >= 0; --i) c[i] = (i ? c[i - 1] : 0.0) - v * c[i];
  const double sgn = (side < 0 && (k & 1)) ? -1.0 : 1.0;
  for (int s = 0; s <= N; ++s) {
    double acc = 0;
    for (int i = 0; i <= k; ++i) acc += c[i] * m[s + i];
    out[s] = sgn * acc;
  }
}

// Populations of xi^k g on one axis: pop[j] = sum_s tab[j][s] vec_side(j)[s].
__device__ inline void xi_power_populations(int kind, int N, int nq, const double* p, const double* tab, double u, double T,
                                     int k, double* pop) {
  double vp[MAXN], vm[MAXN];
  xi_power_vector(kind, N, u, T, k, 1, vp);
  if (kind == 1) xi_power_vector(kind, N, u, T, k, -1, vm);
  for (int j = 0; j < nq; ++j) {
    const double* v = (kind == 1 && p[j] < 0.0) ? vm : vp;
    double g = 0;
    for (int s = 0; s <= N; ++s) g += tab[j * MAXN + s] * v[s];
    pop[j] = g;
  }
}

// f' = n g0 g1 + q0/T^2 g0 g1 xi0 [(xi0^2 + xi1^2)/(5T) - 4/5],
// f'' = T n g0 g1 + q0/T^2 g0 g1 xi0 [(xi0^2 + xi1^2)/5 - 2T/5]:
// Grad's distribution with the heat-flux part only (along axis 0), p^z
// integrated out, projected on the model basis axis by axis.
template <typename real>
__global__ void seed_kernel(real* F, long long cells, int Vp, const __grid_constant__ ModelArgs m, const double* n,
                            const double* u0, const double* u1, const double* T, const double* q0, CellMap map) {
  __shared__ double A[3][MAXQ], B[2][MAXQ];  // axis 0: xi^0, xi^1, xi^3; axis 1: xi^0, xi^2
  for (long long c = blockIdx.x; c < cells; c += gridDim.x) {
    const long long cc = caller_cell(map, c);  // the fields are in the caller's cell order
    const double Tc = T[cc], qc = q0 ? q0[cc] : 0.0;
    if (threadIdx.x < 5) {
      const int t = threadIdx.x;
      if (t < 3) {
        const int k = t == 2 ? 3 : t;
        xi_power_populations(m.kind0, m.N0, m.nq0, m.p0, m.tab0, u0[cc], Tc, k, A[t]);
      } else {
        xi_power_populations(m.kind1, m.N1, m.nq1, m.p1, m.tab1, u1[cc], Tc, 2 * (t - 3), B[t - 3]);
      }
    }
    __syncthreads();
    const int V = m.nq0 * m.nq1;
    const double cq = qc / (Tc * Tc);
    for (int x = threadIdx.x; x < 2 * Vp; x += blockDim.x) {
      const int v = x >> 1, d = x & 1;  // (velocity, field) pairs interleaved
      real val = real(0);
      if (v < V) {
        const int i = v / m.nq1, j = v - i * m.nq1;
        const double base = n[cc] * A[0][i] * B[0][j];
        const double t3 = A[2][i] * B[0][j] + A[1][i] * B[1][j];
        const double t1 = A[1][i] * B[0][j];
        const double full = d ? Tc * base + cq * (0.2 * t3 - 0.4 * Tc * t1) : base + cq * (t3 / (5.0 * Tc) - 0.8 * t1);
        val = real(full - m.w0[i] * m.w1[j]);  // stored as the deviation from R
      }
      F[c * 2 * Vp + x] = val;
    }
    __syncthreads();
  }
}

template <typename real>
cudaError_t launch_seed(real* F, long long cells, int Vp, const ModelArgs& m, const double* n, const double* u0,
                        const double* u1, const double* T, const double* q0, cudaStream_t s, CellMap map) {
  const long long blocks = cells < 152 * 16 ? cells : 152 * 16;
  seed_kernel<real><<<int(blocks > 0 ? blocks : 1), 128, 0, s>>>(F, cells, Vp, m, n, u0, u1, T, q0, map);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Shakhov collision
// The Shakhov collision relaxes towards f_eq + (1 - Pr) G, G the heat-flux part of Grad's
// form for the cell's own q (the seed kernel's term, with both axes):
//   G'  = [q0 (t3_0 / (5T) - 4/5 t1_0) + q1 (t3_1 / (5T) - 4/5 t1_1)] / T^2,
//   G'' = [q0 (t3_0 / 5 - 2T/5 t1_0) + q1 (t3_1 / 5 - 2T/5 t1_1)] / T^2,
//   t3_0 = A3 B0 + A1 B2, t1_0 = A1 B0, t3_1 = A2 B1 + A0 B3, t1_1 = A0 B1,
// A_k, B_k the projections of xi^k g on axes 0 and 1.  Against the BGK stage that the stage
// kernel has written, a stage of weight cc adds cc dt (1 - Pr) G[F_prev] / tau to F_out.
// One warp per cell: the cell's n, u, T and q from F_prev (sums and per-cell scalars in the
// bulk type: they enter a correction term), the projections A_k, B_k by the warp, then G for
// every (velocity, field).
// The model arrays a CTA indexes per thread, staged in shared memory: read from the kernel
// parameters with a different index in every lane they would be serialised.
template <typename real>
struct ModelSmem {
  real p[2][MAXQ], w[2][MAXQ], tab[2][MAXQ * MAXN];
};
template <typename real>
__device__ inline void stage_model(const ModelArgs& m, ModelSmem<real>& ms) {
  for (int k = threadIdx.x; k < MAXQ; k += blockDim.x) {
    if constexpr (sizeof(real) == 4) {
      ms.p[0][k] = m.p0f[k], ms.p[1][k] = m.p1f[k], ms.w[0][k] = m.w0f[k], ms.w[1][k] = m.w1f[k];
    } else {
      ms.p[0][k] = m.p0[k], ms.p[1][k] = m.p1[k], ms.w[0][k] = m.w0[k], ms.w[1][k] = m.w1[k];
    }
  }
  for (int k = threadIdx.x; k < MAXQ * MAXN; k += blockDim.x) {
    if constexpr (sizeof(real) == 4) ms.tab[0][k] = m.tab0f[k], ms.tab[1][k] = m.tab1f[k];
    else ms.tab[0][k] = m.tab0[k], ms.tab[1][k] = m.tab1[k];
  }
  __syncthreads();
}
// The tables A_k = [xi^k g] on axis 0 and B_k on axis 1 (k <= 3, xi_power_populations) for
// the cell's u and T, by one warp: the moment vector of each (axis, semi-axis) once, the
// input vector of each (axis, k, semi-axis), then the rows of the node tables in parallel; in
// the bulk type (the term they build is a correction of the collision).
template <typename R>
__device__ inline void power_tables(const ModelArgs& m, const ModelSmem<R>& ms, R u0, R u1, R T, R (*M)[MAXN + 3],
                                    R (*OV)[MAXN], R (*A)[MAXQ], R (*B)[MAXQ]) {
  const int tid = threadIdx.x & 31;
  if (tid < 4) {  // (axis, side): side 0 the positive semi-axis (or the whole line), side 1 the negative
    const int ax = tid >> 1, side = tid & 1;
    const int kind = ax ? m.kind1 : m.kind0, N = ax ? m.N1 : m.N0;
    const R u = ax ? u1 : u0;
    if (kind == 1 || side == 0) eq_moment_vector<R>(kind, N + 3, (kind == 1 && side) ? -u : u, T, M[tid]);
  }
  __syncwarp();
  if (tid < 16) {  // (axis, k, side), as xi_power_vector
    const int ax = tid >> 3, k = (tid >> 1) & 3, side = tid & 1;
    const int kind = ax ? m.kind1 : m.kind0, N = ax ? m.N1 : m.N0;
    const R u = ax ? u1 : u0;
    R* out = OV[tid];
    if (kind == 0) {
      if (side == 0) {
        R mm[MAXN + 3];
        for (int l = 0; l <= N + 3; ++l) mm[l] = M[2 * ax][l];
        for (int it = 0; it < k; ++it) {
          const int top = N + k - it - 1;
          R prev = R(0);
          for (int l = 0; l <= top; ++l) {
            const R cur = mm[l];
            mm[l] = R(l + 1) * mm[l + 1] + prev - u * cur;
            prev = cur;
          }
        }
        for (int l = 0; l <= N; ++l) out[l] = mm[l];
      }
    } else {
      const R v = side ? -u : u;
      R c[4] = {R(1), R(0), R(0), R(0)};
      for (int it = 0; it < k; ++it)
        for (int i = it + 1; i >= 0; --i) c[i] = (i ? c[i - 1] : R(0)) - v * c[i];
      const R sgn = (side && (k & 1)) ? R(-1) : R(1);
      for (int s2 = 0; s2 <= N; ++s2) {
        R acc = R(0);
        for (int i = 0; i <= k; ++i) acc += c[i] * M[2 * ax + side][s2 + i];
        out[s2] = sgn * acc;
      }
    }
  }
  __syncwarp();
  const int nq = m.nq0 + m.nq1;
  for (int x = tid; x < 4 * nq; x += 32) {
    const int k = x / nq, r = x - k * nq, ax = r >= m.nq0 ? 1 : 0, node = r - ax * m.nq0;
    const int kind = ax ? m.kind1 : m.kind0, N = ax ? m.N1 : m.N0;
    const R* tab = ms.tab[ax];
    const int side = (kind == 1 && ms.p[ax][node] < R(0)) ? 1 : 0;
    const R* v = OV[ax * 8 + k * 2 + side];
    R g = R(0);
    for (int s2 = 0; s2 <= N; ++s2) g += tab[node * MAXN + s2] * v[s2];
    (ax ? B : A)[k][node] = g;
  }
  __syncwarp();
}

// One warp per cell (four per CTA): no CTA barrier on a cell's chain, four times the cells in
// flight of a CTA per cell.
template <typename real>
__global__ void __launch_bounds__(128) shakhov_kernel(real* Fout, const real* Fprev, long long cells, int Vp,
                                                      const __grid_constant__ ModelArgs m, const InstDesc* inst,
                                                      int n_inst, double cc, double omp, double kn_fixed) {
  __shared__ real A[4][4][MAXQ], B[4][4][MAXQ], M[4][4][MAXN + 3], OV[4][16][MAXN];  // per warp
  __shared__ ModelSmem<real> ms;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int V = m.nq0 * m.nq1;
  stage_model<real>(m, ms);
  auto wsum = [&](real x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  for (long long c = (long long)blockIdx.x * 4 + w; c < cells; c += (long long)gridDim.x * 4) {
    const real* f = Fprev + c * 2 * Vp;
    // the instance of the cell (its Kn, tau convention and dt): the last with cell0 <= c
    int ii = 0;
    for (int b0 = 0; b0 < n_inst; b0 += 32) {
      const bool in = b0 + lane < n_inst && inst[b0 + lane].cell0 <= c;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (bal) ii = b0 + 31 - __clz(bal);
      if (bal != 0xffffffffu) break;
    }
    // n and n u (Eq. macro_red), F = D + R; every lane gets the sums
    real a = real(0), b = real(0), g = real(0);
    for (int v = lane; v < V; v += 32) {
      const int i = v / m.nq1, j = v - i * m.nq1;
      const real f1 = f[2 * v] + ms.w[0][i] * ms.w[1][j];
      a += f1;
      b += ms.p[0][i] * f1;
      g += ms.p[1][j] * f1;
    }
    const real n = wsum(a), u0 = wsum(b) / n, u1 = wsum(g) / n;
    // 3 n T = sum (xi0^2 + xi1^2) f' + f'',  q = sum [(xi0^2 + xi1^2) f' + f''] xi / 2
    a = b = g = real(0);
    for (int v = lane; v < V; v += 32) {
      const int i = v / m.nq1, j = v - i * m.nq1;
      const real R = ms.w[0][i] * ms.w[1][j];
      const real x0 = ms.p[0][i] - u0, x1 = ms.p[1][j] - u1;
      const real e = (x0 * x0 + x1 * x1) * (f[2 * v] + R) + (f[2 * v + 1] + R);
      a += e;
      b += e * x0;
      g += e * x1;
    }
    const real T = wsum(a) / (real(3) * n), q0 = real(0.5) * wsum(b), q1 = real(0.5) * wsum(g);
    const InstDesc& d = inst[ii];
    const real tau = kn_fixed > 0.0 ? real(kn_fixed) / (n * T) : relaxation_time<real>(d.tau_mode, real(d.kn), n, T);
    const real coef = real(cc * d.dt * omp) / tau;
    const real iT2 = real(1) / (T * T), a0 = q0 * iT2, a1 = q1 * iT2, i5T = real(1) / (real(5) * T);
    power_tables<real>(m, ms, u0, u1, T, M[w], OV[w], A[w], B[w]);
    const real(*Aw)[MAXQ] = A[w];
    const real(*Bw)[MAXQ] = B[w];
    for (int x = lane; x < 2 * V; x += 32) {
      const int v = x >> 1, fi = x & 1;
      const int i = v / m.nq1, j = v - i * m.nq1;
      const real t3a = Aw[3][i] * Bw[0][j] + Aw[1][i] * Bw[2][j], t1a = Aw[1][i] * Bw[0][j];
      const real t3b = Aw[2][i] * Bw[1][j] + Aw[0][i] * Bw[3][j], t1b = Aw[0][i] * Bw[1][j];
      const real G = fi ? a0 * (real(0.2) * t3a - real(0.4) * T * t1a) + a1 * (real(0.2) * t3b - real(0.4) * T * t1b)
                        : a0 * (t3a * i5T - real(0.8) * t1a) + a1 * (t3b * i5T - real(0.8) * t1b);
      real* y = Fout + c * 2 * Vp + x;
      *y = *y + coef * G;
    }
    __syncwarp();  // A, B, M, OV of this warp are rewritten for its next cell
  }
}

template <typename real>
cudaError_t launch_shakhov(real* Fout, const real* Fprev, long long cells, int Vp, const ModelArgs& m,
                           const InstDesc* inst, int n_inst, double cc, double one_minus_pr, double kn_fixed,
                           cudaStream_t s) {
  long long blocks = (cells + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  shakhov_kernel<real><<<int(blocks > 0 ? blocks : 1), 128, 0, s>>>(Fout, Fprev, cells, Vp, m, inst, n_inst, cc,
                                                                    one_minus_pr, kn_fixed);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- caller layout <-> device layout
// Caller rows hold f' then f'' (V values each); device rows hold the deviation
// from R as interleaved (f', f'') pairs of Vp velocities.  One CTA per cell row
// at a time; the row passes through shared memory, so src and dst may be the
// same buffer when V == Vp.
template <typename real>
__global__ void deviation_kernel(const real* src, real* dst, long long cells, int Vp,
                                 const __grid_constant__ ModelArgs m, int to_dev, CellMap map) {
  __shared__ real buf[2 * MAXQ * MAXQ];
  const int V = m.nq0 * m.nq1;
  for (long long c = blockIdx.x; c < cells; c += gridDim.x) {
    const long long cc = caller_cell(map, c);  // device cell c is the caller's cell cc
    if (to_dev) {
      for (int x = threadIdx.x; x < 2 * V; x += blockDim.x) buf[x] = src[cc * 2 * V + x];
      __syncthreads();
      for (int x = threadIdx.x; x < 2 * Vp; x += blockDim.x) {
        const int v = x >> 1, d = x & 1;
        real val = real(0);
        if (v < V) {
          const int i = v / m.nq1, j = v - i * m.nq1;
          val = real(double(buf[d * V + v]) - m.w0[i] * m.w1[j]);
        }
        dst[c * 2 * Vp + x] = val;
      }
    } else {
      for (int x = threadIdx.x; x < 2 * Vp; x += blockDim.x) buf[x] = src[c * 2 * Vp + x];
      __syncthreads();
      for (int x = threadIdx.x; x < 2 * V; x += blockDim.x) {
        const int d = x >= V, v = x - d * V;
        const int i = v / m.nq1, j = v - i * m.nq1;
        dst[cc * 2 * V + x] = real(double(buf[2 * v + d]) + m.w0[i] * m.w1[j]);
      }
    }
    __syncthreads();
  }
}

template <typename real>
cudaError_t launch_deviation(const real* src, real* dst, long long cells, int Vp, const ModelArgs& m,
                             int to_deviation, cudaStream_t s, CellMap map) {
  const long long blocks = cells < 152 * 8 ? cells : 152 * 8;
  deviation_kernel<real><<<int(blocks > 0 ? blocks : 1), 256, 0, s>>>(src, dst, cells, Vp, m, to_deviation, map);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- moments (FP64), one warp per cell
template <typename real>
__global__ void moments_kernel(const real* F, long long cells, int Vp, const __grid_constant__ ModelArgs m,
                               double* out, CellMap map) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int nq1 = m.nq1, V = m.nq0 * m.nq1;
  for (long long c = warp0; c < cells; c += nwarps) {
    const real* f = F + c * 2 * Vp;
    double sn = 0, s0 = 0, s1 = 0;
    for (int v = lane; v < V; v += 32) {
      const int i = v / nq1, j = v - i * nq1;
      const double f1 = double(f[2 * v]) + m.w0[i] * m.w1[j];  // F = D + R
      sn += f1;
      s0 += m.p0[i] * f1;
      s1 += m.p1[j] * f1;
    }
    sn = warp_sum<real>(sn);
    s0 = warp_sum<real>(s0);
    s1 = warp_sum<real>(s1);
    const double n = sn, u0 = s0 / n, u1 = s1 / n;
    double t00 = 0, t01 = 0, t11 = 0, tr2 = 0, q0 = 0, q1 = 0;
    for (int v = lane; v < V; v += 32) {
      const int i = v / nq1, j = v - i * nq1;
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
    t00 = warp_sum<real>(t00);
    t01 = warp_sum<real>(t01);
    t11 = warp_sum<real>(t11);
    tr2 = warp_sum<real>(tr2);
    q0 = warp_sum<real>(q0);
    q1 = warp_sum<real>(q1);
    if (lane == 0) {
      double* o = out + caller_cell(map, c) * 9;  // in the caller's cell order
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
  }
}

template <typename real>
cudaError_t launch_moments(const real* F, long long cells, int Vp, const ModelArgs& m, double* out, cudaStream_t s,
                           CellMap map) {
  long long blocks = (cells * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  moments_kernel<real><<<int(blocks), 256, 0, s>>>(F, cells, Vp, m, out, map);
  return cudaGetLastError();
}

template int stage_variants<VLB_REAL>(int, int, StageVariant*);
template size_t stage_smem_bytes<VLB_REAL>(StageVariant, int);
template bool stage_split_tables<VLB_REAL>(int, int);
template cudaError_t launch_stage<VLB_REAL>(StageVariant, const StageArgs<VLB_REAL>&, const ModelArgs&,
                                            const KArgs<VLB_REAL>&, int, cudaStream_t, bool);
template cudaError_t launch_init_equilibrium<VLB_REAL>(VLB_REAL*, long long, int, const ModelArgs&, double, double,
                                                       double, double, cudaStream_t);
template size_t channel_smem_bytes<VLB_REAL>(ChanVariant, int, int);
template cudaError_t launch_channel<VLB_REAL>(ChanVariant, const ChanArgs<VLB_REAL>&, const void*, int, int, int,
                                              cudaStream_t, bool);
template bool channel_tables<VLB_REAL>(int, int, const AxisTables*, const ModelArgs&, double,
                                       std::vector<unsigned char>*);
template cudaError_t launch_seed<VLB_REAL>(VLB_REAL*, long long, int, const ModelArgs&, const double*,
                                           const double*, const double*, const double*, const double*, cudaStream_t,
                                           CellMap);
template cudaError_t stage_config<VLB_REAL>(StageVariant, const ModelArgs&, int, int*, int*, bool);
template cudaError_t launch_deviation<VLB_REAL>(const VLB_REAL*, VLB_REAL*, long long, int, const ModelArgs&, int,
                                                cudaStream_t, CellMap);
template cudaError_t launch_moments<VLB_REAL>(const VLB_REAL*, long long, int, const ModelArgs&, double*,
                                              cudaStream_t, CellMap);
template cudaError_t launch_shakhov<VLB_REAL>(VLB_REAL*, const VLB_REAL*, long long, int, const ModelArgs&,
                                              const InstDesc*, int, double, double, double, cudaStream_t);

}  // namespace vlb
