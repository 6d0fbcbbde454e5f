// Momentum-space tables of the mixed-quadrature LB models (Sec. IV.B-D), built
// on the host in long double (IEEE binary128 on aarch64) and rounded to double.
//
// Route (chosen to be independent of the closed forms printed in the paper,
// which the tests compare against):
//  * the weight omega(x) = exp(-x^2/2)/sqrt(2 pi) on [0, inf) (half range) or
//    on the real line (full range) is discretised by composite Gauss-Legendre
//    panels on [0, L] or [-L, L], L = 40 (48 points per panel of width 0.5: the
//    projections of K below integrate products of degree ~2Q; 24 points lost K at Q = 200);
//  * the Stieltjes procedure on that discrete measure gives the three-term
//    recurrence of the orthonormal family psi_l (h_l for the half range, the
//    normalised Hermite polynomials for the full range);
//  * nodes are the eigenvalues of the Jacobi matrix (Sturm bisection, then
//    Newton polishing) and weights the Christoffel numbers 1 / sum_l psi_l(x)^2;
//  * K and K~ are built from their definition (Sec. IV.C, App. D): expand f in
//    psi_l by the quadrature, differentiate the expansion, project back onto
//    psi_s with the discrete measure, and, for the half range, add the jump
//    term delta(p) [f^+(0) - f^-(0)], half of whose projection falls on each
//    semi-axis.
#include "vlb_tables.h"

#include <cmath>
#include <cstdio>

namespace vlb {
namespace {

typedef long double LD;

const LD kPi = 3.141592653589793238462643383279502884197L;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<LD>* x, std::vector<LD>* w) {
  x->assign(n, 0);
  w->assign(n, 0);
  for (int k = 0; k < n; ++k) {
    LD z = cosl(kPi * (k + 0.75L) / (n + 0.5L));
    LD dp = 1;
    for (int it = 0; it < 100; ++it) {
      LD p0 = 1, p1 = z;
      for (int j = 2; j <= n; ++j) {
        LD p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1);
      LD dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-32L) break;
    }
    (*x)[k] = z;
    (*w)[k] = 2 / ((1 - z * z) * dp * dp);
  }
}

struct Measure {
  std::vector<LD> x, W;  // points and weights (omega folded in)
};

Measure discretise(bool half) {
  const LD L = 40, width = 0.5L;
  const int per = 48;  // per panel of width 0.5: resolves the products of the degree-~2Q polynomials up to Q = 200
  std::vector<LD> gx, gw;
  gauss_legendre(per, &gx, &gw);
  Measure m;
  LD a0 = half ? 0 : -L;
  int panels = (int)((L - a0) / width + 0.5L);
  for (int q = 0; q < panels; ++q) {
    LD a = a0 + q * width, b = a + width;
    for (int k = 0; k < per; ++k) {
      LD t = 0.5L * (a + b) + 0.5L * (b - a) * gx[k];
      m.x.push_back(t);
      m.W.push_back(0.5L * (b - a) * gw[k] * expl(-t * t / 2) / sqrtl(2 * kPi));
    }
  }
  return m;
}

// Orthonormal recurrence: b_{k+1} psi_{k+1} = (x - alpha_k) psi_k - b_k psi_{k-1}, psi_0 = 1/sqrt(mu0).
struct Recurrence {
  std::vector<LD> alpha, b;  // b[0] unused
  LD psi0;
};

Recurrence stieltjes(const Measure& m, int n) {
  size_t M = m.x.size();
  std::vector<LD> pm(M, 0), pc(M, 1), pn(M);
  Recurrence r;
  LD mu0 = 0;
  for (size_t i = 0; i < M; ++i) mu0 += m.W[i];
  r.psi0 = 1 / sqrtl(mu0);
  for (size_t i = 0; i < M; ++i) pc[i] = r.psi0;
  r.alpha.assign(n + 1, 0);
  r.b.assign(n + 2, 0);
  for (int k = 0; k <= n; ++k) {
    LD a = 0;
    for (size_t i = 0; i < M; ++i) a += m.W[i] * m.x[i] * pc[i] * pc[i];
    r.alpha[k] = a;
    LD nn = 0;
    for (size_t i = 0; i < M; ++i) {
      pn[i] = (m.x[i] - a) * pc[i] - r.b[k] * pm[i];
      nn += m.W[i] * pn[i] * pn[i];
    }
    LD bk = sqrtl(nn);
    r.b[k + 1] = bk;
    for (size_t i = 0; i < M; ++i) {
      pm[i] = pc[i];
      pc[i] = pn[i] / bk;
    }
  }
  return r;
}

// psi_0..psi_n and their derivatives at x.
void eval_psi(const Recurrence& r, int n, LD x, LD* v, LD* d) {
  v[0] = r.psi0;
  if (d) d[0] = 0;
  for (int k = 0; k < n; ++k) {
    LD prev = k ? v[k - 1] : 0, dprev = (k && d) ? d[k - 1] : 0;
    v[k + 1] = ((x - r.alpha[k]) * v[k] - r.b[k] * prev) / r.b[k + 1];
    if (d) d[k + 1] = (v[k] + (x - r.alpha[k]) * d[k] - r.b[k] * dprev) / r.b[k + 1];
  }
}

// Eigenvalues of the n x n Jacobi matrix by Sturm-count bisection plus Newton on psi_n.
std::vector<LD> jacobi_eigenvalues(const Recurrence& r, int n, LD lo, LD hi) {
  auto below = [&](LD x) {
    int cnt = 0;
    LD d = 1;
    for (int k = 0; k < n; ++k) {
      LD off = k ? r.b[k] * r.b[k] / d : 0;
      d = (r.alpha[k] - x) - off;
      if (d == 0) d = 1e-300L;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  std::vector<LD> ev(n);
  std::vector<LD> v(n + 2), dv(n + 2);
  for (int k = 0; k < n; ++k) {
    LD a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      LD mid = 0.5L * (a + b);
      if (below(mid) > k) b = mid; else a = mid;
      if (b - a < 1e-24L * (1 + fabsl(a))) break;
    }
    LD x = 0.5L * (a + b);
    for (int it = 0; it < 8; ++it) {
      eval_psi(r, n, x, v.data(), dv.data());
      if (dv[n] == 0) break;
      LD dx = v[n] / dv[n];
      x -= dx;
      if (fabsl(dx) < 1e-33L * (1 + fabsl(x))) break;
    }
    ev[k] = x;
  }
  return ev;
}

// Monomial coefficients c[l][s] of psi_l, l = 0..n.
std::vector<std::vector<LD>> psi_coeffs(const Recurrence& r, int n) {
  std::vector<std::vector<LD>> c(n + 1, std::vector<LD>(n + 1, 0));
  c[0][0] = r.psi0;
  for (int k = 0; k < n; ++k) {
    for (int s = 0; s <= k + 1; ++s) {
      LD v = (s ? c[k][s - 1] : 0) - r.alpha[k] * c[k][s] - (k ? r.b[k] * c[k - 1][s] : 0);
      c[k + 1][s] = v / r.b[k + 1];
    }
  }
  return c;
}

}  // namespace

bool build_axis(int kind, int N, int Q, AxisTables* out, std::string* err) {
  if (Q < 1 || N < 0 || N >= Q) {
    *err = "expansion order must satisfy 0 <= N < Q";
    return false;
  }
  const bool half = (kind == 1);
  Measure m = discretise(half);
  Recurrence r = stieltjes(m, Q + 1);
  // positive (half) or all (full) nodes
  LD hi = 6 + 3 * sqrtl((LD)Q);
  std::vector<LD> x = jacobi_eigenvalues(r, Q, half ? 0 : -hi, hi);
  std::vector<LD> wq(Q);
  std::vector<LD> v(Q + 2), dv(Q + 2);
  for (int k = 0; k < Q; ++k) {
    eval_psi(r, Q, x[k], v.data(), nullptr);
    LD s = 0;
    for (int l = 0; l < Q; ++l) s += v[l] * v[l];
    wq[k] = 1 / s;
  }
  const int nq = half ? 2 * Q : Q;
  std::vector<LD> P(nq), Wt(nq), X(nq);
  std::vector<int> sig(nq, 1);
  for (int k = 0; k < Q; ++k) {
    P[k] = x[k];
    Wt[k] = wq[k];
    X[k] = x[k];
    if (half) {
      P[Q + k] = -x[k];
      Wt[Q + k] = wq[k];
      X[Q + k] = x[k];
      sig[Q + k] = -1;
    }
  }
  // psi_l at |p_k| and at 0
  std::vector<std::vector<LD>> psi(nq, std::vector<LD>(Q + 1));
  for (int k = 0; k < nq; ++k) eval_psi(r, Q, X[k], psi[k].data(), nullptr);
  std::vector<LD> psi_at0(Q + 1);
  eval_psi(r, Q, 0, psi_at0.data(), nullptr);

  // projection of the differentiated basis: D[s][l] = int omega (psi_l' - x psi_l) psi_s,
  // Dt[s][l] = int omega ((x psi_l)' - x^2 psi_l) psi_s, over the axis' support
  std::vector<LD> D(Q * Q, 0), Dt(Q * Q, 0);
  for (size_t i = 0; i < m.x.size(); ++i) {
    LD xi = m.x[i];
    eval_psi(r, Q, xi, v.data(), dv.data());
    for (int s = 0; s < Q; ++s) {
      LD ws = m.W[i] * v[s];
      for (int l = 0; l < Q; ++l) {
        D[s * Q + l] += ws * (dv[l] - xi * v[l]);
        Dt[s * Q + l] += ws * (v[l] + xi * dv[l] - xi * xi * v[l]);
      }
    }
  }
  const LD om0 = 1 / sqrtl(2 * kPi);
  out->kind = kind;
  out->N = N;
  out->Q = Q;
  out->nq = nq;
  out->p.resize(nq);
  out->w.resize(nq);
  out->K.assign(nq * nq, 0);
  out->Kt.assign(nq * nq, 0);
  for (int k = 0; k < nq; ++k) {
    out->p[k] = (double)P[k];
    out->w[k] = (double)Wt[k];
  }
  // the projections of the expanded node function kp on psi_s do not depend on the output
  // node k: C[s][kp] = sum_l D[s][l] psi_l(|p_kp|) (likewise Ct), and the jump term's
  // f(0) = sum_l psi_l(0) psi_l(|p_kp|); then K[k][kp] = w_k sum_s psi_s(|p_k|) (...)
  std::vector<LD> C(size_t(Q) * nq), Ct(size_t(Q) * nq), f0v(nq, 0);
  for (int kp = 0; kp < nq; ++kp) {
    for (int l = 0; l < Q; ++l) f0v[kp] += psi_at0[l] * psi[kp][l];
    for (int s = 0; s < Q; ++s) {
      LD cs = 0, cts = 0;
      for (int l = 0; l < Q; ++l) {
        cs += D[s * Q + l] * psi[kp][l];
        cts += Dt[s * Q + l] * psi[kp][l];
      }
      C[size_t(s) * nq + kp] = cs;
      Ct[size_t(s) * nq + kp] = cts;
    }
  }
  for (int k = 0; k < nq; ++k) {
    for (int kp = 0; kp < nq; ++kp) {
      LD acc = 0, acct = 0;
      for (int s = 0; s < Q; ++s) {
        LD cs = 0, cts = 0;
        if (sig[k] == sig[kp]) {
          cs = C[size_t(s) * nq + kp] * sig[k];  // d/dp = sigma d/d|p| on each semi-axis
          cts = Ct[size_t(s) * nq + kp];
        }
        if (half) cs += 0.5L * psi_at0[s] * om0 * sig[kp] * f0v[kp];  // half of delta(p) on each semi-axis
        acc += psi[k][s] * cs;
        acct += psi[k][s] * cts;
      }
      out->K[k * nq + kp] = (double)(Wt[k] * acc);
      out->Kt[k * nq + kp] = (double)(Wt[k] * acct);
    }
  }
  // equilibrium table
  out->eqtab.assign(nq * (N + 1), 0);
  if (half) {
    // g_k = w_k sum_l c_l h_l(|p_k|), c_l = sum_s h_{l,s} M_s (M_s: half-line moments of the
    // Gaussian on the semi-axis of p_k): eqtab[k][s] = w_k sum_{l=s}^{N} h_{l,s} h_l(|p_k|)
    auto c = psi_coeffs(r, N);
    for (int k = 0; k < nq; ++k)
      for (int s = 0; s <= N; ++s) {
        LD a = 0;
        for (int l = s; l <= N; ++l) a += c[l][s] * psi[k][l];
        out->eqtab[k * (N + 1) + s] = (double)(Wt[k] * a);
      }
  } else {
    // g_k = w_k sum_l He_l(p_k) c_l(u, T): eqtab[k][l] = w_k He_l(p_k), He_l = sqrt(l!) psi_l
    for (int k = 0; k < nq; ++k) {
      LD fact = 1;
      for (int l = 0; l <= N; ++l) {
        if (l) fact *= l;
        out->eqtab[k * (N + 1) + l] = (double)(Wt[k] * sqrtl(fact) * psi[k][l]);
      }
    }
  }
  return true;
}

}  // namespace vlb
