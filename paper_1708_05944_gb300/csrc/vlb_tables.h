// Host-side construction of the momentum-space tables of one model axis.
#pragma once
#include <string>
#include <vector>

namespace vlb {

// Tables of one axis of HH(N;Q) or H(N;Q) (Sec. IV.B-D).
struct AxisTables {
  int kind = 0;  // 0 full range, 1 half range
  int N = 0, Q = 0, nq = 0;
  std::vector<double> p, w;     // nodes and weights, nq each
  std::vector<double> K, Kt;    // nq x nq row-major: [d_p f]_k = sum_k' K[k][k'] f_k', [d_p (p f)]_k likewise with Kt
  std::vector<double> eqtab;    // nq x (N+1): g_k = sum_s eqtab[k][s] m_s (see eq_moment_vector in the kernels)
};

// Build the tables; returns false and fills *err on failure.
bool build_axis(int kind, int N, int Q, AxisTables* out, std::string* err);

}  // namespace vlb
