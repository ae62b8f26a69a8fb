// Host Gauss-Lobatto-Legendre tables for every supported order (Section 3, Eq. 3):
// nodes, quadrature weights and the collocation derivative matrix D_ij = l_j'(xi_i).
#include <cmath>
#include <mutex>

#include "sem_internal.h"

namespace sem {
namespace {

// L_N and L_N' at x by the Bonnet recurrence, in long double.
void legendre(int N, long double x, long double& L, long double& dL) {
  long double lm1 = 1.0L, l = x;  // L_0, L_1
  if (N == 0) { L = 1.0L; dL = 0.0L; return; }
  for (int k = 1; k < N; ++k) {
    long double lp1 = ((2 * k + 1) * x * l - k * lm1) / (k + 1);
    lm1 = l;
    l = lp1;
  }
  L = l;
  // (1 - x^2) L_N' = N (L_{N-1} - x L_N); only used at interior points
  dL = (1.0L - x * x) != 0.0L ? N * (lm1 - x * l) / (1.0L - x * x) : 0.0L;
}

GllTable make_table(int N) {
  GllTable t{};
  const int Np = N + 1;
  long double x[kMaxNp];
  x[0] = -1.0L;
  x[N] = 1.0L;
  for (int j = 1; j < N; ++j) {
    // Newton on L_N' from the Chebyshev-Gauss-Lobatto guess; L_N'' from Legendre's equation.
    long double r = -std::cos(static_cast<long double>(M_PI) * j / N);
    for (int it = 0; it < 60; ++it) {
      long double L, dL;
      legendre(N, r, L, dL);
      long double d2L = (2.0L * r * dL - N * (N + 1.0L) * L) / (1.0L - r * r);
      long double step = dL / d2L;
      r -= step;
      if (std::fabs(step) < 1e-22L) break;
    }
    x[j] = r;
  }
  long double LN[kMaxNp];
  for (int j = 0; j < Np; ++j) {
    long double dL;
    legendre(N, x[j], LN[j], dL);
    t.xi[j] = static_cast<double>(x[j]);
    t.w[j] = static_cast<double>(2.0L / (N * (N + 1.0L) * LN[j] * LN[j]));
  }
  // D_ij = L_N(x_i) / (L_N(x_j) (x_i - x_j)) off the diagonal; -N(N+1)/4, +N(N+1)/4 at the
  // two end points and 0 elsewhere on the diagonal.
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      long double d;
      if (i != j) d = LN[i] / (LN[j] * (x[i] - x[j]));
      else if (i == 0) d = -N * (N + 1.0L) / 4.0L;
      else if (i == N) d = N * (N + 1.0L) / 4.0L;
      else d = 0.0L;
      t.D[i * Np + j] = static_cast<double>(d);
    }
  return t;
}

}  // namespace

const GllTable& gll_table(int N) {
  static GllTable tabs[SEM_MAX_N + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int n = 1; n <= SEM_MAX_N; ++n) tabs[n] = make_table(n);
  });
  return tabs[N];
}

}  // namespace sem
