// The ESDIRK tableau of the solver's second method, derived once on the host.
//
// The paper's code integrates with Kvaerno's fifth-order ESDIRK (Sec. 4;
// Kvaerno, BIT 44, 2004) and prints no coefficients. The member of that family
// used here has order 4 with an embedded order-3 solution and five stages,
// fixed by the family's defining conditions:
//   - explicit first stage (c_1 = 0, a_1j = 0), diagonal a_ii = gamma (i >= 2);
//   - stage order 2: sum_j a_ij = c_i, sum_j a_ij c_j = c_i^2 / 2 (so c_2 = 2 gamma);
//   - c_4 = c_5 = 1: row 4 is the embedded solution (moment conditions
//     sum_j a_4j c_j^k = 1/(k+1), k = 0..2), row 5 the solution (k = 0..3);
//   - the remaining order-4 condition sum_i b_i (A c^2)_i = 1/12 fixes c_3;
//   - L-stability, R(infinity) = 0, fixes gamma.
// With gamma and c_3 given, every row is a small linear (Vandermonde) system;
// c_3(gamma) and gamma are roots found by bisection.
#include <cmath>

#include "internal.h"

namespace cbx {
namespace {

// Solve the n x n system M x = r (n <= 4) by Gaussian elimination with partial pivoting.
void solve_small(int n, double M[4][4], double r[4], double x[4]) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(M[i][k]) > std::fabs(M[p][k])) p = i;
    for (int j = 0; j < n; ++j) std::swap(M[k][j], M[p][j]);
    std::swap(r[k], r[p]);
    for (int i = k + 1; i < n; ++i) {
      const double f = M[i][k] / M[k][k];
      for (int j = k; j < n; ++j) M[i][j] -= f * M[k][j];
      r[i] -= f * r[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
}

// Row i (i = 3: embedded, order 3; i = 4: solution, order 4) from the moment
// conditions sum_{j<i} a_ij c_j^k = 1/(k+1) - gamma (c_i = 1), k = 0..i-1.
void moment_row(double A[5][5], const double c[5], double gamma, int i) {
  double M[4][4], r[4], x[4];
  for (int k = 0; k < i; ++k) {
    for (int j = 0; j < i; ++j) M[k][j] = std::pow(c[j], k);
    r[k] = 1.0 / (k + 1) - gamma;
  }
  solve_small(i, M, r, x);
  for (int j = 0; j < i; ++j) A[i][j] = x[j];
  A[i][i] = gamma;
}

void rows(double gamma, double c3, double A[5][5], double c[5]) {
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) A[i][j] = 0.0;
  c[0] = 0.0;
  c[1] = 2.0 * gamma;
  c[2] = c3;
  c[3] = c[4] = 1.0;
  A[1][0] = A[1][1] = gamma;
  A[2][2] = gamma;
  A[2][1] = (0.5 * c3 * c3 - gamma * c3) / c[1];
  A[2][0] = c3 - gamma - A[2][1];
  moment_row(A, c, gamma, 3);
  moment_row(A, c, gamma, 4);
}

double tree_bac2(double gamma, double c3) {
  double A[5][5], c[5];
  rows(gamma, c3, A, c);
  double s = 0.0;
  for (int i = 0; i < 5; ++i) {
    double ac2 = 0.0;
    for (int j = 0; j < 5; ++j) ac2 += A[i][j] * c[j] * c[j];
    s += A[4][i] * ac2;
  }
  return s - 1.0 / 12.0;
}

template <typename F>
double bisect(F f, double lo, double hi) {
  double flo = f(lo);
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const double fm = f(mid);
    if ((fm < 0.0) == (flo < 0.0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

double c3_of(double gamma) {
  return bisect([&](double x) { return tree_bac2(gamma, x); }, 0.4, 0.8);
}

// R(infinity) of the stiffly accurate method: stages 2..5 tend to
// -A~^{-1} a y0 (A~ the implicit lower-triangular block, a its first column);
// R(infinity) is the last component. Forward substitution.
double r_infinity(double gamma) {
  double A[5][5], c[5];
  rows(gamma, c3_of(gamma), A, c);
  double x[5];
  for (int i = 1; i < 5; ++i) {
    double s = A[i][0];
    for (int j = 1; j < i; ++j) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
  return -x[4];
}

EsdirkTableau derive() {
  EsdirkTableau t;
  t.gamma = bisect(r_infinity, 0.56, 0.59);
  rows(t.gamma, c3_of(t.gamma), t.a, t.c);
  return t;
}

}  // namespace

const EsdirkTableau& esdirk_tableau() {
  static const EsdirkTableau t = derive();
  return t;
}

}  // namespace cbx

extern "C" int cbx_esdirk_tableau(double* a, double* c, double* gamma) {
  const cbx::EsdirkTableau& t = cbx::esdirk_tableau();
  if (a)
    for (int i = 0; i < 25; ++i) a[i] = t.a[i / 5][i % 5];
  if (c)
    for (int i = 0; i < 5; ++i) c[i] = t.c[i];
  if (gamma) *gamma = t.gamma;
  return CBX_OK;
}
