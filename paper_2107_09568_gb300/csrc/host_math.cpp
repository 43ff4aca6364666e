// Host-side numerics used while planning: Gauss-Legendre rules and B-spline
// bases on one knot span.  Nothing here runs on the hot path.
#include <cmath>
#include <vector>

#include "common.h"

namespace msasm {

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  // Roots of P_n by Newton's method from the Chebyshev-like first guess; the
  // three-term recurrence (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1} gives P_n and
  // P_n' = n (t P_n - P_{n-1}) / (t^2 - 1).  Weight 2 / ((1 - t^2) P_n'(t)^2) on [-1,1].
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double t = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 0) ? 1.0 : p1;
      double pm = (n == 1) ? 1.0 : p0;
      if (n == 1) { pn = t; pm = 1.0; }
      dp = n * (t * pn - pm) / (t * t - 1.0);
      double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    // recompute the derivative at the converged root for the weight
    double p0 = 1.0, p1 = t;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    double pn = p1, pm = (n == 1) ? 1.0 : p0;
    dp = n * (t * pn - pm) / (t * t - 1.0);
    // map to [0,1], ascending order
    x[n - 1 - i] = 0.5 * (1.0 + t);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);  // = 0.5 * 2 / (...)
  }
}

int bspline_find_span(const double* t, int n_knots, int p, double u) {
  int n = n_knots - p - 1;  // number of basis functions
  if (u >= t[n]) {
    // last non-empty span
    int k = n - 1;
    while (k > p && !(t[k + 1] > t[k])) --k;
    return k;
  }
  int k = p;
  while (k < n - 1 && u >= t[k + 1]) ++k;
  return k;
}

// Triangular Cox-de Boor recursion over the degree+1 functions alive on the span.
static void span_values(const double* t, int p, int span, double u, double* N) {
  double left[16], right[16];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = u - t[span + 1 - j];
    right[j] = t[span + j] - u;
    double carry = 0.0;
    for (int r = 0; r < j; ++r) {
      double f = N[r] / (right[r + 1] + left[j - r]);
      N[r] = carry + right[r + 1] * f;
      carry = left[j - r] * f;
    }
    N[j] = carry;
  }
}

void bspline_span_basis(const double* t, int p, int span, double u, double* vals, double* ders) {
  span_values(t, p, span, u, vals);
  if (p == 0) {
    ders[0] = 0.0;
    return;
  }
  double low[16];
  span_values(t, p - 1, span, u, low);  // functions span-p+1 .. span of degree p-1
  for (int k = 0; k <= p; ++k) {
    int i = span - p + k;
    double a = (k >= 1) ? low[k - 1] : 0.0;          // N_{i, p-1}
    double b = (k <= p - 1) ? low[k] : 0.0;          // N_{i+1, p-1}
    double da = t[i + p] - t[i], db = t[i + p + 1] - t[i + 1];
    ders[k] = (da > 0 ? p * a / da : 0.0) - (db > 0 ? p * b / db : 0.0);
  }
}

}  // namespace msasm
