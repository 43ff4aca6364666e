// Small dense linear algebra on the host (n <= 128), used only while fitting the surrogate's
// low-rank basis: Cholesky factorisation with an inverse of the factor, and the cyclic Jacobi
// eigenvalue method for symmetric matrices (Golub & Van Loan, Sec. 8.5).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace msasm {

// A = R^T R (R upper triangular); returns false if A is not positive definite.
// On success Rinv holds R^-1 (upper triangular), row-major n x n.
bool cholesky_upper_inverse(const std::vector<double>& A, int n, std::vector<double>& Rinv) {
  std::vector<double> R(size_t(n) * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[size_t(j) * n + j];
    for (int k = 0; k < j; ++k) s -= R[size_t(k) * n + j] * R[size_t(k) * n + j];
    if (!(s > 0.0)) return false;
    const double rjj = std::sqrt(s);
    R[size_t(j) * n + j] = rjj;
    for (int i = j + 1; i < n; ++i) {
      double t = A[size_t(j) * n + i];
      for (int k = 0; k < j; ++k) t -= R[size_t(k) * n + j] * R[size_t(k) * n + i];
      R[size_t(j) * n + i] = t / rjj;
    }
  }
  Rinv.assign(size_t(n) * n, 0.0);
  for (int j = 0; j < n; ++j) {          // back substitution, column by column of the identity
    for (int i = j; i >= 0; --i) {
      double t = (i == j) ? 1.0 : 0.0;
      for (int k = i + 1; k <= j; ++k) t -= R[size_t(i) * n + k] * Rinv[size_t(k) * n + j];
      Rinv[size_t(i) * n + j] = t / R[size_t(i) * n + i];
    }
  }
  return true;
}

// Eigen-decomposition of a symmetric n x n matrix: eigenvalues descending in w, eigenvectors as
// the columns of V (row-major), by cyclic Jacobi rotations until the off-diagonal part vanishes.
void symmetric_eigen(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V) {
  V.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
  auto at = [&](int i, int j) -> double& { return A[size_t(i) * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += at(i, j) * at(i, j);
        if (i != j) off += at(i, j) * at(i, j);
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = at(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {          // A <- A J
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {          // A <- J^T A
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {          // V <- V J
          const double vkp = V[size_t(k) * n + p], vkq = V[size_t(k) * n + q];
          V[size_t(k) * n + p] = c * vkp - s * vkq;
          V[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return at(a, a) > at(b, b); });
  w.resize(n);
  std::vector<double> Vs(size_t(n) * n);
  for (int j = 0; j < n; ++j) {
    w[j] = at(order[j], order[j]);
    for (int i = 0; i < n; ++i) Vs[size_t(i) * n + j] = V[size_t(i) * n + order[j]];
  }
  V.swap(Vs);
}

}  // namespace msasm
