// spline.cpp -- TEST INFRASTRUCTURE ONLY (see oracle.hpp).
// Univariate B-splines of Sec. 2.1 and Gauss-Legendre quadrature.
#include <cmath>
#include <stdexcept>

#include "oracle.hpp"

namespace oracle {

int64_t Csr::find(int64_t i, int32_t j) const {
  int64_t lo = ptr[i], hi = ptr[i + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (col[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  return (lo < ptr[i + 1] && col[lo] == j) ? lo : -1;
}

// Sec. 2.1: open knot vector (end multiplicity q+1), breakpoints k/N of
// multiplicity 1, so the regularity at interior breakpoints is alpha = q-1.
Knots open_uniform(int N, int q) {
  Knots K;
  K.N = N;
  K.q = q;
  for (int i = 0; i < q; ++i) K.xi.push_back(0.0);
  for (int k = 0; k <= N; ++k) K.xi.push_back((double)k / N);
  for (int i = 0; i < q; ++i) K.xi.push_back(1.0);
  return K;  // N + 2q + 1 knots = nfun + q + 1
}

// Quotient used by the Cox-de Boor recursion with the convention 0/0 = 0.
static double ratio(double num, double den) { return den == 0.0 ? 0.0 : num / den; }

// Cox-de Boor recursion (Sec. 2.1), written from its definition:
//   B_{i,0}(x) = 1 on the knot span of the element, 0 elsewhere,
//   B_{i,r}(x) = (x - xi_i)/(xi_{i+r} - xi_i) B_{i,r-1}(x)
//              + (xi_{i+r+1} - x)/(xi_{i+r+1} - xi_{i+1}) B_{i+1,r-1}(x),
//   B'_{i,q}(x) = q/(xi_{i+q} - xi_i) B_{i,q-1}(x)
//               - q/(xi_{i+q+1} - xi_{i+1}) B_{i+1,q-1}(x).
// Element e is the knot span [xi_{e+q}, xi_{e+q+1}); we fix the span instead
// of searching for it, so that x on the closed right end is handled.
void eval_basis(const Knots& K, int e, double x, double* val, double* der) {
  const int q = K.q;
  const int s = e + q;  // knot span index
  const std::vector<double>& xi = K.xi;
  // table[r][i - (s - q)] holds B_{i,r} for i in [s-q, s]; only i in
  // [s-r, s] can be nonzero at degree r.
  double table[16][16];
  for (int r = 0; r <= q; ++r)
    for (int t = 0; t <= q; ++t) table[r][t] = 0.0;
  table[0][q] = 1.0;  // B_{s,0}
  for (int r = 1; r <= q; ++r) {
    for (int i = s - r; i <= s; ++i) {
      const int t = i - (s - q);
      double left = (t >= 0 && t <= q) ? table[r - 1][t] : 0.0;
      double right = (t + 1 <= q) ? table[r - 1][t + 1] : 0.0;
      table[r][t] = ratio(x - xi[i], xi[i + r] - xi[i]) * left +
                    ratio(xi[i + r + 1] - x, xi[i + r + 1] - xi[i + 1]) * right;
    }
  }
  for (int t = 0; t <= q; ++t) {
    const int i = s - q + t;  // function index == e + t
    val[t] = table[q][t];
    if (q == 0) {
      der[t] = 0.0;
      continue;
    }
    double left = table[q - 1][t];
    double right = (t + 1 <= q) ? table[q - 1][t + 1] : 0.0;
    der[t] = ratio(q, xi[i + q] - xi[i]) * left - ratio(q, xi[i + q + 1] - xi[i + 1]) * right;
  }
}

void eval_one(const Knots& K, int i, int e, double x, double* v, double* d) {
  double val[16], der[16];
  eval_basis(K, e, x, val, der);
  int t = i - e;
  if (t < 0 || t > K.q) {
    *v = 0.0;
    *d = 0.0;
  } else {
    *v = val[t];
    *d = der[t];
  }
}

// Gauss-Legendre nodes and weights on [-1,1]: Newton iteration on the
// Legendre polynomial P_n, evaluated by the three-term recurrence
// (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  if (n < 1 || n > 15) throw std::runtime_error("gauss_legendre: n out of range");
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? z : p1;
    double pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (z * pn - pnm1) / (z * z - 1.0);
    x[n - 1 - i] = z;  // ascending order
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace oracle
