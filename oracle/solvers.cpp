// solvers.cpp -- TEST INFRASTRUCTURE ONLY (see oracle.hpp).
// Sec. 5: preconditioned MINRES on the Stokes matrix with the block diagonal
// preconditioner diag(M_A, M_Q) of eq. general_precond_M, where M_A^{-1} is a
// relaxed inner conjugate-gradient solve on A_h preconditioned by IC(0)
// (Sec. 6.4) and M_Q = Diag(Q_nu), Q_nu = Q/(2 nu) (Sec. 5.1), or a CG solve
// with Q_nu preconditioned by IC(0) of Q (Sec. 6.4, "IC(0)-PCG(A,Q)").
#include <cmath>
#include <stdexcept>

#include "oracle.hpp"

namespace oracle {

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

void spmv(const Csr& M, const double* x, double* y) {
  for (int64_t i = 0; i < M.nrows; ++i) {
    double s = 0.0;
    for (int64_t t = M.ptr[i]; t < M.ptr[i + 1]; ++t) s += M.val[t] * x[M.col[t]];
    y[i] = s;
  }
}

// [y_u; y_p] = [A B^T; B 0] [x_u; x_p]   (eq. stokes_linsys)
void stokes_apply(const Problem& P, const double* x, double* y) {
  const double* xu = x;
  const double* xp = x + P.n_u;
  double* yu = y;
  double* yp = y + P.n_u;
  spmv(P.A, xu, yu);
  for (int64_t k = 0; k < P.B.nrows; ++k)
    for (int64_t t = P.B.ptr[k]; t < P.B.ptr[k + 1]; ++t) yu[P.B.col[t]] += P.B.val[t] * xp[k];
  spmv(P.B, xu, yp);
}

// IC(0) (Sec. 6.4): L L^T = perm A perm^T on every position of the lower
// pattern, with no fill.  Row i (in permuted order) is computed from rows
// k < i:  L_ik = (A_ik - sum_{j<k, j in pat(i) and pat(k)} L_ij L_kj) / L_kk,
//         L_ii = sqrt(A_ii - sum_{k<i} L_ik^2).
int64_t ic0(const Csr& A, const std::vector<int32_t>& perm, Csr& L) {
  const int64_t n = L.nrows;
  std::vector<int64_t> mark(n, -1);
  std::vector<double> li(n, 0.0);  // entries of the current row, by column
  for (int64_t i = 0; i < n; ++i) {
    const int64_t b = L.ptr[i], e = L.ptr[i + 1];
    if (e - b < 1 || L.col[e - 1] != i) throw std::runtime_error("ic0: missing diagonal");
    for (int64_t t = b; t < e; ++t) mark[L.col[t]] = i;
    double diag = 0.0;
    for (int64_t t = b; t < e - 1; ++t) {
      const int32_t k = L.col[t];
      int64_t pos = A.find(perm[i], perm[k]);
      double s = A.val[pos];
      for (int64_t u = L.ptr[k]; u < L.ptr[k + 1] - 1; ++u) {
        const int32_t j = L.col[u];  // j < k
        if (mark[j] == i) s -= li[j] * L.val[u];
      }
      const double lkk = L.val[L.ptr[k + 1] - 1];
      const double lik = s / lkk;
      li[k] = lik;
      L.val[t] = lik;
      diag += lik * lik;
    }
    const double aii = A.val[A.find(perm[i], perm[i])];
    const double piv = aii - diag;
    if (!(piv > 0.0)) return i;
    L.val[e - 1] = std::sqrt(piv);
  }
  return -1;
}

// z = (L L^T)^{-1} r in permuted numbering: forward then backward solve.
static void ic0_solve(const Csr& L, const double* r, double* z, std::vector<double>& y) {
  const int64_t n = L.nrows;
  y.assign(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    double s = r[i];
    for (int64_t t = L.ptr[i]; t < L.ptr[i + 1] - 1; ++t) s -= L.val[t] * y[L.col[t]];
    y[i] = s / L.val[L.ptr[i + 1] - 1];
  }
  // L^T z = y, column sweep over the rows of L from the last one
  for (int64_t i = 0; i < n; ++i) z[i] = y[i];
  for (int64_t i = n - 1; i >= 0; --i) {
    z[i] /= L.val[L.ptr[i + 1] - 1];
    for (int64_t t = L.ptr[i]; t < L.ptr[i + 1] - 1; ++t) z[L.col[t]] -= L.val[t] * z[i];
  }
}

static void ic0_apply(const Csr& L, const std::vector<int32_t>& perm, const double* r, double* z) {
  const int64_t n = L.nrows;
  std::vector<double> rp(n), zp(n), tmp;
  for (int64_t i = 0; i < n; ++i) rp[i] = r[perm[i]];
  ic0_solve(L, rp.data(), zp.data(), tmp);
  for (int64_t i = 0; i < n; ++i) z[perm[i]] = zp[i];
}

// Preconditioned CG on the SPD matrix Mat with the IC(0) factor L of
// perm Mat perm^T (Sec. 5.1 "PCG", Sec. 6.4 with IC(0)): x_0 = 0; stop when
// ||r||_2 <= tol ||b||_2 or after max_it iterations; with forced_its >= 0
// exactly forced_its iterations are run.  The count is the number of
// products with Mat.
static int pcg(const Csr& Mat, const Csr& L, const std::vector<int32_t>& perm, double tol, int max_it,
               const double* b, double* x, int forced_its) {
  const int64_t n = Mat.nrows;
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  const double bnorm = std::sqrt(dot(b, b, n));
  if (bnorm == 0.0 || forced_its == 0) return 0;
  std::vector<double> r(b, b + n), z(n), p(n), q(n);
  ic0_apply(L, perm, r.data(), z.data());
  p = z;
  double rho = dot(r.data(), z.data(), n);
  int it = 0;
  for (;;) {
    spmv(Mat, p.data(), q.data());
    ++it;
    const double alpha = rho / dot(p.data(), q.data(), n);
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    if (forced_its > 0) {
      if (it >= forced_its) break;
    } else {
      const double rnorm = std::sqrt(dot(r.data(), r.data(), n));
      if (rnorm <= tol * bnorm || it >= max_it) break;
    }
    ic0_apply(L, perm, r.data(), z.data());
    const double rho_new = dot(r.data(), z.data(), n);
    const double beta = rho_new / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
  return it;
}

// CG with the Jacobi preconditioner z = r / diag(Mat) (Sec. 6.2: "the
// preconditioner is simply the diagonal"), same iteration as pcg() above.
int pcg_jacobi(const Csr& Mat, double tol, int max_it, const double* b, double* x, int forced_its) {
  const int64_t n = Mat.nrows;
  std::vector<double> d(n);
  for (int64_t i = 0; i < n; ++i) d[i] = Mat.val[Mat.find(i, (int32_t)i)];
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  const double bnorm = std::sqrt(dot(b, b, n));
  if (bnorm == 0.0 || forced_its == 0) return 0;
  std::vector<double> r(b, b + n), z(n), p(n), q(n);
  for (int64_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
  p = z;
  double rho = dot(r.data(), z.data(), n);
  int it = 0;
  for (;;) {
    spmv(Mat, p.data(), q.data());
    ++it;
    const double alpha = rho / dot(p.data(), q.data(), n);
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    if (forced_its > 0) {
      if (it >= forced_its) break;
    } else {
      const double rnorm = std::sqrt(dot(r.data(), r.data(), n));
      if (rnorm <= tol * bnorm || it >= max_it) break;
    }
    for (int64_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
    const double rho_new = dot(r.data(), z.data(), n);
    const double beta = rho_new / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
  return it;
}

// Inner CG on A_h (Sec. 5.1 "PCG(A)").
int pcg_ic0(const Problem& P, Precond& M, const double* b, double* x, int forced_its) {
  return pcg(P.A, *M.L, *M.perm, M.inner_tol, M.max_inner, b, x, forced_its);
}

// CG on the pressure mass matrix Q (Sec. 6.4, "PCG(Q)").
int pcg_ic0_q(const Problem& P, Precond& M, const double* b, double* x, int forced_its) {
  if (!M.LQ || !M.permQ) throw std::runtime_error("pressure CG needs the IC(0) factor of Q");
  return pcg(P.Q, *M.LQ, *M.permQ, M.inner_tol, M.max_inner, b, x, forced_its);
}

// z = M^{-1} r with M = diag(M_A, M_Q): M_Q = Diag(Q_nu), or the CG solve
// with Q_nu = Q / (2 nu), i.e. z_p = 2 nu y with Q y ~= r_p (the relative
// stopping test is unchanged by the scaling).
void precond_apply(const Problem& P, Precond& M, const double* r, double* z) {
  int forced = -1;
  const int64_t app = (int64_t)M.counts.size();
  if (M.forced) {
    if (app >= M.nforced) throw std::runtime_error("replay: ran out of forced counts");
    forced = M.forced[app];
  }
  int its = 0;
  if (M.velocity == VELOCITY_DIAG) {
    for (int64_t i = 0; i < P.n_u; ++i) z[i] = r[i] / P.A.val[P.A.find(i, (int32_t)i)];
  } else if (M.velocity == VELOCITY_JACOBI_PCG) {
    its = pcg_jacobi(P.A, M.inner_tol, M.max_inner, r, z, forced);
  } else {
    its = pcg_ic0(P, M, r, z, forced);
  }
  M.counts.push_back(its);
  if (M.pressure == PRESSURE_PCG || M.pressure == PRESSURE_JACOBI_PCG) {
    int forced_q = -1;
    if (M.forced_q) {
      if (app >= M.nforced_q) throw std::runtime_error("replay: ran out of forced pressure counts");
      forced_q = M.forced_q[app];
    }
    std::vector<double> y(P.n_p);
    M.qcounts.push_back(M.pressure == PRESSURE_PCG
                            ? pcg_ic0_q(P, M, r + P.n_u, y.data(), forced_q)
                            : pcg_jacobi(P.Q, M.inner_tol, M.max_inner, r + P.n_u, y.data(), forced_q));
    for (int64_t k = 0; k < P.n_p; ++k) z[P.n_u + k] = 2.0 * P.nu * y[k];
    return;
  }
  for (int64_t k = 0; k < P.n_p; ++k) {
    double qkk = P.Q.val[P.Q.find(k, (int32_t)k)];
    z[P.n_u + k] = 2.0 * P.nu * r[P.n_u + k] / qkk;
  }
}

// Preconditioned MINRES (Sec. 5, eq. opt_condition with the M^{-1}-norm of
// eq. linsys_precond): Lanczos three-term recurrence in the M^{-1} inner
// product, QR of the tridiagonal matrix by Givens rotations, update of x by
// the search directions w.  eta tracks ||r_j||_{M^{-1}}.  The solve stops when
// ||b - K x_j||_2 / ||b||_2 <= tol (STOP_RESIDUAL, the residual recomputed
// from x_j after every step) or when |eta| / gamma_1 <= tol (STOP_ESTIMATE).
// Zero initial guess.
void minres(const Problem& P, Precond& M, const double* b, double* x, double tol,
            int max_outer, MinresInfo& info, int stop_rule) {
  const int64_t n = P.n_u + P.n_p;
  std::vector<double> v_prev(n, 0.0), v(b, b + n), v_next(n), z(n), z_next(n), q(n);
  std::vector<double> w_prev(n, 0.0), w(n, 0.0), w_next(n);
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  info = MinresInfo();
  precond_apply(P, M, v.data(), z.data());
  double gamma = std::sqrt(dot(z.data(), v.data(), n));
  const double bnorm = std::sqrt(dot(b, b, n));
  if (!(gamma > 0.0)) {
    info.status = (bnorm == 0.0) ? 0 : 2;
    return;
  }
  double gamma_prev = 1.0;
  const double gamma1 = gamma;
  info.gamma.push_back(gamma1);
  double eta = gamma;
  double s_prev = 0.0, s = 0.0, c_prev = 1.0, c = 1.0;
  info.status = 1;
  for (int j = 1; j <= max_outer; ++j) {
    for (int64_t i = 0; i < n; ++i) z[i] /= gamma;
    stokes_apply(P, z.data(), q.data());
    const double delta = dot(q.data(), z.data(), n);
    for (int64_t i = 0; i < n; ++i)
      v_next[i] = q[i] - (delta / gamma) * v[i] - (gamma / gamma_prev) * v_prev[i];
    precond_apply(P, M, v_next.data(), z_next.data());
    const double gg = dot(z_next.data(), v_next.data(), n);
    if (gg < 0.0) {  // preconditioner not positive: cannot continue
      info.status = 2;
      info.outer = j;
      break;
    }
    const double gamma_next = std::sqrt(gg);
    info.delta.push_back(delta);
    info.gamma.push_back(gamma_next);
    const double a0 = c * delta - c_prev * s * gamma;
    const double a1 = std::sqrt(a0 * a0 + gamma_next * gamma_next);
    const double a2 = s * delta + c_prev * c * gamma;
    const double a3 = s_prev * gamma;
    const double c_next = a0 / a1;
    const double s_next = gamma_next / a1;
    for (int64_t i = 0; i < n; ++i) {
      w_next[i] = (z[i] - a3 * w_prev[i] - a2 * w[i]) / a1;
      x[i] += c_next * eta * w_next[i];
    }
    eta = -s_next * eta;
    // shift the recurrences
    v_prev.swap(v);
    v.swap(v_next);
    z.swap(z_next);
    w_prev.swap(w);
    w.swap(w_next);
    gamma_prev = gamma;
    gamma = gamma_next;
    c_prev = c;
    c = c_next;
    s_prev = s;
    s = s_next;
    info.outer = j;
    info.relres_est = std::fabs(eta) / gamma1;
    info.hist.push_back(info.relres_est);
    double rel = info.relres_est;
    if (stop_rule == STOP_RESIDUAL) {
      stokes_apply(P, x, q.data());
      double rr = 0.0;
      for (int64_t i = 0; i < n; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
      rel = std::sqrt(rr) / bnorm;
      info.hist2.push_back(rel);
    }
    if (rel <= tol) {
      info.status = 0;
      break;
    }
  }
  std::vector<double> r(n);
  stokes_apply(P, x, r.data());
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  info.relres_true = bnorm > 0 ? std::sqrt(dot(r.data(), r.data(), n)) / bnorm : 0.0;
}

// Zero-mean pressure (Sec. 6.4: the constraint is imposed after the solve by
// filtering): p <- p - (w^T p / w^T 1) 1 with w_k = integral of phi_k.
void pressure_filter(const Problem& P, double* pres) {
  double wp = 0.0, w1 = 0.0;
  for (int64_t k = 0; k < P.n_p; ++k) {
    wp += P.wmean[k] * pres[k];
    w1 += P.wmean[k];
  }
  const double m = wp / w1;
  for (int64_t k = 0; k < P.n_p; ++k) pres[k] -= m;
}

}  // namespace oracle
