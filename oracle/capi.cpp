// capi.cpp -- TEST INFRASTRUCTURE ONLY (see oracle.hpp).
// extern "C" entry points of the oracle, loaded through ctypes by the tests,
// the smoke check and the benchmark's CPU-baseline leg.
#include <cstring>
#include <exception>
#include <string>

#include "oracle.hpp"

using namespace oracle;

namespace {
struct Handle {
  Problem P;
  int ordering = 0;
  bool full = true;
  std::vector<int32_t> perm;
  Csr L;
  std::vector<int32_t> level, rlevel;
  bool factored = false;
  std::vector<int32_t> counts;
  std::vector<double> hist, hist2, delta, gamma;
  // pressure mass matrix: ordering, IC(0) factor and its levels
  std::vector<int32_t> permQ;
  Csr LQ;
  std::vector<int32_t> levelQ, rlevelQ;
  bool qfactored = false;
  std::vector<int32_t> qcounts;
};
thread_local std::string g_err;
}  // namespace

#define OR_TRY(...)                \
  try {                            \
    __VA_ARGS__                    \
  } catch (const std::exception& e) { \
    g_err = e.what();              \
    return -99;                    \
  }

extern "C" {

const char* or_last_error() { return g_err.c_str(); }

void* or_create(int dim, int N, int p, double nu, double cpen, int ordering, int qordering,
                const char* sel_u, const char* sel_p) {
  try {
    Handle* h = new Handle();
    h->ordering = ordering;
    std::vector<char> su, sp;
    const std::vector<char>*psu = nullptr, *psp = nullptr;
    Problem probe;
    if (sel_u || sel_p) {
      h->full = false;
      // sizes first, to size the selection masks
      Problem& P = h->P;
      P.dim = dim;
      P.N = N;
      P.p = p;
      int64_t nu_ = 0;
      for (int c = 0; c < dim; ++c) {
        int64_t m = 1;
        for (int k = 0; k < dim; ++k) m *= (k == c ? N + p - 2 : N + p - 1);
        nu_ += m;
      }
      int64_t np_ = 1;
      for (int k = 0; k < dim; ++k) np_ *= (N + p - 1);
      su.assign(nu_, 0);
      sp.assign(np_, 0);
      if (sel_u) std::memcpy(su.data(), sel_u, nu_);
      if (sel_p) std::memcpy(sp.data(), sel_p, np_);
      psu = &su;
      psp = &sp;
    }
    setup_problem(h->P, dim, N, p, nu, cpen, psu, psp);
    if (h->full) {
      make_ordering(h->P, ordering, h->perm);
      lower_pattern(h->P.A, h->perm, h->L);
      level_sets(h->L, h->level, h->rlevel);
      make_pressure_ordering(h->P, qordering, h->permQ);
      lower_pattern(h->P.Q, h->permQ, h->LQ);
      level_sets(h->LQ, h->levelQ, h->rlevelQ);
    }
    return h;
  } catch (const std::exception& e) {
    g_err = e.what();
    return nullptr;
  }
}

void or_destroy(void* hv) { delete static_cast<Handle*>(hv); }

int or_sizes(void* hv, int64_t* out) {
  Handle* h = static_cast<Handle*>(hv);
  out[0] = h->P.n_u;
  out[1] = h->P.n_p;
  out[2] = h->P.A.nnz();
  out[3] = h->P.B.nnz();
  out[4] = h->P.Q.nnz();
  out[5] = h->L.nnz();
  int32_t ml = -1, mr = -1;
  for (int32_t v : h->level) ml = v > ml ? v : ml;
  for (int32_t v : h->rlevel) mr = v > mr ? v : mr;
  out[6] = ml + 1;
  out[7] = mr + 1;
  out[8] = h->LQ.nnz();
  ml = mr = -1;
  for (int32_t v : h->levelQ) ml = v > ml ? v : ml;
  for (int32_t v : h->rlevelQ) mr = v > mr ? v : mr;
  out[9] = ml + 1;
  out[10] = mr + 1;
  return 0;
}

int or_csr(void* hv, int which, int64_t* ptr, int32_t* col, double* val) {
  Handle* h = static_cast<Handle*>(hv);
  const Csr* M = which == 0 ? &h->P.A : which == 1 ? &h->P.B : which == 2 ? &h->P.Q : which == 3 ? &h->L : &h->LQ;
  if (ptr) std::memcpy(ptr, M->ptr.data(), sizeof(int64_t) * (M->nrows + 1));
  if (col) std::memcpy(col, M->col.data(), sizeof(int32_t) * M->nnz());
  if (val) std::memcpy(val, M->val.data(), sizeof(double) * M->nnz());
  return 0;
}

int or_wmean(void* hv, double* w) {
  Handle* h = static_cast<Handle*>(hv);
  std::memcpy(w, h->P.wmean.data(), sizeof(double) * h->P.n_p);
  return 0;
}

int or_perm(void* hv, int32_t* perm, int32_t* level, int32_t* rlevel) {
  Handle* h = static_cast<Handle*>(hv);
  int64_t n = h->P.n_u;
  if (perm) std::memcpy(perm, h->perm.data(), sizeof(int32_t) * n);
  if (level) std::memcpy(level, h->level.data(), sizeof(int32_t) * n);
  if (rlevel) std::memcpy(rlevel, h->rlevel.data(), sizeof(int32_t) * n);
  return 0;
}

// Colour of every velocity DOF (natural numbering) under the multicolour
// rule, whatever ordering the problem uses.
int or_colours(void* hv, int64_t* out) {
  Handle* h = static_cast<Handle*>(hv);
  for (int64_t i = 0; i < h->P.n_u; ++i) out[i] = velocity_colour(h->P, i);
  return 0;
}

int or_perm_q(void* hv, int32_t* perm, int32_t* level, int32_t* rlevel) {
  Handle* h = static_cast<Handle*>(hv);
  int64_t n = h->P.n_p;
  if (perm) std::memcpy(perm, h->permQ.data(), sizeof(int32_t) * n);
  if (level) std::memcpy(level, h->levelQ.data(), sizeof(int32_t) * n);
  if (rlevel) std::memcpy(rlevel, h->rlevelQ.data(), sizeof(int32_t) * n);
  return 0;
}

// IC(0) of the reordered Q: -1 on success, the permuted breakdown row otherwise.
int64_t or_factor_q(void* hv) {
  Handle* h = static_cast<Handle*>(hv);
  try {
    int64_t r = ic0(h->P.Q, h->permQ, h->LQ);
    h->qfactored = (r < 0);
    return r;
  } catch (const std::exception& e) {
    g_err = e.what();
    return -99;
  }
}

// Returns -1 on success, the permuted breakdown row otherwise.
int64_t or_factor(void* hv) {
  Handle* h = static_cast<Handle*>(hv);
  try {
    int64_t r = ic0(h->P.A, h->perm, h->L);
    h->factored = (r < 0);
    return r;
  } catch (const std::exception& e) {
    g_err = e.what();
    return -99;
  }
}

int or_load_fourier(void* hv, int nmodes, const int* kappa, const double* amp, double* f) {
  Handle* h = static_cast<Handle*>(hv);
  OR_TRY(std::vector<double> v; load_fourier(h->P, nmodes, kappa, amp, v);
         std::memcpy(f, v.data(), sizeof(double) * v.size()); return 0;)
}

int or_load_manufactured(void* hv, double* f) {
  Handle* h = static_cast<Handle*>(hv);
  OR_TRY(std::vector<double> v; load_manufactured(h->P, v);
         std::memcpy(f, v.data(), sizeof(double) * v.size()); return 0;)
}

int or_load_cavity(void* hv, double* f) {
  Handle* h = static_cast<Handle*>(hv);
  OR_TRY(std::vector<double> v; load_cavity(h->P, v);
         std::memcpy(f, v.data(), sizeof(double) * v.size()); return 0;)
}

int or_manufactured_errors(void* hv, const double* u, const double* p, double* out) {
  Handle* h = static_cast<Handle*>(hv);
  OR_TRY(manufactured_errors(h->P, u, p, out); return 0;)
}

void or_manufactured_point(double nu, double x, double y, double* out) {
  manufactured_point(nu, x, y, out);
}

// info[0] outer its, [1] relres estimate, [2] true relres, [3] status.
// pressure: PRESSURE_DIAG or PRESSURE_PCG (needs or_factor_q); forced /
// forced_q replay the inner counts of the velocity / pressure CG.
int or_minres(void* hv, const double* b, double* x, double tol, double inner_tol, int max_outer,
              int max_inner, const int32_t* forced, int64_t nforced, int pressure,
              const int32_t* forced_q, int64_t nforced_q, int velocity, int stop_rule, double* info) {
  Handle* h = static_cast<Handle*>(hv);
  if ((velocity == VELOCITY_IC0_PCG && !h->factored) || (pressure == PRESSURE_PCG && !h->qfactored)) {
    g_err = "factor first";
    return -1;
  }
  OR_TRY(Precond M; M.P = &h->P; M.L = &h->L; M.perm = &h->perm; M.inner_tol = inner_tol;
         M.max_inner = max_inner; M.forced = forced; M.nforced = forced ? nforced : 0;
         M.pressure = pressure; M.velocity = velocity; M.LQ = &h->LQ; M.permQ = &h->permQ;
         M.forced_q = forced_q; M.nforced_q = forced_q ? nforced_q : 0;
         MinresInfo mi; minres(h->P, M, b, x, tol, max_outer, mi, stop_rule);
         pressure_filter(h->P, x + h->P.n_u); h->counts = M.counts; h->qcounts = M.qcounts;
         h->hist = mi.hist; h->hist2 = mi.hist2; h->delta = mi.delta; h->gamma = mi.gamma; info[0] = mi.outer; info[1] = mi.relres_est; info[2] = mi.relres_true;
         info[3] = mi.status; return 0;)
}

int64_t or_qcounts(void* hv, int32_t* out, int64_t cap) {
  Handle* h = static_cast<Handle*>(hv);
  int64_t n = (int64_t)h->qcounts.size();
  for (int64_t i = 0; i < n && i < cap; ++i) out[i] = h->qcounts[i];
  return n;
}

int64_t or_counts(void* hv, int32_t* out, int64_t cap) {
  Handle* h = static_cast<Handle*>(hv);
  int64_t n = (int64_t)h->counts.size();
  for (int64_t i = 0; i < n && i < cap; ++i) out[i] = h->counts[i];
  return n;
}

// which 0: |eta|/gamma_1 after each step; 1: ||b - K x_j|| / ||b|| (STOP_RESIDUAL);
// 2: Lanczos diagonal delta_j; 3: Lanczos gamma_1, gamma_2, ...
int64_t or_hist(void* hv, int which, double* out, int64_t cap) {
  Handle* h = static_cast<Handle*>(hv);
  const std::vector<double>& v = which == 0 ? h->hist : which == 1 ? h->hist2 : which == 2 ? h->delta : h->gamma;
  int64_t n = (int64_t)v.size();
  for (int64_t i = 0; i < n && i < cap; ++i) out[i] = v[i];
  return n;
}

int or_pcg(void* hv, const double* b, double* x, double inner_tol, int max_inner) {
  Handle* h = static_cast<Handle*>(hv);
  OR_TRY(Precond M; M.P = &h->P; M.L = &h->L; M.perm = &h->perm; M.inner_tol = inner_tol;
         M.max_inner = max_inner; return pcg_ic0(h->P, M, b, x, -1);)
}

int or_pcg_q(void* hv, const double* b, double* x, double inner_tol, int max_inner) {
  Handle* h = static_cast<Handle*>(hv);
  if (!h->qfactored) {
    g_err = "factor Q first";
    return -1;
  }
  OR_TRY(Precond M; M.P = &h->P; M.LQ = &h->LQ; M.permQ = &h->permQ; M.inner_tol = inner_tol;
         M.max_inner = max_inner; return pcg_ic0_q(h->P, M, b, x, -1);)
}

int or_precond(void* hv, const double* r, double* z, double inner_tol, int max_inner, int pressure) {
  Handle* h = static_cast<Handle*>(hv);
  OR_TRY(Precond M; M.P = &h->P; M.L = &h->L; M.perm = &h->perm; M.inner_tol = inner_tol;
         M.max_inner = max_inner; M.pressure = pressure; M.LQ = &h->LQ; M.permQ = &h->permQ;
         precond_apply(h->P, M, r, z); return M.counts[0];)
}

int or_stokes_apply(void* hv, const double* x, double* y) {
  Handle* h = static_cast<Handle*>(hv);
  stokes_apply(h->P, x, y);
  return 0;
}

int or_filter(void* hv, double* p) {
  Handle* h = static_cast<Handle*>(hv);
  pressure_filter(h->P, p);
  return 0;
}

// dL/dnu = -lambda_u^T A_0 u with A_0 = A_h / nu (A_h is linear in nu).
double or_dnu(void* hv, const double* lam, const double* u) {
  Handle* h = static_cast<Handle*>(hv);
  std::vector<double> Au(h->P.n_u);
  spmv(h->P.A, u, Au.data());
  double s = 0.0;
  for (int64_t i = 0; i < h->P.n_u; ++i) s += lam[i] * Au[i];
  return -s / h->P.nu;
}

int or_basis(int N, int q, int e, double x, double* val, double* der) {
  Knots K = open_uniform(N, q);
  eval_basis(K, e, x, val, der);
  return 0;
}

int or_gauss(int n, double* x, double* w) {
  OR_TRY(std::vector<double> gx, gw; gauss_legendre(n, gx, gw);
         std::memcpy(x, gx.data(), sizeof(double) * n);
         std::memcpy(w, gw.data(), sizeof(double) * n); return 0;)
}

}  // extern "C"
