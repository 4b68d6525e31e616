// assembly.cpp -- TEST INFRASTRUCTURE ONLY (see oracle.hpp).
// Divergence-conforming spaces (Sec. 3.2) and the discrete Stokes system
// with Nitsche's no-slip terms (Sec. 4), by plain element-loop Gauss
// quadrature on the identity map of the unit square / cube.
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "oracle.hpp"

namespace oracle {

int64_t Problem::vindex(int c, const int* a) const {
  int64_t idx = 0;
  for (int k = 0; k < dim; ++k) {
    int l = (k == c) ? a[k] - 1 : a[k];
    idx = idx * vlen(c, k) + l;
  }
  return voff[c] + idx;
}

void Problem::vdecode(int64_t i, int* c, int* a) const {
  int cc = 0;
  while (cc + 1 < dim && i >= voff[cc + 1]) ++cc;
  int64_t r = i - voff[cc];
  for (int k = dim - 1; k >= 0; --k) {
    int l = (int)(r % vlen(cc, k));
    r /= vlen(cc, k);
    a[k] = (k == cc) ? l + 1 : l;
  }
  *c = cc;
}

int64_t Problem::pindex(const int* a) const {
  int64_t idx = 0;
  for (int k = 0; k < dim; ++k) idx = idx * plen() + a[k];
  return idx;
}

void Problem::pdecode(int64_t k, int* a) const {
  for (int d = dim - 1; d >= 0; --d) {
    a[d] = (int)(k % plen());
    k /= plen();
  }
}

// ------------------------------------------------------------------------
// 1D tables: basis values/derivatives of both degrees at the Gauss points of
// every element.  tab[e][g][t] for function index e+t.
struct Table1D {
  int q = 0, ng = 0, N = 0;
  std::vector<double> x, w;  // physical points and weights per element (e*ng+g)
  std::vector<double> val, der;  // [(e*ng+g)*(q+1)+t]
  double v(int e, int g, int t) const { return val[((size_t)e * ng + g) * (q + 1) + t]; }
  double d(int e, int g, int t) const { return der[((size_t)e * ng + g) * (q + 1) + t]; }
};

static Table1D make_table(const Knots& K, int ng) {
  Table1D T;
  T.q = K.q;
  T.ng = ng;
  T.N = K.N;
  std::vector<double> gx, gw;
  gauss_legendre(ng, gx, gw);
  T.x.resize((size_t)K.N * ng);
  T.w.resize((size_t)K.N * ng);
  T.val.resize((size_t)K.N * ng * (K.q + 1));
  T.der.resize((size_t)K.N * ng * (K.q + 1));
  const double h = 1.0 / K.N;
  for (int e = 0; e < K.N; ++e) {
    for (int g = 0; g < ng; ++g) {
      double x = (e + 0.5 * (gx[g] + 1.0)) * h;
      T.x[(size_t)e * ng + g] = x;
      T.w[(size_t)e * ng + g] = 0.5 * gw[g] * h;
      eval_basis(K, e, x, &T.val[((size_t)e * ng + g) * (K.q + 1)],
                 &T.der[((size_t)e * ng + g) * (K.q + 1)]);
    }
  }
  return T;
}

// A velocity or pressure basis function living on one element.
struct LocalFun {
  int64_t gidx;
  int comp;   // velocity component (-1 for pressure)
  int off[3]; // 1D offsets: function index = e_k + off[k]
};

static void element_vfuns(const Problem& P, const int* e, std::vector<LocalFun>& out) {
  out.clear();
  for (int c = 0; c < P.dim; ++c) {
    int cnt[3] = {1, 1, 1};
    for (int k = 0; k < P.dim; ++k) cnt[k] = P.deg(c, k) + 1;
    for (int o0 = 0; o0 < cnt[0]; ++o0)
      for (int o1 = 0; o1 < cnt[1]; ++o1)
        for (int o2 = 0; o2 < (P.dim == 3 ? cnt[2] : 1); ++o2) {
          int off[3] = {o0, o1, o2};
          int a[3];
          for (int k = 0; k < P.dim; ++k) a[k] = e[k] + off[k];
          // removed normal-boundary functions of V_{0,h} (Sec. 3.2)
          if (a[c] == 0 || a[c] == P.N + P.p - 1) continue;
          LocalFun f;
          f.gidx = P.vindex(c, a);
          f.comp = c;
          for (int k = 0; k < 3; ++k) f.off[k] = off[k];
          out.push_back(f);
        }
  }
}

static void element_pfuns(const Problem& P, const int* e, std::vector<LocalFun>& out) {
  out.clear();
  const int cnt = P.p;  // degree p-1 -> p functions per direction
  for (int o0 = 0; o0 < cnt; ++o0)
    for (int o1 = 0; o1 < cnt; ++o1)
      for (int o2 = 0; o2 < (P.dim == 3 ? cnt : 1); ++o2) {
        int off[3] = {o0, o1, o2};
        int a[3];
        for (int k = 0; k < P.dim; ++k) a[k] = e[k] + off[k];
        LocalFun f;
        f.gidx = P.pindex(a);
        f.comp = -1;
        for (int k = 0; k < 3; ++k) f.off[k] = off[k];
        out.push_back(f);
      }
}

// Elements in the support of a degree-q function with 1D index a.
static void support_range(int a, int q, int N, int* lo, int* hi) {
  *lo = std::max(0, a - q);
  *hi = std::min(N - 1, a);
}

template <class F>
static void for_each_element_in_box(int dim, const int* lo, const int* hi, F fn) {
  int e[3] = {0, 0, 0};
  for (e[0] = lo[0]; e[0] <= hi[0]; ++e[0])
    for (e[1] = lo[1]; e[1] <= hi[1]; ++e[1])
      for (e[2] = (dim == 3 ? lo[2] : 0); e[2] <= (dim == 3 ? hi[2] : 0); ++e[2]) fn(e);
}

// Pattern of a matrix whose rows are the functions `rowfun` and columns the
// functions sharing an element with them (support overlap).
static void build_pattern(const Problem& P, bool rows_velocity, bool cols_velocity,
                          const std::vector<char>* sel, Csr& M) {
  const int64_t nr = rows_velocity ? P.n_u : P.n_p;
  M.nrows = nr;
  M.ncols = cols_velocity ? P.n_u : P.n_p;
  M.ptr.assign(nr + 1, 0);
  std::vector<std::vector<int32_t>> rows(nr);
  std::vector<LocalFun> funs;
  for (int64_t i = 0; i < nr; ++i) {
    if (sel && !(*sel)[i]) continue;
    int a[3] = {0, 0, 0}, c = -1;
    if (rows_velocity) P.vdecode(i, &c, a);
    else P.pdecode(i, a);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < P.dim; ++k) {
      int q = rows_velocity ? P.deg(c, k) : P.p - 1;
      support_range(a[k], q, P.N, &lo[k], &hi[k]);
    }
    std::vector<int32_t>& r = rows[i];
    for_each_element_in_box(P.dim, lo, hi, [&](const int* e) {
      if (cols_velocity) element_vfuns(P, e, funs);
      else element_pfuns(P, e, funs);
      for (const LocalFun& f : funs) r.push_back((int32_t)f.gidx);
    });
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
  }
  for (int64_t i = 0; i < nr; ++i) M.ptr[i + 1] = M.ptr[i] + (int64_t)rows[i].size();
  M.col.resize(M.ptr[nr]);
  for (int64_t i = 0; i < nr; ++i)
    std::copy(rows[i].begin(), rows[i].end(), M.col.begin() + M.ptr[i]);
  M.val.assign(M.ptr[nr], 0.0);
}

// Value and gradient of a velocity function at tensor quadrature point g[]
// of element e, from the 1D tables (identity geometric map).
struct PointEval {
  double val;
  double grad[3];
};

static PointEval eval_vfun(const Problem& P, const Table1D* T /*[0]=deg p,[1]=deg p-1*/,
                           const LocalFun& f, const int* e, const int* g) {
  PointEval r;
  double v1[3], d1[3];
  for (int k = 0; k < P.dim; ++k) {
    const Table1D& Tk = T[P.deg(f.comp, k) == P.p ? 0 : 1];
    v1[k] = Tk.v(e[k], g[k], f.off[k]);
    d1[k] = Tk.d(e[k], g[k], f.off[k]);
  }
  r.val = 1.0;
  for (int k = 0; k < P.dim; ++k) r.val *= v1[k];
  for (int m = 0; m < P.dim; ++m) {
    double gm = d1[m];
    for (int k = 0; k < P.dim; ++k)
      if (k != m) gm *= v1[k];
    r.grad[m] = gm;
  }
  return r;
}

static double eval_pfun(const Problem& P, const Table1D& Tq, const LocalFun& f, const int* e,
                        const int* g) {
  double v = 1.0;
  for (int k = 0; k < P.dim; ++k) v *= Tq.v(e[k], g[k], f.off[k]);
  return v;
}

// Symmetric gradient (Sec. 3.1, a(w,v) = (2 nu grad^s w, grad^s v)) of the
// vector field Phi = phi e_c: S = (grad Phi + grad Phi^T)/2.
static void sym_grad(int dim, int comp, const double* grad, double S[3][3]) {
  double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // G[a][b] = d Phi_a / d x_b
  for (int b = 0; b < dim; ++b) G[comp][b] = grad[b];
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) S[a][b] = 0.5 * (G[a][b] + G[b][a]);
}

void setup_problem(Problem& P, int dim, int N, int p, double nu, double cpen,
                   const std::vector<char>* rows_u, const std::vector<char>* rows_p) {
  if (dim != 2 && dim != 3) throw std::runtime_error("dim must be 2 or 3");
  if (p < 2 || N < 1) throw std::runtime_error("need p >= 2, N >= 1");
  P.dim = dim;
  P.N = N;
  P.p = p;
  P.nu = nu;
  P.cpen = cpen;
  P.Kp = open_uniform(N, p);
  P.Kq = open_uniform(N, p - 1);
  int64_t off = 0;
  for (int c = 0; c < 3; ++c) {
    P.voff[c] = off;
    if (c >= dim) {
      P.nvc[c] = 0;
      continue;
    }
    int64_t n = 1;
    for (int k = 0; k < dim; ++k) n *= P.vlen(c, k);
    P.nvc[c] = n;
    off += n;
  }
  P.n_u = off;
  P.n_p = 1;
  for (int k = 0; k < dim; ++k) P.n_p *= P.plen();

  build_pattern(P, true, true, rows_u, P.A);
  build_pattern(P, false, true, rows_p, P.B);
  build_pattern(P, false, false, rows_p, P.Q);

  // ---- element loop (Sec. 4): A_h = a - eta_h, B_{kj} = -(div Phi_j, phi_k),
  // Q_{kl} = (phi_l, phi_k).  (p+1)-point Gauss rule per direction: exact for
  // the polynomial integrands of degree <= 2p per direction.
  const int ng = p + 1;
  Table1D T[2] = {make_table(P.Kp, ng), make_table(P.Kq, ng)};
  const double hF = 1.0 / N;  // h_F: element width normal to the boundary face
  std::vector<LocalFun> vf, pf;
  std::vector<double> Ae, Be, Qe;
  std::vector<PointEval> pe;
  std::vector<double> pv;
  int lo[3] = {0, 0, 0}, hi[3] = {N - 1, N - 1, dim == 3 ? N - 1 : 0};
  for_each_element_in_box(dim, lo, hi, [&](const int* e) {
    element_vfuns(P, e, vf);
    element_pfuns(P, e, pf);
    bool any_u = !rows_u, any_p = !rows_p;
    if (rows_u)
      for (auto& f : vf) any_u = any_u || (*rows_u)[f.gidx];
    if (rows_p)
      for (auto& f : pf) any_p = any_p || (*rows_p)[f.gidx];
    if (!any_u && !any_p) return;
    const size_t nv = vf.size(), np = pf.size();
    Ae.assign(nv * nv, 0.0);
    Be.assign(np * nv, 0.0);
    Qe.assign(np * np, 0.0);
    pe.resize(nv);
    pv.resize(np);
    // interior terms
    int g[3] = {0, 0, 0};
    for (g[0] = 0; g[0] < ng; ++g[0])
      for (g[1] = 0; g[1] < ng; ++g[1])
        for (g[2] = 0; g[2] < (dim == 3 ? ng : 1); ++g[2]) {
          double w = 1.0;
          for (int k = 0; k < dim; ++k) w *= T[0].w[(size_t)e[k] * ng + g[k]];
          for (size_t a = 0; a < nv; ++a) pe[a] = eval_vfun(P, T, vf[a], e, g);
          for (size_t a = 0; a < np; ++a) pv[a] = eval_pfun(P, T[1], pf[a], e, g);
          for (size_t i = 0; i < nv; ++i) {
            double Si[3][3];
            sym_grad(dim, vf[i].comp, pe[i].grad, Si);
            for (size_t j = 0; j < nv; ++j) {
              double Sj[3][3];
              sym_grad(dim, vf[j].comp, pe[j].grad, Sj);
              double contr = 0.0;
              for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) contr += Si[a][b] * Sj[a][b];
              Ae[i * nv + j] += w * 2.0 * nu * contr;
            }
          }
          for (size_t k = 0; k < np; ++k)
            for (size_t j = 0; j < nv; ++j) {
              double divj = pe[j].grad[vf[j].comp];
              Be[k * nv + j] += -w * pv[k] * divj;
            }
          for (size_t k = 0; k < np; ++k)
            for (size_t l = 0; l < np; ++l) Qe[k * np + l] += w * pv[k] * pv[l];
        }
    // Nitsche boundary terms eta_h (Sec. 4, eq. nitsche_lhs) on the faces of
    // this element that lie on the boundary; g = 0 (no slip everywhere).
    for (int k = 0; k < dim; ++k) {
      for (int side = 0; side < 2; ++side) {
        if (side == 0 && e[k] != 0) continue;
        if (side == 1 && e[k] != N - 1) continue;
        const double xk = side == 0 ? 0.0 : 1.0;
        double nrm[3] = {0, 0, 0};
        nrm[k] = side == 0 ? -1.0 : 1.0;
        // 1D values in direction k at the face, both degrees
        double fv[2][16], fd[2][16];
        eval_basis(P.Kp, e[k], xk, fv[0], fd[0]);
        eval_basis(P.Kq, e[k], xk, fv[1], fd[1]);
        int gf[3] = {0, 0, 0};
        for (gf[0] = 0; gf[0] < (k == 0 ? 1 : ng); ++gf[0])
          for (gf[1] = 0; gf[1] < (k == 1 ? 1 : ng); ++gf[1])
            for (gf[2] = 0; gf[2] < ((dim == 3 && k != 2) ? ng : 1); ++gf[2]) {
              double w = 1.0;
              for (int m = 0; m < dim; ++m)
                if (m != k) w *= T[0].w[(size_t)e[m] * ng + gf[m]];
              // evaluate velocity functions on the face point
              for (size_t a = 0; a < nv; ++a) {
                const LocalFun& f = vf[a];
                double v1[3], d1[3];
                for (int m = 0; m < dim; ++m) {
                  int sel = P.deg(f.comp, m) == p ? 0 : 1;
                  if (m == k) {
                    v1[m] = fv[sel][f.off[m]];
                    d1[m] = fd[sel][f.off[m]];
                  } else {
                    v1[m] = T[sel].v(e[m], gf[m], f.off[m]);
                    d1[m] = T[sel].d(e[m], gf[m], f.off[m]);
                  }
                }
                PointEval r;
                r.val = 1.0;
                for (int m = 0; m < dim; ++m) r.val *= v1[m];
                for (int m = 0; m < dim; ++m) {
                  double gm = d1[m];
                  for (int mm = 0; mm < dim; ++mm)
                    if (mm != m) gm *= v1[mm];
                  r.grad[m] = gm;
                }
                pe[a] = r;
              }
              for (size_t i = 0; i < nv; ++i) {
                double Si[3][3];
                sym_grad(dim, vf[i].comp, pe[i].grad, Si);
                double ti[3] = {0, 0, 0};  // (grad^s Phi_i) n
                for (int a = 0; a < dim; ++a)
                  for (int b = 0; b < dim; ++b) ti[a] += Si[a][b] * nrm[b];
                for (size_t j = 0; j < nv; ++j) {
                  double Sj[3][3];
                  sym_grad(dim, vf[j].comp, pe[j].grad, Sj);
                  double tj[3] = {0, 0, 0};
                  for (int a = 0; a < dim; ++a)
                    for (int b = 0; b < dim; ++b) tj[a] += Sj[a][b] * nrm[b];
                  double Phi_i[3] = {0, 0, 0}, Phi_j[3] = {0, 0, 0};
                  Phi_i[vf[i].comp] = pe[i].val;
                  Phi_j[vf[j].comp] = pe[j].val;
                  double ti_Pj = 0, tj_Pi = 0, Pi_Pj = 0;
                  for (int a = 0; a < dim; ++a) {
                    ti_Pj += ti[a] * Phi_j[a];
                    tj_Pi += tj[a] * Phi_i[a];
                    Pi_Pj += Phi_i[a] * Phi_j[a];
                  }
                  double eta = 2.0 * nu * (ti_Pj + tj_Pi - (cpen / hF) * Pi_Pj);
                  Ae[i * nv + j] -= w * eta;
                }
              }
            }
      }
    }
    // scatter into the global CSR (rows kept only if selected)
    for (size_t i = 0; i < nv; ++i) {
      int64_t gi = vf[i].gidx;
      if (rows_u && !(*rows_u)[gi]) continue;
      for (size_t j = 0; j < nv; ++j) {
        int64_t pos = P.A.find(gi, (int32_t)vf[j].gidx);
        if (pos < 0) throw std::runtime_error("A pattern miss");
        P.A.val[pos] += Ae[i * nv + j];
      }
    }
    for (size_t k = 0; k < np; ++k) {
      int64_t gk = pf[k].gidx;
      if (rows_p && !(*rows_p)[gk]) continue;
      for (size_t j = 0; j < nv; ++j) {
        int64_t pos = P.B.find(gk, (int32_t)vf[j].gidx);
        if (pos < 0) throw std::runtime_error("B pattern miss");
        P.B.val[pos] += Be[k * nv + j];
      }
      for (size_t l = 0; l < np; ++l) {
        int64_t pos = P.Q.find(gk, (int32_t)pf[l].gidx);
        if (pos < 0) throw std::runtime_error("Q pattern miss");
        P.Q.val[pos] += Qe[k * np + l];
      }
    }
  });

  // w_k = integral of pressure function k (zero-mean filter, Sec. 6.4).
  P.wmean.assign(P.n_p, 0.0);
  for_each_element_in_box(dim, lo, hi, [&](const int* e) {
    element_pfuns(P, e, pf);
    int g[3] = {0, 0, 0};
    for (g[0] = 0; g[0] < ng; ++g[0])
      for (g[1] = 0; g[1] < ng; ++g[1])
        for (g[2] = 0; g[2] < (dim == 3 ? ng : 1); ++g[2]) {
          double w = 1.0;
          for (int k = 0; k < dim; ++k) w *= T[1].w[(size_t)e[k] * ng + g[k]];
          for (const LocalFun& f : pf) P.wmean[f.gidx] += w * eval_pfun(P, T[1], f, e, g);
        }
  });
}

// ------------------------------------------------------------------------
// Loads.  Quadrature with p+3 points per direction (the forcing is not a
// polynomial; the extra points only move results at discretisation level).
template <class Fn>
static void load_generic(const Problem& P, Fn forcing, std::vector<double>& f) {
  const int ng = P.p + 3;
  Table1D T[2] = {make_table(P.Kp, ng), make_table(P.Kq, ng)};
  f.assign(P.n_u, 0.0);
  std::vector<LocalFun> vf;
  int lo[3] = {0, 0, 0}, hi[3] = {P.N - 1, P.N - 1, P.dim == 3 ? P.N - 1 : 0};
  for_each_element_in_box(P.dim, lo, hi, [&](const int* e) {
    element_vfuns(P, e, vf);
    int g[3] = {0, 0, 0};
    for (g[0] = 0; g[0] < ng; ++g[0])
      for (g[1] = 0; g[1] < ng; ++g[1])
        for (g[2] = 0; g[2] < (P.dim == 3 ? ng : 1); ++g[2]) {
          double w = 1.0, x[3] = {0, 0, 0};
          for (int k = 0; k < P.dim; ++k) {
            w *= T[0].w[(size_t)e[k] * ng + g[k]];
            x[k] = T[0].x[(size_t)e[k] * ng + g[k]];
          }
          double fx[3] = {0, 0, 0};
          forcing(x, fx);
          for (const LocalFun& fn : vf) {
            PointEval r = eval_vfun(P, T, fn, e, g);
            f[fn.gidx] += w * fx[fn.comp] * r.val;
          }
        }
  });
}

void load_fourier(const Problem& P, int nmodes, const int* kappa, const double* amp,
                  std::vector<double>& f) {
  const double pi = 3.14159265358979323846;
  const int dim = P.dim;
  load_generic(
      P,
      [&](const double* x, double* fx) {
        for (int d = 0; d < dim; ++d) fx[d] = 0.0;
        for (int m = 0; m < nmodes; ++m) {
          double prod = 1.0;
          for (int k = 0; k < dim; ++k) prod *= std::sin(pi * kappa[m * dim + k] * x[k]);
          for (int d = 0; d < dim; ++d) fx[d] += amp[m * dim + d] * prod;
        }
      },
      f);
}

// Sec. 6.2 manufactured solution, with the sign of u_2 read so that div u = 0:
// u = (psi_y, -psi_x), psi = e^x g(x) h(y), g = x^2 (x-1)^2, h = (y^2-y)^2.
// The printed u_1 equals psi_y; the printed u_2 equals +psi_x, which is not
// divergence free, so it is read as -psi_x.  The pressure is as printed, and
// f = -div(2 nu grad^s u) + grad p = -nu lap u + grad p (eq. manufactured_force).
struct Manu {
  double u[2], du[2][2], p, f[2];
};
static Manu manu_eval(double nu, double x, double y) {
  const double ex = std::exp(x);
  // g and derivatives
  const double g = x * x * (x - 1) * (x - 1);
  const double g1 = 4 * x * x * x - 6 * x * x + 2 * x;
  const double g2 = 12 * x * x - 12 * x + 2;
  const double g3 = 24 * x - 12;
  const double h = y * y * (y - 1) * (y - 1);
  const double h1 = 4 * y * y * y - 6 * y * y + 2 * y;
  const double h2 = 12 * y * y - 12 * y + 2;
  const double h3 = 24 * y - 12;
  // G = e^x g and its derivatives
  const double G0 = ex * g;
  const double G1 = ex * (g + g1);
  const double G2 = ex * (g + 2 * g1 + g2);
  const double G3 = ex * (g + 3 * g1 + 3 * g2 + g3);
  Manu m;
  m.u[0] = G0 * h1;    // psi_y
  m.u[1] = -G1 * h;    // -psi_x
  m.du[0][0] = G1 * h1;
  m.du[0][1] = G0 * h2;
  m.du[1][0] = -G2 * h;
  m.du[1][1] = -G1 * h1;
  // lap psi = G'' h + G h'';  lap u = (d_y lap psi, -d_x lap psi)
  const double dy_lap = G2 * h1 + G0 * h3;
  const double dx_lap = G3 * h + G1 * h2;
  // pressure as printed: p = -424 + 156 e + s (-456 + e^x Pp(x,s)), s = y^2 - y
  const double s = y * y - y, sy = 2 * y - 1;
  const double Pp = 456 + x * x * (228 - 5 * s) + 2 * x * (-228 + s) + 2 * x * x * x * (-36 + s) +
                    x * x * x * x * (12 + s);
  const double Pp_x = 2 * x * (228 - 5 * s) + 2 * (-228 + s) + 6 * x * x * (-36 + s) +
                      4 * x * x * x * (12 + s);
  const double Pp_s = -5 * x * x + 2 * x + 2 * x * x * x + x * x * x * x;
  const double e1 = std::exp(1.0);
  m.p = -424 + 156 * e1 + s * (-456 + ex * Pp);
  const double px = s * ex * (Pp + Pp_x);
  const double py = sy * (-456 + ex * Pp) + s * ex * Pp_s * sy;
  m.f[0] = -nu * dy_lap + px;
  m.f[1] = nu * dx_lap + py;
  return m;
}

// Lid-driven cavity load (Sec. 6.4): no body force, and the Nitsche
// right-hand side of eq. nitsche_rhs,
//   l_h(v) = sum_F int_F 2 nu ( -((grad^s v) n) . g + (C_pen / h_F) g . v ) dS,
// with the lid velocity g = e_1 on the face x_dim = 1 and g = 0 on the other
// faces.  Gauss quadrature with p+1 points per direction on the lid faces.
void load_cavity(const Problem& P, std::vector<double>& f) {
  f.assign(P.n_u, 0.0);
  const int dim = P.dim, N = P.N, p = P.p, ng = p + 1;
  const Table1D T[2] = {make_table(P.Kp, ng), make_table(P.Kq, ng)};
  const double hF = 1.0 / N;
  const int k = dim - 1;  // lid normal direction
  double nrm[3] = {0, 0, 0}, gl[3] = {1.0, 0, 0};
  nrm[k] = 1.0;
  double fv[2][16], fd[2][16];
  eval_basis(P.Kp, N - 1, 1.0, fv[0], fd[0]);
  eval_basis(P.Kq, N - 1, 1.0, fv[1], fd[1]);
  std::vector<LocalFun> vf;
  int64_t nface = 1;  // elements of the lid face
  for (int m = 0; m < dim; ++m)
    if (m != k) nface *= N;
  for (int64_t fe = 0; fe < nface; ++fe) {
    int e[3] = {0, 0, 0};
    int64_t rest = fe;
    for (int m = 0; m < dim; ++m) {
      if (m == k) {
        e[m] = N - 1;
      } else {
        e[m] = (int)(rest % N);
        rest /= N;
      }
    }
    element_vfuns(P, e, vf);
    int gq[3] = {0, 0, 0};
    for (gq[0] = 0; gq[0] < (k == 0 ? 1 : ng); ++gq[0])
      for (gq[1] = 0; gq[1] < (k == 1 ? 1 : ng); ++gq[1])
        for (gq[2] = 0; gq[2] < ((dim == 3 && k != 2) ? ng : 1); ++gq[2]) {
          double w = 1.0;
          for (int m = 0; m < dim; ++m)
            if (m != k) w *= T[0].w[(size_t)e[m] * ng + gq[m]];
          for (const LocalFun& fn : vf) {
            double v1[3], d1[3];
            for (int m = 0; m < dim; ++m) {
              const int sel = P.deg(fn.comp, m) == p ? 0 : 1;
              v1[m] = (m == k) ? fv[sel][fn.off[m]] : T[sel].v(e[m], gq[m], fn.off[m]);
              d1[m] = (m == k) ? fd[sel][fn.off[m]] : T[sel].d(e[m], gq[m], fn.off[m]);
            }
            double val = 1.0, grad[3] = {0, 0, 0};
            for (int m = 0; m < dim; ++m) val *= v1[m];
            for (int m = 0; m < dim; ++m) {
              grad[m] = d1[m];
              for (int mm = 0; mm < dim; ++mm)
                if (mm != m) grad[m] *= v1[mm];
            }
            double S[3][3];
            sym_grad(dim, fn.comp, grad, S);
            double tg = 0.0;  // ((grad^s Phi) n) . g
            for (int r = 0; r < dim; ++r)
              for (int c = 0; c < dim; ++c) tg += gl[r] * S[r][c] * nrm[c];
            const double phig = val * gl[fn.comp];
            f[fn.gidx] += w * 2.0 * P.nu * (-tg + (P.cpen / hF) * phig);
          }
        }
  }
}

void manufactured_point(double nu, double x, double y, double out[5]) {
  Manu m = manu_eval(nu, x, y);
  out[0] = m.u[0];
  out[1] = m.u[1];
  out[2] = m.p;
  out[3] = m.f[0];
  out[4] = m.f[1];
}

void load_manufactured(const Problem& P, std::vector<double>& f) {
  if (P.dim != 2) throw std::runtime_error("manufactured solution is 2D");
  const double nu = P.nu;
  load_generic(
      P,
      [&](const double* x, double* fx) {
        Manu m = manu_eval(nu, x[0], x[1]);
        fx[0] = m.f[0];
        fx[1] = m.f[1];
      },
      f);
}

void manufactured_errors(const Problem& P, const double* u, const double* pres, double out[3]) {
  if (P.dim != 2) throw std::runtime_error("manufactured solution is 2D");
  const int ng = P.p + 3;
  Table1D T[2] = {make_table(P.Kp, ng), make_table(P.Kq, ng)};
  std::vector<LocalFun> vf, pf;
  double eH1 = 0, eL2 = 0, ep = 0;
  int lo[3] = {0, 0, 0}, hi[3] = {P.N - 1, P.N - 1, 0};
  for_each_element_in_box(2, lo, hi, [&](const int* e) {
    element_vfuns(P, e, vf);
    element_pfuns(P, e, pf);
    int g[3] = {0, 0, 0};
    for (g[0] = 0; g[0] < ng; ++g[0])
      for (g[1] = 0; g[1] < ng; ++g[1]) {
        double w = T[0].w[(size_t)e[0] * ng + g[0]] * T[0].w[(size_t)e[1] * ng + g[1]];
        double x = T[0].x[(size_t)e[0] * ng + g[0]], y = T[0].x[(size_t)e[1] * ng + g[1]];
        double uh[2] = {0, 0}, duh[2][2] = {{0, 0}, {0, 0}}, ph = 0;
        for (const LocalFun& fn : vf) {
          PointEval r = eval_vfun(P, T, fn, e, g);
          uh[fn.comp] += u[fn.gidx] * r.val;
          for (int b = 0; b < 2; ++b) duh[fn.comp][b] += u[fn.gidx] * r.grad[b];
        }
        for (const LocalFun& fn : pf) ph += pres[fn.gidx] * eval_pfun(P, T[1], fn, e, g);
        Manu m = manu_eval(P.nu, x, y);
        for (int a = 0; a < 2; ++a) {
          eL2 += w * (m.u[a] - uh[a]) * (m.u[a] - uh[a]);
          for (int b = 0; b < 2; ++b) eH1 += w * (m.du[a][b] - duh[a][b]) * (m.du[a][b] - duh[a][b]);
        }
        ep += w * (m.p - ph) * (m.p - ph);
      }
  });
  out[0] = std::sqrt(eH1);
  out[1] = std::sqrt(eL2);
  out[2] = std::sqrt(ep);
}

}  // namespace oracle
