// assemble.cu -- device assembly of A_h, B, Diag(Q), w and load vectors.
//
// On the identity map of the unit square/cube every integrand of Sec. 4 is a
// product of 1D factors (tensor-product B-splines, constant nu), so each
// entry of A_h, B and Q is a short sum of products of 1D integrals
//   I(q_i, o_i, a; q_j, o_j, b) = int_0^1 D^{o_i} B^{q_i}_a D^{o_j} B^{q_j}_b dx
// (and of end-point values for the Nitsche face terms).  The 1D integrals are
// computed once by Gauss quadrature with p+1 points per element (exact for
// these polynomial integrands); each nonzero is then formed independently,
// which is the GPU-friendly restatement of the element loop.
#include <cmath>
#include <vector>

#include "gbs_device.cuh"
#include "gbs_internal.h"

namespace gbs {

namespace {

// Gauss-Legendre rule on [-1, 1] by bisection on sign changes of P_n and the
// weight formula w = 2 (1 - x^2) / (n P_{n-1}(x))^2.
void legendre_pair(int n, double x, double* pn, double* pn1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (n == 0) {
    *pn = 1.0;
    *pn1 = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  *pn = b;   // P_n
  *pn1 = a;  // P_{n-1}
}

void gauss_rule_host(int n, double* x, double* w) {
  const int M = 400 * n;
  int found = 0;
  double prevx = -1.0, prevp, dummy;
  legendre_pair(n, prevx, &prevp, &dummy);
  for (int s = 1; s <= M && found < n; ++s) {
    double cx = -std::cos(M_PI * s / M);  // fine grid clustered at the ends
    double cp;
    legendre_pair(n, cx, &cp, &dummy);
    if ((prevp < 0) != (cp < 0) || cp == 0.0) {
      double lo = prevx, hi = cx, plo = prevp;
      for (int it = 0; it < 200 && hi - lo > 0; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double pm;
        legendre_pair(n, mid, &pm, &dummy);
        if ((pm < 0) == (plo < 0)) {
          lo = mid;
          plo = pm;
        } else {
          hi = mid;
        }
      }
      double r = 0.5 * (lo + hi), pn, pn1;
      legendre_pair(n, r, &pn, &pn1);
      x[found] = r;
      w[found] = 2.0 * (1.0 - r * r) / ((double)n * n * pn1 * pn1);
      ++found;
    }
    prevx = cx;
    prevp = cp;
  }
  if (found != n) fail(GB_ERR_INVALID_ARG, "gauss rule: root search failed");
}

struct Rule {
  int n;
  double x[12], w[12];
};

Rule make_rule(int n) {
  Rule r;
  r.n = n;
  gauss_rule_host(n, r.x, r.w);
  return r;
}

struct SpaceDev {
  int dim, N, p;
  int voff[4];
  int len[3][3];  // len[c][k]
  int lo[3][3];
};

SpaceDev make_space(const Ctx& c) {
  SpaceDev s;
  s.dim = c.dim;
  s.N = c.N;
  s.p = c.p;
  int off = 0;
  for (int cc = 0; cc < 4; ++cc) {
    s.voff[cc] = off;
    if (cc < c.dim) {
      int m = 1;
      for (int k = 0; k < c.dim; ++k) {
        s.lo[cc][k] = (k == cc) ? 1 : 0;
        s.len[cc][k] = (k == cc) ? c.N + c.p - 2 : c.N + c.p - 1;
        m *= s.len[cc][k];
      }
      off += m;
    }
  }
  return s;
}

__device__ __forceinline__ void vdecode_dev(const SpaceDev& S, int i, int* c, int* a) {
  int cc = S.dim - 1;
  while (cc > 0 && i < S.voff[cc]) --cc;
  int r = i - S.voff[cc];
  for (int k = S.dim - 1; k >= 0; --k) {
    int l = S.len[cc][k];
    a[k] = r % l + S.lo[cc][k];
    r /= l;
  }
  *c = cc;
}

__device__ __forceinline__ void pdecode_dev(const SpaceDev& S, int i, int* a) {
  const int m = S.N + S.p - 1;
  for (int k = S.dim - 1; k >= 0; --k) {
    a[k] = i % m;
    i /= m;
  }
}

// 1D table layout: integrals I[si][sj][oi][oj][a][o] with si, sj in {0: degree
// p, 1: degree p-1}, oi, oj in {0: value, 1: derivative}, a the row function,
// o = b - a + q_si the band offset (0 .. q_si + q_sj); then face values
// F[s][side][o][a]; then W1[a] = integral of the degree p-1 function a.
struct Tab {
  int nmax, bw;
  size_t off_face, off_w, total;
};

Tab tab_layout(int N, int p) {
  Tab t;
  t.nmax = N + p;
  t.bw = 2 * p + 1;
  t.off_face = (size_t)16 * t.nmax * t.bw;
  t.off_w = t.off_face + (size_t)2 * 2 * 2 * t.nmax;
  t.total = t.off_w + t.nmax;
  return t;
}

__device__ __forceinline__ size_t tab_idx(const Tab& T, int si, int sj, int oi, int oj, int a, int o) {
  return ((size_t)(((si * 2 + sj) * 2 + oi) * 2 + oj) * T.nmax + a) * T.bw + o;
}

__global__ void k_tables_1d(int N, int p, Rule rule, Tab T, double* tab) {
  // one thread per (si, sj, oi, oj, a, o) entry, plus face/W entries
  const size_t nint = (size_t)16 * T.nmax * T.bw;
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < nint) {
    int o = (int)(id % T.bw);
    size_t r = id / T.bw;
    int a = (int)(r % T.nmax);
    r /= T.nmax;
    int oj = (int)(r % 2);
    r /= 2;
    int oi = (int)(r % 2);
    r /= 2;
    int sj = (int)(r % 2);
    int si = (int)(r / 2);
    const int qi = si == 0 ? p : p - 1, qj = sj == 0 ? p : p - 1;
    const int b = a - qi + o;
    double acc = 0.0;
    if (a < N + qi && b >= 0 && b < N + qj && o <= qi + qj) {
      // shared elements: [max(a-qi, b-qj), min(a, b)] within [0, N-1]
      int e0 = max(max(a - qi, b - qj), 0), e1 = min(min(a, b), N - 1);
      for (int e = e0; e <= e1; ++e) {
        for (int g = 0; g < rule.n; ++g) {
          const double x = (e + 0.5 * (rule.x[g] + 1.0)) / N;
          const double wgt = 0.5 * rule.w[g] / N;
          double vi[8], di[8], vj[8], dj[8];
          bspline_element(N, qi, e, x, vi, di);
          bspline_element(N, qj, e, x, vj, dj);
          const double fi = oi ? di[a - e] : vi[a - e];
          const double fj = oj ? dj[b - e] : vj[b - e];
          acc += wgt * fi * fj;
        }
      }
    }
    tab[id] = acc;
    return;
  }
  const size_t id2 = id - nint;
  const size_t nface = (size_t)2 * 2 * 2 * T.nmax;
  if (id2 < nface) {
    int a = (int)(id2 % T.nmax);
    size_t r = id2 / T.nmax;
    int o = (int)(r % 2);
    r /= 2;
    int side = (int)(r % 2);
    int s = (int)(r / 2);
    const int q = s == 0 ? p : p - 1;
    double out = 0.0;
    if (a < N + q) {
      const int e = side == 0 ? 0 : N - 1;
      const double x = side == 0 ? 0.0 : 1.0;
      if (a >= e && a <= e + q) {
        double v[8], d[8];
        bspline_element(N, q, e, x, v, d);
        out = o ? d[a - e] : v[a - e];
      }
    }
    tab[T.off_face + id2] = out;
    return;
  }
  const size_t id3 = id2 - nface;
  if (id3 < (size_t)T.nmax) {
    const int a = (int)id3, q = p - 1;
    double acc = 0.0;
    if (a < N + q) {
      for (int e = max(a - q, 0); e <= min(a, N - 1); ++e)
        for (int g = 0; g < rule.n; ++g) {
          const double x = (e + 0.5 * (rule.x[g] + 1.0)) / N;
          double v[8], d[8];
          bspline_element(N, q, e, x, v, d);
          acc += 0.5 * rule.w[g] / N * v[a - e];
        }
    }
    tab[T.off_w + id3] = acc;
  }
}

struct AsmParams {
  SpaceDev S;
  Tab T;
  const double* tab;
  double nu, cpen;
};

__device__ __forceinline__ double I1(const AsmParams& P, int si, int sj, int oi, int oj, int a, int b) {
  const int qi = si == 0 ? P.S.p : P.S.p - 1;
  return P.tab[tab_idx(P.T, si, sj, oi, oj, a, b - a + qi)];
}

__device__ __forceinline__ double F1(const AsmParams& P, int s, int side, int o, int a) {
  return P.tab[P.T.off_face + ((size_t)(s * 2 + side) * 2 + o) * P.T.nmax + a];
}

// [A_h]_ij = a(Phi_j, Phi_i) - eta_h(Phi_j, Phi_i) for velocity functions
// i = (ci, a) and j = (cj, b) (Sec. 4), from 1D factors.
//   grad^s Phi_i : grad^s Phi_j = 1/2 [ci==cj] sum_m d_m phi_i d_m phi_j
//                                + 1/2 d_{cj} phi_i d_{ci} phi_j
//   on a face x_k = side with outward normal n = +-e_k:
//   (grad^s Phi_i n).Phi_j = n/2 ([ci==cj] d_k phi_i + [k==ci] d_{cj} phi_i) phi_j
__device__ double entry_A(const AsmParams& P, int ci, const int* a, int cj, const int* b) {
  const int dim = P.S.dim;
  int si[3], sj[3];
  for (int k = 0; k < dim; ++k) {
    si[k] = (k == ci) ? 0 : 1;
    sj[k] = (k == cj) ? 0 : 1;
  }
  double val = 0.0;
  if (ci == cj) {
    for (int m = 0; m < dim; ++m) {
      double prod = 1.0;
      for (int k = 0; k < dim; ++k) prod *= I1(P, si[k], sj[k], k == m, k == m, a[k], b[k]);
      val += 0.5 * prod;
    }
  }
  {
    double prod = 1.0;
    for (int k = 0; k < dim; ++k) prod *= I1(P, si[k], sj[k], k == cj, k == ci, a[k], b[k]);
    val += 0.5 * prod;
  }
  val *= 2.0 * P.nu;
  const double hF = 1.0 / P.S.N;
  for (int k = 0; k < dim; ++k) {
    for (int side = 0; side < 2; ++side) {
      const double fi0 = F1(P, si[k], side, 0, a[k]), fi1 = F1(P, si[k], side, 1, a[k]);
      const double fj0 = F1(P, sj[k], side, 0, b[k]), fj1 = F1(P, sj[k], side, 1, b[k]);
      if ((fi0 == 0.0 && fi1 == 0.0) || (fj0 == 0.0 && fj1 == 0.0)) continue;
      const double nk = side == 0 ? -1.0 : 1.0;
      // T(di, dj): derivative direction on phi_i / phi_j (-1: none)
      auto term = [&](int di, int dj) {
        double prod = (di == k ? fi1 : fi0) * (dj == k ? fj1 : fj0);
        for (int m = 0; m < dim; ++m)
          if (m != k) prod *= I1(P, si[m], sj[m], di == m, dj == m, a[m], b[m]);
        return prod;
      };
      double eta = 0.0;
      if (ci == cj) {
        eta += 0.5 * nk * term(k, -1);
        eta += 0.5 * nk * term(-1, k);
        eta -= (P.cpen / hF) * term(-1, -1);
      }
      if (k == ci) eta += 0.5 * nk * term(cj, -1);
      if (k == cj) eta += 0.5 * nk * term(-1, ci);
      val -= 2.0 * P.nu * eta;
    }
  }
  return val;
}

// One warp per internal row of A_h; lanes over the row's nonzeros.
__global__ void k_assemble_A(AsmParams P, int n, const int32_t* __restrict__ ptr,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ order,
                             double* __restrict__ val, float* __restrict__ val32) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n; r += nwarps) {
    int ci, a[3] = {0, 0, 0};
    vdecode_dev(P.S, order[r], &ci, a);
    for (int t = ptr[r] + lane; t < ptr[r + 1]; t += 32) {
      int cj, b[3] = {0, 0, 0};
      vdecode_dev(P.S, order[col[t]], &cj, b);
      const double v = entry_A(P, ci, a, cj, b);
      val[t] = v;
      val32[t] = (float)v;
    }
  }
}

// [B]_kj = -(div Phi_j, phi_k) = -prod_m I(p-1, 0, a_m; q(cj,m), [m==cj], b_m).
__global__ void k_assemble_B(AsmParams P, int np, const int32_t* __restrict__ ptr,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ order,
                             double* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int kr = warp; kr < np; kr += nwarps) {
    int a[3] = {0, 0, 0};
    pdecode_dev(P.S, kr, a);
    for (int t = ptr[kr] + lane; t < ptr[kr + 1]; t += 32) {
      int cj, b[3] = {0, 0, 0};
      vdecode_dev(P.S, order[col[t]], &cj, b);
      double prod = -1.0;
      for (int m = 0; m < P.S.dim; ++m) prod *= I1(P, 1, m == cj ? 0 : 1, 0, m == cj, a[m], b[m]);
      val[t] = prod;
    }
  }
}

__global__ void k_gather_bt(int nnz, const int32_t* __restrict__ map, const double* __restrict__ bval,
                            double* __restrict__ btval) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += gridDim.x * blockDim.x)
    btval[t] = bval[map[t]];
}

// Diag(Q)_kk = prod_m I(p-1, 0, a_m; p-1, 0, a_m);  w_k = prod_m W1[a_m].
__global__ void k_pressure_diag(AsmParams P, int np, double* __restrict__ qdiag, double* __restrict__ w) {
  for (int kr = blockIdx.x * blockDim.x + threadIdx.x; kr < np; kr += gridDim.x * blockDim.x) {
    int a[3] = {0, 0, 0};
    pdecode_dev(P.S, kr, a);
    double q = 1.0, ww = 1.0;
    for (int m = 0; m < P.S.dim; ++m) {
      q *= I1(P, 1, 1, 0, 0, a[m], a[m]);
      ww *= P.tab[P.T.off_w + a[m]];
    }
    qdiag[kr] = q;
    w[kr] = ww;
  }
}

// Q_kl = prod_m I(p-1, 0, a_m; p-1, 0, b_m) = (phi_l, phi_k) on the pattern of
// Q (natural numbering, one thread per row), with its FP32 copy.
__global__ void k_assemble_Q(AsmParams P, int np, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                             double* __restrict__ val, float* __restrict__ val32) {
  for (int kr = blockIdx.x * blockDim.x + threadIdx.x; kr < np; kr += gridDim.x * blockDim.x) {
    int a[3] = {0, 0, 0};
    pdecode_dev(P.S, kr, a);
    for (int t = ptr[kr]; t < ptr[kr + 1]; ++t) {
      int b[3] = {0, 0, 0};
      pdecode_dev(P.S, col[t], b);
      double q = 1.0;
      for (int m = 0; m < P.S.dim; ++m) q *= I1(P, 1, 1, 0, 0, a[m], b[m]);
      val[t] = q;
      val32[t] = (float)q;
    }
  }
}

// Lower band of the 1D mass matrix Q1 of the m = N + p - 1 degree-(p-1)
// B-splines: q1[a * p + o] = Q1[a][a - o] for o = 0 .. p-1 (0 where a < o).
__global__ void k_mass_band(AsmParams P, int m, double* __restrict__ q1) {
  const int p = P.S.p;
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < m * p; id += gridDim.x * blockDim.x) {
    const int a = id / p, o = id % p;
    q1[id] = a >= o ? I1(P, 1, 1, 0, 0, a, a - o) : 0.0;
  }
}

// ---- loads -------------------------------------------------------------
// S[m][k][s][a] = int_0^1 sin(pi kappa_{m,k} x) B^{q_s}_a(x) dx, Gauss p+3.
__global__ void k_fourier_1d(int N, int p, int dim, int nmodes, const int32_t* __restrict__ kappa,
                             Rule rule, int nmax, double* __restrict__ S) {
  const int total = nmodes * dim * 2 * nmax;
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < total; id += gridDim.x * blockDim.x) {
    int a = id % nmax;
    int r = id / nmax;
    int s = r % 2;
    r /= 2;
    int k = r % dim;
    int m = r / dim;
    const int q = s == 0 ? p : p - 1;
    double acc = 0.0;
    if (a < N + q) {
      const double kap = M_PI * kappa[m * dim + k];
      for (int e = max(a - q, 0); e <= min(a, N - 1); ++e)
        for (int g = 0; g < rule.n; ++g) {
          const double x = (e + 0.5 * (rule.x[g] + 1.0)) / N;
          double v[8], d[8];
          bspline_element(N, q, e, x, v, d);
          acc += 0.5 * rule.w[g] / N * sin(kap * x) * v[a - e];
        }
    }
    S[id] = acc;
  }
}

__global__ void k_fourier_load(SpaceDev Sp, int nmodes, const double* __restrict__ amp,
                               const double* __restrict__ S, int nmax, double* __restrict__ f, int n_u) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_u; i += gridDim.x * blockDim.x) {
    int c, a[3] = {0, 0, 0};
    vdecode_dev(Sp, i, &c, a);
    double acc = 0.0;
    for (int m = 0; m < nmodes; ++m) {
      double prod = amp[m * Sp.dim + c];
      for (int k = 0; k < Sp.dim; ++k) {
        const int s = (k == c) ? 0 : 1;
        prod *= S[((size_t)(m * Sp.dim + k) * 2 + s) * nmax + a[k]];
      }
      acc += prod;
    }
    f[i] = acc;
  }
}

// Manufactured forcing of Sec. 6.2 (2D): with G(x) = x^2 (x-1)^2 and
// H(y) = (y^2 - y)^2, u = (e^x G H', -(e^x G)' H) and the printed pressure
// p = -424 + 156 e + s (-456 + e^x (P0(x) + s P1(x))), s = y^2 - y.
// f = -nu lap u + grad p (div u = 0).
__device__ inline void manufactured_force(double nu, double x, double y, double* f) {
  auto horner = [](const double* c, int n, double t) {
    double r = c[n - 1];
    for (int i = n - 2; i >= 0; --i) r = r * t + c[i];
    return r;
  };
  // coefficients, lowest degree first
  const double G[5] = {0, 0, 1, -2, 1}, G1[4] = {0, 2, -6, 4}, G2[3] = {2, -12, 12}, G3[2] = {-12, 24};
  const double g = horner(G, 5, x), g1 = horner(G1, 4, x), g2 = horner(G2, 3, x), g3 = horner(G3, 2, x);
  const double h = horner(G, 5, y), h1 = horner(G1, 4, y), h2 = horner(G2, 3, y), h3 = horner(G3, 2, y);
  const double ex = exp(x);
  const double lap_u1 = ex * ((g + 2 * g1 + g2) * h1 + g * h3);
  const double lap_u2 = -ex * ((g + 3 * g1 + 3 * g2 + g3) * h + (g + g1) * h2);
  const double P0c[5] = {456, -456, 228, -72, 12}, P0d[4] = {-456, 456, -216, 48};
  const double P1c[5] = {0, 2, -5, 2, 1}, P1d[4] = {2, -10, 6, 4};
  const double s = y * y - y, sy = 2 * y - 1;
  const double P0 = horner(P0c, 5, x), P1 = horner(P1c, 5, x);
  const double dP0 = horner(P0d, 4, x), dP1 = horner(P1d, 4, x);
  const double px = s * ex * (P0 + s * P1 + dP0 + s * dP1);
  const double py = sy * (-456.0 + ex * (P0 + 2.0 * s * P1));
  f[0] = -nu * lap_u1 + px;
  f[1] = -nu * lap_u2 + py;
}

__global__ void k_manufactured_load(SpaceDev Sp, Rule rule, double nu, double* __restrict__ f, int n_u) {
  const int N = Sp.N, p = Sp.p;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_u; i += gridDim.x * blockDim.x) {
    int c, a[3] = {0, 0, 0};
    vdecode_dev(Sp, i, &c, a);
    const int q0 = (c == 0) ? p : p - 1, q1 = (c == 1) ? p : p - 1;
    double acc = 0.0;
    for (int e0 = max(a[0] - q0, 0); e0 <= min(a[0], N - 1); ++e0)
      for (int e1 = max(a[1] - q1, 0); e1 <= min(a[1], N - 1); ++e1)
        for (int g0 = 0; g0 < rule.n; ++g0) {
          const double x = (e0 + 0.5 * (rule.x[g0] + 1.0)) / N;
          double v0[8], d0[8];
          bspline_element(N, q0, e0, x, v0, d0);
          for (int g1 = 0; g1 < rule.n; ++g1) {
            const double y = (e1 + 0.5 * (rule.x[g1] + 1.0)) / N;
            double v1[8], d1[8];
            bspline_element(N, q1, e1, y, v1, d1);
            double fv[2];
            manufactured_force(nu, x, y, fv);
            acc += 0.25 * rule.w[g0] * rule.w[g1] / ((double)N * N) * fv[c] * v0[a[0] - e0] * v1[a[1] - e1];
          }
        }
    f[i] = acc;
  }
}

// Lid-driven cavity load (Sec. 6.4): the Nitsche right-hand side of
// eq. nitsche_rhs with lid velocity g = e_1 on the face x_k = 1, k = dim - 1.
// Only the first velocity component has a tangential trace along e_1 there:
// for Phi = phi e_1, ((grad^s Phi) n) . g = (1/2) d_k phi, so
//   l = 2 nu prod_{m != k} (int_0^1 B_{a_m}) * (-(1/2) B'_{a_k}(1) + (C_pen / h_F) B_{a_k}(1)),
// with int_0^1 B^q_a = (xi_{a+q+1} - xi_a) / (q+1) and the end values from
// Cox-de Boor on the last element.  Other components give 0 (their normal
// trace on the lid is removed from the space, so phi = d_1 phi = 0 there).
__global__ void k_cavity_load(SpaceDev Sp, double nu, double cpen, double* __restrict__ f, int n_u) {
  const int N = Sp.N, p = Sp.p, k = Sp.dim - 1;
  double v[8], d[8];
  bspline_element(N, p - 1, N - 1, 1.0, v, d);  // degree p-1 functions N-1 .. N+p-2 at x = 1
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_u; i += gridDim.x * blockDim.x) {
    int c, a[3] = {0, 0, 0};
    vdecode_dev(Sp, i, &c, a);
    double out = 0.0;
    if (c == 0 && a[k] >= N - 1) {
      const int t = a[k] - (N - 1);
      double w = 1.0;
      for (int m = 0; m < Sp.dim; ++m) {
        if (m == k) continue;
        const int q = (m == 0) ? p : p - 1;  // degree of component 1 in direction m
        w *= (open_knot(a[m] + q + 1, q, N) - open_knot(a[m], q, N)) / (q + 1);
      }
      out = 2.0 * nu * w * (-0.5 * d[t] + cpen * N * v[t]);
    }
    f[i] = out;
  }
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

}  // namespace

void assemble(Ctx& c, double nu, double cpen) {
  if (!(nu > 0.0) || !std::isfinite(nu)) fail(GB_ERR_INVALID_ARG, "nu must be positive");
  if (!std::isfinite(cpen)) fail(GB_ERR_INVALID_ARG, "cpen must be finite");
  if (cpen <= 0.0) cpen = 5.0 * c.p;  // C_pen = 5 (k' + 1), k' = p - 1 (Sec. 6.2)
  c.nu = nu;
  c.cpen = cpen;
  const Tab T = tab_layout(c.N, c.p);
  c.tab1d.alloc(T.total);
  const Rule rule = make_rule(c.p + 1);
  const size_t nthreads = (size_t)16 * T.nmax * T.bw + 8 * T.nmax + T.nmax;
  k_tables_1d<<<(unsigned)((nthreads + 127) / 128), 128, 0, c.stream>>>(c.N, c.p, rule, T, c.tab1d.p);
  GBS_CUDA(cudaGetLastError());
  AsmParams P;
  P.S = make_space(c);
  P.T = T;
  P.tab = c.tab1d.p;
  P.nu = nu;
  P.cpen = cpen;
  k_assemble_A<<<grid_for(c.n_u * 32, 256), 256, 0, c.stream>>>(P, (int)c.n_u, c.A_ptr.p, c.A_col.p,
                                                                  c.order_d.p, c.A_val.p, c.A_val32.p);
  GBS_CUDA(cudaGetLastError());
  k_assemble_B<<<grid_for(c.n_p * 32, 256), 256, 0, c.stream>>>(P, (int)c.n_p, c.B_ptr.p, c.B_col.p,
                                                                  c.order_d.p, c.B_val.p);
  GBS_CUDA(cudaGetLastError());
  k_gather_bt<<<grid_for(c.nnzB, 256), 256, 0, c.stream>>>((int)c.nnzB, c.Bt_map.p, c.B_val.p, c.Bt_val.p);
  GBS_CUDA(cudaGetLastError());
  sell_refill(c, c.sA, c.A_val.p);
  k_pressure_diag<<<grid_for(c.n_p, 256), 256, 0, c.stream>>>(P, (int)c.n_p, c.Qdiag.p, c.wmean.p);
  GBS_CUDA(cudaGetLastError());
  k_assemble_Q<<<grid_for(c.n_p, 256), 256, 0, c.stream>>>(P, (int)c.n_p, c.Q_ptr.p, c.Q_col.p, c.Q_val.p,
                                                            c.Q_val32.p);
  GBS_CUDA(cudaGetLastError());
  k_mass_band<<<grid_for((int64_t)(c.N + c.p - 1) * c.p, 256), 256, 0, c.stream>>>(P, c.N + c.p - 1, c.q1.p);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  c.assembled = true;
  c.factored = false;
  c.q_factored = false;
  c.ws.graph_valid = false;
}

void load_fourier(Ctx& c, int nmodes, const int32_t* kappa, const double* amp, double* f_dev) {
  if (nmodes < 1 || nmodes > 4096 || !kappa || !amp || !f_dev)
    fail(GB_ERR_INVALID_ARG, "load_fourier: bad arguments");
  const int nmax = c.N + c.p;
  DevBuf<int32_t> kd;
  DevBuf<double> ad, S;
  kd.upload(kappa, (size_t)nmodes * c.dim, c.stream);
  ad.upload(amp, (size_t)nmodes * c.dim, c.stream);
  S.alloc((size_t)nmodes * c.dim * 2 * nmax);
  const Rule rule = make_rule(c.p + 3);
  k_fourier_1d<<<grid_for((int64_t)nmodes * c.dim * 2 * nmax, 128), 128, 0, c.stream>>>(
      c.N, c.p, c.dim, nmodes, kd.p, rule, nmax, S.p);
  GBS_CUDA(cudaGetLastError());
  k_fourier_load<<<grid_for(c.n_u, 256), 256, 0, c.stream>>>(make_space(c), nmodes, ad.p, S.p, nmax,
                                                              f_dev, (int)c.n_u);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  kd.free_();
  ad.free_();
  S.free_();
}

void load_cavity(Ctx& c, double* f_dev) {
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "assemble first (the load uses nu and C_pen)");
  if (!f_dev) fail(GB_ERR_INVALID_ARG, "null output");
  k_cavity_load<<<grid_for(c.n_u, 128), 128, 0, c.stream>>>(make_space(c), c.nu, c.cpen, f_dev, (int)c.n_u);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaStreamSynchronize(c.stream));
}

void load_manufactured(Ctx& c, double* f_dev) {
  if (c.dim != 2) fail(GB_ERR_INVALID_ARG, "the manufactured solution is two-dimensional");
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "assemble first (the forcing uses nu)");
  if (!f_dev) fail(GB_ERR_INVALID_ARG, "null output");
  const Rule rule = make_rule(c.p + 3);
  k_manufactured_load<<<grid_for(c.n_u, 128), 128, 0, c.stream>>>(make_space(c), rule, c.nu, f_dev,
                                                                   (int)c.n_u);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace gbs
