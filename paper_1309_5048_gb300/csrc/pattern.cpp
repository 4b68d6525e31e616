// pattern.cpp -- host construction of the discrete spaces, sparsity
// patterns, ordering, IC(0) level sets and the internal numbering (no CUDA;
// setup uploads the result, pattern.h).
//
// Spaces (Sec. 3.2): velocity component c is the tensor-product B-spline
// space of degree p in direction c and p-1 in the other directions (maximal
// continuity, uniform open knots, N elements per direction) without the
// first and last function in direction c (normal component zero on the
// boundary: V_{0,h}); pressure is degree p-1 in every direction (Q_h).
// Two 1D B-splines of degrees q (index a) and q' (index b) share an element
// iff b - a lies in [-q, q'], so every pattern here has a closed form.
#include "pattern.h"

#include <algorithm>
#include <climits>
#include <deque>
#include <numeric>
#include <thread>

namespace gbs {

namespace {

// Run fn(lo, hi) over [0, n) split across hardware threads.
template <class F>
void parallel_ranges(int64_t n, F fn) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < 20000) nt = 1;
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=] { fn(lo, hi); });
  }
  for (auto& t : th) t.join();
}

struct Numbering {
  int dim, N, p;
  int64_t voff[4];
  int64_t n_u, n_p;
  int deg(int c, int k) const { return k == c ? p : p - 1; }
  // kept 1D index range of component c in direction k (original indices)
  int lo(int c, int k) const { return k == c ? 1 : 0; }
  int hi(int, int) const { return N + p - 2; }
  int len(int c, int k) const { return hi(c, k) - lo(c, k) + 1; }
  int64_t vindex(int c, const int* a) const {
    int64_t r = 0;
    for (int k = 0; k < dim; ++k) r = r * len(c, k) + (a[k] - lo(c, k));
    return voff[c] + r;
  }
  void vdecode(int64_t i, int* c, int* a) const {
    int cc = dim - 1;
    while (cc > 0 && i < voff[cc]) --cc;
    int64_t r = i - voff[cc];
    for (int k = dim - 1; k >= 0; --k) {
      a[k] = (int)(r % len(cc, k)) + lo(cc, k);
      r /= len(cc, k);
    }
    *c = cc;
  }
  int64_t pindex(const int* a) const {
    int64_t r = 0;
    for (int k = 0; k < dim; ++k) r = r * (N + p - 1) + a[k];
    return r;
  }
  void pdecode(int64_t i, int* a) const {
    for (int k = dim - 1; k >= 0; --k) {
      a[k] = (int)(i % (N + p - 1));
      i /= (N + p - 1);
    }
  }
  // Velocity neighbours of velocity DOF i (natural), ascending.
  template <class F>
  void vel_neighbours(int64_t i, F emit) const {
    int c, a[3] = {0, 0, 0};
    vdecode(i, &c, a);
    for (int c2 = 0; c2 < dim; ++c2) {
      int l[3] = {0, 0, 0}, h[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) {
        l[k] = std::max(a[k] - deg(c, k), lo(c2, k));
        h[k] = std::min(a[k] + deg(c2, k), hi(c2, k));
      }
      int b[3] = {0, 0, 0};
      for (b[0] = l[0]; b[0] <= h[0]; ++b[0])
        for (b[1] = l[1]; b[1] <= h[1]; ++b[1])
          for (b[2] = (dim == 3 ? l[2] : 0); b[2] <= (dim == 3 ? h[2] : 0); ++b[2])
            emit(vindex(c2, b));
    }
  }
  int64_t vel_degree(int64_t i) const {
    int c, a[3] = {0, 0, 0};
    vdecode(i, &c, a);
    int64_t tot = 0;
    for (int c2 = 0; c2 < dim; ++c2) {
      int64_t prod = 1;
      for (int k = 0; k < dim; ++k) {
        int l = std::max(a[k] - deg(c, k), lo(c2, k));
        int h = std::min(a[k] + deg(c2, k), hi(c2, k));
        prod *= std::max(0, h - l + 1);
      }
      tot += prod;
    }
    return tot;
  }
  // Velocity columns of pressure row k (natural), ascending.
  template <class F>
  void pres_row(int64_t kk, F emit) const {
    int a[3] = {0, 0, 0};
    pdecode(kk, a);
    for (int c2 = 0; c2 < dim; ++c2) {
      int l[3] = {0, 0, 0}, h[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) {
        l[k] = std::max(a[k] - (p - 1), lo(c2, k));
        h[k] = std::min(a[k] + deg(c2, k), hi(c2, k));
      }
      int b[3] = {0, 0, 0};
      for (b[0] = l[0]; b[0] <= h[0]; ++b[0])
        for (b[1] = l[1]; b[1] <= h[1]; ++b[1])
          for (b[2] = (dim == 3 ? l[2] : 0); b[2] <= (dim == 3 ? h[2] : 0); ++b[2])
            emit(vindex(c2, b));
    }
  }
};

Numbering make_numbering(int dim, int N, int p) {
  Numbering nb;
  nb.dim = dim;
  nb.N = N;
  nb.p = p;
  int64_t off = 0;
  for (int c = 0; c < 4; ++c) {
    nb.voff[c] = off;
    if (c < dim) {
      int64_t m = 1;
      for (int k = 0; k < dim; ++k) m *= nb.len(c, k);
      off += m;
    }
  }
  nb.n_u = off;
  nb.n_p = 1;
  for (int k = 0; k < dim; ++k) nb.n_p *= (N + p - 1);
  return nb;
}

// ---- orderings -------------------------------------------------------------
// Reverse Cuthill-McKee from a George-Liu pseudo-peripheral node: start from
// the unnumbered node of least degree (lowest index on ties), repeatedly jump
// to the least-degree node of the farthest BFS level while that increases the
// eccentricity; number breadth-first visiting neighbours by (degree, index);
// reverse the result.
void order_rcm(const Numbering& nb, std::vector<int32_t>& perm) {
  const int64_t n = nb.n_u;
  std::vector<int32_t> deg(n);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) deg[i] = (int32_t)(nb.vel_degree(i) - 1);
  });
  std::vector<char> done(n, 0);
  std::vector<int32_t> dist(n, -1), seq;
  seq.reserve(n);
  std::vector<int32_t> touched;
  auto eccentricity = [&](int32_t root, int32_t* far_node) {
    // BFS over unnumbered nodes; returns eccentricity and the least-degree
    // node (lowest index on ties) of the last level.
    touched.clear();
    std::deque<int32_t> q;
    dist[root] = 0;
    touched.push_back(root);
    q.push_back(root);
    int ecc = 0;
    while (!q.empty()) {
      int32_t u = q.front();
      q.pop_front();
      ecc = std::max(ecc, dist[u]);
      nb.vel_neighbours(u, [&](int64_t v) {
        if (v == u || done[v] || dist[v] >= 0) return;
        dist[v] = dist[u] + 1;
        touched.push_back((int32_t)v);
        q.push_back((int32_t)v);
      });
    }
    int32_t best = -1;
    for (int32_t v : touched)
      if (dist[v] == ecc && (best < 0 || deg[v] < deg[best] || (deg[v] == deg[best] && v < best)))
        best = v;
    for (int32_t v : touched) dist[v] = -1;
    *far_node = best;
    return ecc;
  };
  std::vector<int32_t> nbrs;
  int64_t scan = 0;
  while ((int64_t)seq.size() < n) {
    int32_t r = -1;
    for (int64_t i = 0; i < n; ++i)
      if (!done[i] && (r < 0 || deg[i] < deg[r])) r = (int32_t)i;
    (void)scan;
    int32_t far;
    int ecc = eccentricity(r, &far);
    for (;;) {
      int32_t far2;
      int e2 = eccentricity(far, &far2);
      if (e2 > ecc) {
        r = far;
        ecc = e2;
        far = far2;
      } else {
        break;
      }
    }
    size_t head = seq.size();
    seq.push_back(r);
    done[r] = 1;
    while (head < seq.size()) {
      int32_t u = seq[head++];
      nbrs.clear();
      nb.vel_neighbours(u, [&](int64_t v) {
        if (!done[v]) nbrs.push_back((int32_t)v);
      });
      std::sort(nbrs.begin(), nbrs.end(), [&](int32_t x, int32_t y) {
        return deg[x] != deg[y] ? deg[x] < deg[y] : x < y;
      });
      for (int32_t v : nbrs) {
        done[v] = 1;
        seq.push_back(v);
      }
    }
  }
  perm.assign(seq.rbegin(), seq.rend());
}

// Multicolour ordering: DOF (c, a) of component c gets the colour
// (c, (a_k - lo_k) mod (deg(c,k)+1) for each k); equal colours never couple in
// A_h.  Rows are sorted by colour, natural order inside a colour.
int order_multicolour(const Numbering& nb, std::vector<int32_t>& perm) {
  const int64_t n = nb.n_u;
  std::vector<int64_t> colour(n);
  int64_t ncol_total = 0;
  std::vector<int64_t> base(nb.dim + 1, 0);
  for (int c = 0; c < nb.dim; ++c) {
    int64_t m = 1;
    for (int k = 0; k < nb.dim; ++k) m *= nb.deg(c, k) + 1;
    base[c] = ncol_total;
    ncol_total += m;
  }
  for (int64_t i = 0; i < n; ++i) {
    int c, a[3] = {0, 0, 0};
    nb.vdecode(i, &c, a);
    int64_t col = 0;
    for (int k = 0; k < nb.dim; ++k) {
      int m = nb.deg(c, k) + 1;
      col = col * m + ((a[k] - nb.lo(c, k)) % m);
    }
    colour[i] = base[c] + col;
  }
  // counting sort by colour (stable)
  std::vector<int64_t> cnt(ncol_total + 1, 0);
  for (int64_t i = 0; i < n; ++i) cnt[colour[i] + 1]++;
  for (int64_t c = 0; c < ncol_total; ++c) cnt[c + 1] += cnt[c];
  perm.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) perm[cnt[colour[i]]++] = (int32_t)i;
  return (int)ncol_total;
}

}  // namespace

HostPattern build_pattern(int dim, int N, int p, int ordering) {
  if (dim != 2 && dim != 3) throw PatternError("dim must be 2 or 3");
  if (p < 2 || p > 6) throw PatternError("p must be in [2, 6]");
  if (N < 1 || N > 100000) throw PatternError("N out of range");
  if (ordering < 0 || ordering > 2) throw PatternError("unknown ordering");
  HostPattern P;
  P.dim = dim;
  P.N = N;
  P.p = p;
  const Numbering nb = make_numbering(dim, N, p);
  P.n_u = nb.n_u;
  P.n_p = nb.n_p;
  if (nb.n_u >= INT32_MAX || nb.n_p >= INT32_MAX) throw PatternError("too many unknowns");
  const int64_t n = nb.n_u;

  // ---- ordering
  P.ncolours = 0;
  if (ordering == 0) {
    P.perm.resize(n);
    std::iota(P.perm.begin(), P.perm.end(), 0);
  } else if (ordering == 1) {
    order_rcm(nb, P.perm);
  } else {
    P.ncolours = order_multicolour(nb, P.perm);
  }
  std::vector<int32_t> ipos(n);  // natural -> ordering position
  for (int64_t i = 0; i < n; ++i) ipos[P.perm[i]] = (int32_t)i;

  // ---- level sets of the factor's DAG (ordering numbering):
  // level(i) = 1 + max level(k) over lower neighbours k < i (0 without any),
  // rlevel the same over upper neighbours, processed from the last row.
  P.level.assign(n, 0);
  P.rlevel.assign(n, 0);
  int maxlev = 0, maxrlev = 0;
  for (int64_t i = 0; i < n; ++i) {
    int lv = -1;
    nb.vel_neighbours(P.perm[i], [&](int64_t v) {
      int32_t k = ipos[v];
      if (k < i) lv = std::max(lv, P.level[k]);
    });
    P.level[i] = lv + 1;
    maxlev = std::max(maxlev, lv + 1);
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    int lv = -1;
    nb.vel_neighbours(P.perm[i], [&](int64_t v) {
      int32_t k = ipos[v];
      if (k > i) lv = std::max(lv, P.rlevel[k]);
    });
    P.rlevel[i] = lv + 1;
    maxrlev = std::max(maxrlev, lv + 1);
  }
  P.nlev = maxlev + 1;
  P.nrlev = maxrlev + 1;

  // ---- internal numbering: ordering positions sorted by level (stable)
  P.lev_ptr.assign(P.nlev + 1, 0);
  for (int64_t i = 0; i < n; ++i) P.lev_ptr[P.level[i] + 1]++;
  for (int l = 0; l < P.nlev; ++l) P.lev_ptr[l + 1] += P.lev_ptr[l];
  P.int_to_pos.assign(n, 0);
  {
    std::vector<int32_t> fill(P.lev_ptr.begin(), P.lev_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) P.int_to_pos[fill[P.level[i]]++] = (int32_t)i;
  }
  P.order.resize(n);
  std::vector<int32_t> iorder(n);  // natural -> internal
  for (int64_t r = 0; r < n; ++r) {
    P.order[r] = P.perm[P.int_to_pos[r]];
    iorder[P.order[r]] = (int32_t)r;
  }

  // ---- A pattern in internal numbering
  std::vector<int64_t> rowlen(n);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) rowlen[r] = nb.vel_degree(P.order[r]);
  });
  std::vector<int64_t> ptr64(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) ptr64[r + 1] = ptr64[r] + rowlen[r];
  if (ptr64[n] >= INT32_MAX) throw PatternError("nnz(A) exceeds 32-bit indexing");
  P.nnzA = ptr64[n];
  P.hA_ptr.assign(n + 1, 0);
  for (int64_t r = 0; r <= n; ++r) P.hA_ptr[r] = (int32_t)ptr64[r];
  P.hA_col.resize(P.nnzA);
  std::vector<int32_t> hdiag(n);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) {
      int32_t* out = P.hA_col.data() + P.hA_ptr[r];
      int64_t t = 0;
      nb.vel_neighbours(P.order[r], [&](int64_t v) { out[t++] = iorder[v]; });
      std::sort(out, out + t);
      hdiag[r] = (int32_t)(std::lower_bound(out, out + t, (int32_t)r) - P.hA_col.data());
    }
  });

  // ---- L (strict lower = prefix of each A row) and U = L^T (strict upper)
  std::vector<int32_t> Lptr(n + 1, 0), Uptr(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) {
    Lptr[r + 1] = Lptr[r] + (hdiag[r] - P.hA_ptr[r]);
    Uptr[r + 1] = Uptr[r] + (P.hA_ptr[r + 1] - hdiag[r] - 1);
  }
  P.nnzL = Lptr[n] + n;
  std::vector<int32_t> Lcol(Lptr[n]), Ucol(Uptr[n]), Umap(Uptr[n]);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) {
      std::copy(P.hA_col.begin() + P.hA_ptr[r], P.hA_col.begin() + hdiag[r], Lcol.begin() + Lptr[r]);
      int32_t t = Uptr[r];
      for (int32_t s = hdiag[r] + 1; s < P.hA_ptr[r + 1]; ++s, ++t) {
        int32_t j = P.hA_col[s];  // j > r: entry L(j, r) lives in row j's prefix
        const int32_t* b = P.hA_col.data() + P.hA_ptr[j];
        const int32_t* e = P.hA_col.data() + hdiag[j];
        const int32_t* f = std::lower_bound(b, e, (int32_t)r);
        Ucol[t] = j;
        Umap[t] = Lptr[j] + (int32_t)(f - b);
      }
    }
  });

  // ---- B (pressure rows natural, velocity columns internal) and B^T
  const int64_t np = nb.n_p;
  std::vector<int64_t> Bptr64(np + 1, 0);
  for (int64_t k = 0; k < np; ++k) {
    int64_t cnt = 0;
    nb.pres_row(k, [&](int64_t) { ++cnt; });
    Bptr64[k + 1] = Bptr64[k] + cnt;
  }
  if (Bptr64[np] >= INT32_MAX) throw PatternError("nnz(B) exceeds 32-bit indexing");
  P.nnzB = Bptr64[np];
  P.hB_ptr.assign(np + 1, 0);
  for (int64_t k = 0; k <= np; ++k) P.hB_ptr[k] = (int32_t)Bptr64[k];
  P.hB_col.resize(P.nnzB);
  parallel_ranges(np, [&](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k) {
      int32_t* out = P.hB_col.data() + P.hB_ptr[k];
      int64_t t = 0;
      nb.pres_row(k, [&](int64_t v) { out[t++] = iorder[v]; });
      std::sort(out, out + t);
    }
  });
  // transpose (counting), rows internal velocity, cols ascending pressure
  std::vector<int32_t> Btptr(n + 1, 0), Btcol(P.nnzB), Btmap(P.nnzB);
  for (int64_t t = 0; t < P.nnzB; ++t) Btptr[P.hB_col[t] + 1]++;
  for (int64_t r = 0; r < n; ++r) Btptr[r + 1] += Btptr[r];
  {
    std::vector<int32_t> fill(Btptr.begin(), Btptr.end() - 1);
    for (int64_t k = 0; k < np; ++k)
      for (int32_t t = P.hB_ptr[k]; t < P.hB_ptr[k + 1]; ++t) {
        int32_t r = P.hB_col[t];
        Btcol[fill[r]] = (int32_t)k;
        Btmap[fill[r]] = t;
        fill[r]++;
      }
  }
  // structural nnz of Q: (2(p-1)+1)-band per direction, clipped
  {
    int64_t m = nb.N + nb.p - 1, per = 0;
    for (int64_t a = 0; a < m; ++a)
      per += std::min<int64_t>(m - 1, a + (nb.p - 1)) - std::max<int64_t>(0, a - (nb.p - 1)) + 1;
    P.nnzQ = 1;
    for (int k = 0; k < nb.dim; ++k) P.nnzQ *= per;
  }
  // pattern of Q (natural pressure numbering, ascending columns): pressure
  // functions k and l couple iff |a_d - b_d| <= p - 1 in every direction
  if (P.nnzQ >= INT32_MAX) throw PatternError("Q exceeds 32-bit indexing");
  std::vector<int32_t> Qptr(np + 1, 0), Qcol(P.nnzQ);
  {
    const int m = nb.N + nb.p - 1, w = nb.p - 1;
    auto row_len = [&](int64_t k) {
      int a[3] = {0, 0, 0};
      nb.pdecode(k, a);
      int64_t len = 1;
      for (int d = 0; d < nb.dim; ++d) len *= std::min(m - 1, a[d] + w) - std::max(0, a[d] - w) + 1;
      return len;
    };
    for (int64_t k = 0; k < np; ++k) Qptr[k + 1] = Qptr[k] + (int32_t)row_len(k);
    parallel_ranges(np, [&](int64_t lo, int64_t hi) {
      for (int64_t k = lo; k < hi; ++k) {
        int a[3] = {0, 0, 0}, l[3] = {0, 0, 0}, h[3] = {0, 0, 0}, b[3] = {0, 0, 0};
        nb.pdecode(k, a);
        for (int d = 0; d < nb.dim; ++d) {
          l[d] = std::max(0, a[d] - w);
          h[d] = std::min(m - 1, a[d] + w);
        }
        int32_t t = Qptr[k];
        for (b[0] = l[0]; b[0] <= h[0]; ++b[0])
          for (b[1] = (nb.dim > 1 ? l[1] : 0); b[1] <= (nb.dim > 1 ? h[1] : 0); ++b[1])
            for (b[2] = (nb.dim > 2 ? l[2] : 0); b[2] <= (nb.dim > 2 ? h[2] : 0); ++b[2])
              Qcol[t++] = (int32_t)nb.pindex(b);
      }
    });
  }

  P.iorder = std::move(iorder);
  P.A_diag = std::move(hdiag);
  P.L_ptr = std::move(Lptr);
  P.L_col = std::move(Lcol);
  P.U_ptr = std::move(Uptr);
  P.U_col = std::move(Ucol);
  P.U_map = std::move(Umap);
  P.Bt_ptr = std::move(Btptr);
  P.Bt_col = std::move(Btcol);
  P.Bt_map = std::move(Btmap);
  P.Q_ptr = std::move(Qptr);
  P.Q_col = std::move(Qcol);
  return P;
}

}  // namespace gbs
