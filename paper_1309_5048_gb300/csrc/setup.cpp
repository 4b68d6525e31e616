// setup.cpp -- host-side construction of the discrete spaces, sparsity
// patterns, ordering, IC(0) level sets and the internal numbering.
//
// Spaces (Sec. 3.2): velocity component c is the tensor-product B-spline
// space of degree p in direction c and p-1 in the other directions (maximal
// continuity, uniform open knots, N elements per direction) without the
// first and last function in direction c (normal component zero on the
// boundary: V_{0,h}); pressure is degree p-1 in every direction (Q_h).
// Two 1D B-splines of degrees q (index a) and q' (index b) share an element
// iff b - a lies in [-q, q'], so every pattern here has a closed form.
#include <algorithm>
#include <cstring>
#include <deque>
#include <numeric>
#include <thread>

#include "gbs_internal.h"

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

// SELL-32 copy of a CSR pattern (rows in internal numbering) with slices of
// 32 rows that never cross a level boundary (lev_ptr).
void build_sell(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                const std::vector<int32_t>& lev_ptr, std::vector<int32_t>& lev_slice, Sell& S,
                cudaStream_t stream) {
  const int nlev = (int)lev_ptr.size() - 1;
  std::vector<int32_t> row0, off, rowlen(ptr.size() - 1);
  lev_slice.assign(nlev + 1, 0);
  int64_t slots = 0;
  for (int l = 0; l < nlev; ++l) {
    lev_slice[l] = (int32_t)row0.size();
    for (int32_t r = lev_ptr[l]; r < lev_ptr[l + 1]; r += 32) {
      const int32_t r1 = std::min(r + 32, lev_ptr[l + 1]);
      int32_t len = 0;
      for (int32_t q = r; q < r1; ++q) len = std::max(len, ptr[q + 1] - ptr[q]);
      row0.push_back(r);
      off.push_back((int32_t)slots);
      slots += (int64_t)32 * len;
    }
  }
  lev_slice[nlev] = (int32_t)row0.size();
  if (slots >= INT32_MAX) fail(GB_ERR_INVALID_ARG, "SELL copy exceeds 32-bit indexing");
  S.nslices = (int)row0.size();
  row0.push_back(lev_ptr[nlev]);
  off.push_back((int32_t)slots);
  std::vector<int32_t> scol(slots, 0), ssrc(slots, -1);
  for (int s = 0; s < S.nslices; ++s)
    for (int32_t q = row0[s]; q < row0[s + 1]; ++q) {
      const int lane = q - row0[s];
      rowlen[q] = ptr[q + 1] - ptr[q];
      for (int32_t k = 0; k < rowlen[q]; ++k) {
        const int64_t slot = off[s] + (int64_t)32 * k + lane;
        scol[slot] = col[ptr[q] + k];
        ssrc[slot] = ptr[q] + k;
      }
    }
  S.slots = slots;
  S.row0.upload(row0.data(), row0.size(), stream);
  S.off.upload(off.data(), off.size(), stream);
  S.rowlen.upload(rowlen.data(), rowlen.size(), stream);
  S.col.upload(scol.data(), std::max<size_t>(1, scol.size()), stream);
  S.src.upload(ssrc.data(), std::max<size_t>(1, ssrc.size()), stream);
  S.val.alloc(std::max<int64_t>(1, slots));
  S.val32.alloc(std::max<int64_t>(1, slots));
}

// Upload of the staged partition of one sweep (layouts.h); an unavailable
// layout (a row longer than a block) stays empty with ok false.
void build_staged(const std::vector<int32_t>& ptr, const std::vector<int32_t>& lev_ptr, int n_sm,
                  Staged& T, cudaStream_t stream) {
  StagedLayout h = staged_layout(ptr, lev_ptr, n_sm);
  T.ok = h.ok;
  T.lev_b = std::move(h.lev_b);
  T.lev_nb = std::move(h.lev_nb);
  T.lev_ecap = std::move(h.lev_ecap);
  T.lev_rcap = std::move(h.lev_rcap);
  T.lev_mean = std::move(h.lev_mean);
  T.ecap = h.ecap;
  T.rcap = h.rcap;
  if (T.ok) T.desc.upload(h.desc.data(), h.desc.size(), stream);
}

// Upload of the packed copy of one sweep (layouts.h; split 0, +1 forward or
// -1 backward); values are filled from the factor after factorisation.
void build_packed(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                  const std::vector<int32_t>& lev_ptr, int n_sm, Packed& T, cudaStream_t stream,
                  int split = 0) {
  PackedLayout h = packed_layout(ptr, col, lev_ptr, n_sm, split);
  T.ok = h.ok;
  T.lev_b = std::move(h.lev_b);
  T.lev_nb = std::move(h.lev_nb);
  T.lev_mean = std::move(h.lev_mean);
  T.cap = h.cap;
  T.rcap = h.rcap;
  if (!T.ok) return;
  T.desc.upload(h.desc.data(), h.desc.size(), stream);
  Sell& S = T.data;
  S.slots = (int64_t)h.col.size();
  S.col.upload(h.col.data(), std::max<size_t>(1, h.col.size()), stream);
  S.src.upload(h.src.data(), std::max<size_t>(1, h.src.size()), stream);
  S.val.alloc(std::max<int64_t>(1, S.slots));
  S.val32.alloc(std::max<int64_t>(1, S.slots));
}

}  // namespace

void setup_pattern(Ctx& c, const gb_problem& prob) {
  if (prob.dim != 2 && prob.dim != 3) fail(GB_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (prob.p < 2 || prob.p > 6) fail(GB_ERR_INVALID_ARG, "p must be in [2, 6]");
  if (prob.N < 1 || prob.N > 100000) fail(GB_ERR_INVALID_ARG, "N out of range");
  if (prob.ordering < 0 || prob.ordering > 2) fail(GB_ERR_INVALID_ARG, "unknown ordering");
  c.prob = prob;
  c.dim = prob.dim;
  c.N = prob.N;
  c.p = prob.p;
  const Numbering nb = make_numbering(prob.dim, prob.N, prob.p);
  c.n_u = nb.n_u;
  c.n_p = nb.n_p;
  if (nb.n_u >= INT32_MAX || nb.n_p >= INT32_MAX) fail(GB_ERR_INVALID_ARG, "too many unknowns");
  const int64_t n = nb.n_u;

  // ---- ordering
  c.ncolours = 0;
  if (prob.ordering == GB_ORDER_NATURAL) {
    c.perm.resize(n);
    std::iota(c.perm.begin(), c.perm.end(), 0);
  } else if (prob.ordering == GB_ORDER_RCM) {
    order_rcm(nb, c.perm);
  } else {
    c.ncolours = order_multicolour(nb, c.perm);
  }
  std::vector<int32_t> ipos(n);  // natural -> ordering position
  for (int64_t i = 0; i < n; ++i) ipos[c.perm[i]] = (int32_t)i;

  // ---- level sets of the factor's DAG (ordering numbering):
  // level(i) = 1 + max level(k) over lower neighbours k < i (0 without any),
  // rlevel the same over upper neighbours, processed from the last row.
  c.level.assign(n, 0);
  c.rlevel.assign(n, 0);
  int maxlev = 0, maxrlev = 0;
  for (int64_t i = 0; i < n; ++i) {
    int lv = -1;
    nb.vel_neighbours(c.perm[i], [&](int64_t v) {
      int32_t k = ipos[v];
      if (k < i) lv = std::max(lv, c.level[k]);
    });
    c.level[i] = lv + 1;
    maxlev = std::max(maxlev, lv + 1);
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    int lv = -1;
    nb.vel_neighbours(c.perm[i], [&](int64_t v) {
      int32_t k = ipos[v];
      if (k > i) lv = std::max(lv, c.rlevel[k]);
    });
    c.rlevel[i] = lv + 1;
    maxrlev = std::max(maxrlev, lv + 1);
  }
  c.nlev = maxlev + 1;
  c.nrlev = maxrlev + 1;

  // ---- internal numbering: ordering positions sorted by level (stable)
  c.lev_ptr.assign(c.nlev + 1, 0);
  for (int64_t i = 0; i < n; ++i) c.lev_ptr[c.level[i] + 1]++;
  for (int l = 0; l < c.nlev; ++l) c.lev_ptr[l + 1] += c.lev_ptr[l];
  c.int_to_pos.assign(n, 0);
  {
    std::vector<int32_t> fill(c.lev_ptr.begin(), c.lev_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) c.int_to_pos[fill[c.level[i]]++] = (int32_t)i;
  }
  c.order.resize(n);
  std::vector<int32_t> iorder(n);  // natural -> internal
  for (int64_t r = 0; r < n; ++r) {
    c.order[r] = c.perm[c.int_to_pos[r]];
    iorder[c.order[r]] = (int32_t)r;
  }

  // ---- A pattern in internal numbering
  std::vector<int64_t> rowlen(n);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) rowlen[r] = nb.vel_degree(c.order[r]);
  });
  std::vector<int64_t> ptr64(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) ptr64[r + 1] = ptr64[r] + rowlen[r];
  if (ptr64[n] >= INT32_MAX) fail(GB_ERR_INVALID_ARG, "nnz(A) exceeds 32-bit indexing");
  c.nnzA = ptr64[n];
  c.hA_ptr.assign(n + 1, 0);
  for (int64_t r = 0; r <= n; ++r) c.hA_ptr[r] = (int32_t)ptr64[r];
  c.hA_col.resize(c.nnzA);
  std::vector<int32_t> hdiag(n);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) {
      int32_t* out = c.hA_col.data() + c.hA_ptr[r];
      int64_t t = 0;
      nb.vel_neighbours(c.order[r], [&](int64_t v) { out[t++] = iorder[v]; });
      std::sort(out, out + t);
      hdiag[r] = (int32_t)(std::lower_bound(out, out + t, (int32_t)r) - c.hA_col.data());
    }
  });

  // ---- L (strict lower = prefix of each A row) and U = L^T (strict upper)
  std::vector<int32_t> Lptr(n + 1, 0), Uptr(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) {
    Lptr[r + 1] = Lptr[r] + (hdiag[r] - c.hA_ptr[r]);
    Uptr[r + 1] = Uptr[r] + (c.hA_ptr[r + 1] - hdiag[r] - 1);
  }
  c.nnzL = Lptr[n] + n;
  std::vector<int32_t> Lcol(Lptr[n]), Ucol(Uptr[n]), Umap(Uptr[n]);
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) {
      std::copy(c.hA_col.begin() + c.hA_ptr[r], c.hA_col.begin() + hdiag[r], Lcol.begin() + Lptr[r]);
      int32_t t = Uptr[r];
      for (int32_t s = hdiag[r] + 1; s < c.hA_ptr[r + 1]; ++s, ++t) {
        int32_t j = c.hA_col[s];  // j > r: entry L(j, r) lives in row j's prefix
        const int32_t* b = c.hA_col.data() + c.hA_ptr[j];
        const int32_t* e = c.hA_col.data() + hdiag[j];
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
  if (Bptr64[np] >= INT32_MAX) fail(GB_ERR_INVALID_ARG, "nnz(B) exceeds 32-bit indexing");
  c.nnzB = Bptr64[np];
  c.hB_ptr.assign(np + 1, 0);
  for (int64_t k = 0; k <= np; ++k) c.hB_ptr[k] = (int32_t)Bptr64[k];
  c.hB_col.resize(c.nnzB);
  parallel_ranges(np, [&](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k) {
      int32_t* out = c.hB_col.data() + c.hB_ptr[k];
      int64_t t = 0;
      nb.pres_row(k, [&](int64_t v) { out[t++] = iorder[v]; });
      std::sort(out, out + t);
    }
  });
  // transpose (counting), rows internal velocity, cols ascending pressure
  std::vector<int32_t> Btptr(n + 1, 0), Btcol(c.nnzB), Btmap(c.nnzB);
  for (int64_t t = 0; t < c.nnzB; ++t) Btptr[c.hB_col[t] + 1]++;
  for (int64_t r = 0; r < n; ++r) Btptr[r + 1] += Btptr[r];
  {
    std::vector<int32_t> fill(Btptr.begin(), Btptr.end() - 1);
    for (int64_t k = 0; k < np; ++k)
      for (int32_t t = c.hB_ptr[k]; t < c.hB_ptr[k + 1]; ++t) {
        int32_t r = c.hB_col[t];
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
    c.nnzQ = 1;
    for (int k = 0; k < nb.dim; ++k) c.nnzQ *= per;
  }
  // pattern of Q (natural pressure numbering, ascending columns): pressure
  // functions k and l couple iff |a_d - b_d| <= p - 1 in every direction
  if (c.nnzQ >= INT32_MAX) fail(GB_ERR_INVALID_ARG, "Q exceeds 32-bit indexing");
  std::vector<int32_t> Qptr(np + 1, 0), Qcol(c.nnzQ);
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

  // ---- upload
  cudaStream_t s = c.stream;
  c.order_d.upload(c.order.data(), n, s);
  c.iorder_d.upload(iorder.data(), n, s);
  c.pos_d.upload(c.int_to_pos.data(), n, s);
  c.A_ptr.upload(c.hA_ptr.data(), n + 1, s);
  c.A_col.upload(c.hA_col.data(), c.nnzA, s);
  c.A_diag.upload(hdiag.data(), n, s);
  c.A_val.alloc(c.nnzA);
  c.A_val32.alloc(c.nnzA);
  c.L_ptr.upload(Lptr.data(), n + 1, s);
  c.L_col.upload(Lcol.data(), Lcol.size(), s);
  c.L_val.alloc(std::max<size_t>(1, Lcol.size()));
  c.L_val32.alloc(std::max<size_t>(1, Lcol.size()));
  c.L_diag.alloc(n);
  c.L_inv.alloc(n);
  c.L_inv32.alloc(n);
  c.U_ptr.upload(Uptr.data(), n + 1, s);
  c.U_col.upload(Ucol.data(), Ucol.size(), s);
  c.U_map.upload(Umap.data(), Umap.size(), s);
  c.U_val.alloc(std::max<size_t>(1, Ucol.size()));
  c.U_val32.alloc(std::max<size_t>(1, Ucol.size()));
  c.B_ptr.upload(c.hB_ptr.data(), np + 1, s);
  c.B_col.upload(c.hB_col.data(), c.nnzB, s);
  c.B_val.alloc(c.nnzB);
  c.Bt_ptr.upload(Btptr.data(), n + 1, s);
  c.Bt_col.upload(Btcol.data(), c.nnzB, s);
  c.Bt_map.upload(Btmap.data(), c.nnzB, s);
  c.Bt_val.alloc(c.nnzB);
  c.Qdiag.alloc(np);
  c.wmean.alloc(np);
  c.Q_ptr.upload(Qptr.data(), np + 1, s);
  c.Q_col.upload(Qcol.data(), c.nnzQ, s);
  c.Q_val.alloc(c.nnzQ);
  c.Q_val32.alloc(c.nnzQ);
  {
    const size_t band = (size_t)(nb.N + nb.p - 1) * nb.p;
    c.q1.alloc(band);
    c.l1.alloc(band);
    c.l1_32.alloc(band);
  }
  build_sell(c.hA_ptr, c.hA_col, c.lev_ptr, c.lev_slice, c.sA, s);
  build_sell(Lptr, Lcol, c.lev_ptr, c.lev_slice, c.sL, s);
  build_sell(Uptr, Ucol, c.lev_ptr, c.lev_slice, c.sU, s);
  {
    int dev = 0;
    GBS_CUDA(cudaGetDevice(&dev));
    GBS_CUDA(cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  build_staged(Lptr, c.lev_ptr, c.n_sm, c.tL, s);
  build_staged(Uptr, c.lev_ptr, c.n_sm, c.tU, s);
  build_packed(Lptr, Lcol, c.lev_ptr, c.n_sm, c.pL, s);
  build_packed(Uptr, Ucol, c.lev_ptr, c.n_sm, c.pU, s);
  build_packed(Lptr, Lcol, c.lev_ptr, c.n_sm, c.qL, s, +1);
  build_packed(Uptr, Ucol, c.lev_ptr, c.n_sm, c.qU, s, -1);
  c.max_lrow = 0;
  for (int64_t r = 0; r < n; ++r)
    c.max_lrow = std::max({c.max_lrow, Lptr[r + 1] - Lptr[r], Uptr[r + 1] - Uptr[r]});
  c.status_d.alloc(16);
  c.status_d.zero(s);
  GBS_CUDA(cudaStreamSynchronize(s));
}

namespace {
template <class T>
size_t bytes_of(const DevBuf<T>& b) {
  return b.p ? b.n * sizeof(T) : 0;
}
size_t bytes_of(const Sell& s) {
  return bytes_of(s.off) + bytes_of(s.row0) + bytes_of(s.rowlen) + bytes_of(s.col) + bytes_of(s.src) +
         bytes_of(s.val) + bytes_of(s.val32);
}
size_t bytes_of(const Packed& p) { return bytes_of(p.data) + bytes_of(p.desc); }
}  // namespace

bool trsv_available(const Ctx& c, int v) {
  if (v >= 2 && v <= 4) return c.tL.ok && c.tU.ok;
  if (v >= 5 && v <= 6) return c.pL.ok && c.pU.ok;
  if (v >= 7 && v <= 8) return c.qL.ok && c.qU.ok;
  return true;
}

size_t held_bytes(const Ctx& c) {
  size_t b = bytes_of(c.order_d) + bytes_of(c.iorder_d) + bytes_of(c.pos_d);
  b += bytes_of(c.A_ptr) + bytes_of(c.A_col) + bytes_of(c.A_diag) + bytes_of(c.A_val) + bytes_of(c.A_val32);
  b += bytes_of(c.L_ptr) + bytes_of(c.L_col) + bytes_of(c.L_val) + bytes_of(c.L_diag) + bytes_of(c.L_inv) +
       bytes_of(c.L_val32) + bytes_of(c.L_inv32);
  b += bytes_of(c.U_ptr) + bytes_of(c.U_col) + bytes_of(c.U_map) + bytes_of(c.U_val) + bytes_of(c.U_val32);
  b += bytes_of(c.B_ptr) + bytes_of(c.B_col) + bytes_of(c.Bt_ptr) + bytes_of(c.Bt_col) + bytes_of(c.Bt_map) +
       bytes_of(c.B_val) + bytes_of(c.Bt_val);
  b += bytes_of(c.Qdiag) + bytes_of(c.wmean) + bytes_of(c.tab1d);
  b += bytes_of(c.Q_ptr) + bytes_of(c.Q_col) + bytes_of(c.Q_val) + bytes_of(c.Q_val32) + bytes_of(c.q1) +
       bytes_of(c.l1) + bytes_of(c.l1_32);
  b += bytes_of(c.sA) + bytes_of(c.sL) + bytes_of(c.sU) + bytes_of(c.tL.desc) + bytes_of(c.tU.desc);
  b += bytes_of(c.pL) + bytes_of(c.pU) + bytes_of(c.qL) + bytes_of(c.qU) + bytes_of(c.status_d);
  return b;
}

}  // namespace gbs
