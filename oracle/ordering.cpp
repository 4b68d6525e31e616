// ordering.cpp -- TEST INFRASTRUCTURE ONLY (see oracle.hpp).
// Orderings applied to A_h before IC(0) (Sec. 6.4 reorders A by reverse
// Cuthill-McKee) and the level sets of the triangular factor's DAG.
#include <algorithm>
#include <deque>
#include <stdexcept>

#include "oracle.hpp"

namespace oracle {

// Breadth-first level structure from root over the graph of A (diagonal
// ignored), restricted to nodes with alive[i] set.  Returns the eccentricity
// (number of levels - 1) and fills the last level.
static int bfs_levels(const Csr& A, int32_t root, const std::vector<char>& alive,
                      std::vector<int32_t>& last) {
  const int64_t n = A.nrows;
  std::vector<int32_t> dist(n, -1);
  std::deque<int32_t> q;
  dist[root] = 0;
  q.push_back(root);
  int ecc = 0;
  while (!q.empty()) {
    int32_t u = q.front();
    q.pop_front();
    ecc = std::max(ecc, dist[u]);
    for (int64_t t = A.ptr[u]; t < A.ptr[u + 1]; ++t) {
      int32_t v = A.col[t];
      if (v == u || !alive[v] || dist[v] >= 0) continue;
      dist[v] = dist[u] + 1;
      q.push_back(v);
    }
  }
  last.clear();
  for (int64_t i = 0; i < n; ++i)
    if (dist[i] == ecc) last.push_back((int32_t)i);
  return ecc;
}

// Reverse Cuthill-McKee.  Start node: George-Liu pseudo-peripheral node,
// searched from the alive node of minimum degree (ties: smallest index),
// moving to the minimum-degree node of the last BFS level while the
// eccentricity grows.  Cuthill-McKee visits unnumbered neighbours in order
// of increasing degree (ties: smallest index); the final order is reversed.
static void rcm(const Csr& A, std::vector<int32_t>& perm) {
  const int64_t n = A.nrows;
  std::vector<int32_t> deg(n);
  for (int64_t i = 0; i < n; ++i) {
    int d = 0;
    for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t)
      if (A.col[t] != i) ++d;
    deg[i] = d;
  }
  std::vector<char> alive(n, 1);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> last, nb;
  while ((int64_t)order.size() < n) {
    int32_t r = -1;
    for (int64_t i = 0; i < n; ++i)
      if (alive[i] && (r < 0 || deg[i] < deg[r])) r = (int32_t)i;
    int ecc = bfs_levels(A, r, alive, last);
    for (;;) {
      int32_t x = -1;
      for (int32_t v : last)
        if (x < 0 || deg[v] < deg[x] || (deg[v] == deg[x] && v < x)) x = v;
      std::vector<int32_t> last_x;
      int ecc_x = bfs_levels(A, x, alive, last_x);
      if (ecc_x > ecc) {
        r = x;
        ecc = ecc_x;
        last = last_x;
      } else {
        break;
      }
    }
    // Cuthill-McKee from r
    size_t head = order.size();
    order.push_back(r);
    alive[r] = 0;
    while (head < order.size()) {
      int32_t u = order[head++];
      nb.clear();
      for (int64_t t = A.ptr[u]; t < A.ptr[u + 1]; ++t) {
        int32_t v = A.col[t];
        if (alive[v]) nb.push_back(v);
      }
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      for (int32_t v : nb) {
        alive[v] = 0;
        order.push_back(v);
      }
    }
  }
  perm.assign(order.rbegin(), order.rend());
}

// Multicolour ordering: velocity DOF (c, l) gets colour
// (c, l_k mod m_k for each direction k) with m_k = deg(c,k)+1.  Two DOFs of
// one component couple in A only if |l_k - l'_k| <= deg(c,k) in every
// direction, so DOFs of one colour are mutually uncoupled.  Order: by colour,
// then by natural index.
int64_t velocity_colour(const Problem& P, int64_t i) {
  int c, a[3] = {0, 0, 0};
  P.vdecode(i, &c, a);
  int64_t col = c;
  for (int k = 0; k < P.dim; ++k) {
    int m = P.deg(c, k) + 1;
    int l = (k == c) ? a[k] - 1 : a[k];
    col = col * m + (l % m);
  }
  return col;
}

static void multicolour(const Problem& P, std::vector<int32_t>& perm) {
  const int64_t n = P.n_u;
  std::vector<int64_t> colour(n);
  for (int64_t i = 0; i < n; ++i) colour[i] = velocity_colour(P, i);
  perm.resize(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  std::stable_sort(perm.begin(), perm.end(),
                   [&](int32_t a, int32_t b) { return colour[a] < colour[b]; });
}

// Multicolour ordering of the pressure space: DOF (l_1..l_d) of degree p-1
// gets colour (l_k mod p for each direction k); two pressure DOFs couple in
// Q only if |l_k - l'_k| <= p-1 in every direction.
static void multicolour_pressure(const Problem& P, std::vector<int32_t>& perm) {
  const int64_t n = P.n_p;
  std::vector<int64_t> colour(n);
  for (int64_t i = 0; i < n; ++i) {
    int a[3] = {0, 0, 0};
    P.pdecode(i, a);
    int64_t col = 0;
    for (int k = 0; k < P.dim; ++k) col = col * P.p + (a[k] % P.p);
    colour[i] = col;
  }
  perm.resize(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  std::stable_sort(perm.begin(), perm.end(),
                   [&](int32_t a, int32_t b) { return colour[a] < colour[b]; });
}

void make_pressure_ordering(const Problem& P, int kind, std::vector<int32_t>& perm) {
  const int64_t n = P.n_p;
  if (kind == 0) {
    perm.resize(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  } else if (kind == 1) {
    rcm(P.Q, perm);
  } else if (kind == 2) {
    multicolour_pressure(P, perm);
  } else {
    throw std::runtime_error("unknown ordering");
  }
}

void make_ordering(const Problem& P, int kind, std::vector<int32_t>& perm) {
  const int64_t n = P.n_u;
  if (kind == 0) {
    perm.resize(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  } else if (kind == 1) {
    rcm(P.A, perm);
  } else if (kind == 2) {
    multicolour(P, perm);
  } else {
    throw std::runtime_error("unknown ordering");
  }
}

void lower_pattern(const Csr& A, const std::vector<int32_t>& perm, Csr& L) {
  const int64_t n = A.nrows;
  std::vector<int32_t> iperm(n);
  for (int64_t i = 0; i < n; ++i) iperm[perm[i]] = (int32_t)i;
  L.nrows = L.ncols = n;
  L.ptr.assign(n + 1, 0);
  std::vector<int32_t> row;
  std::vector<std::vector<int32_t>> rows(n);
  for (int64_t i = 0; i < n; ++i) {
    int32_t old = perm[i];
    row.clear();
    for (int64_t t = A.ptr[old]; t < A.ptr[old + 1]; ++t) {
      int32_t j = iperm[A.col[t]];
      if (j <= i) row.push_back(j);
    }
    std::sort(row.begin(), row.end());
    rows[i] = row;
    L.ptr[i + 1] = L.ptr[i] + (int64_t)row.size();
  }
  L.col.resize(L.ptr[n]);
  for (int64_t i = 0; i < n; ++i) std::copy(rows[i].begin(), rows[i].end(), L.col.begin() + L.ptr[i]);
  L.val.assign(L.ptr[n], 0.0);
}

void level_sets(const Csr& L, std::vector<int32_t>& level, std::vector<int32_t>& rlevel) {
  const int64_t n = L.nrows;
  level.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    int32_t lv = -1;
    for (int64_t t = L.ptr[i]; t < L.ptr[i + 1]; ++t)
      if (L.col[t] < i) lv = std::max(lv, level[L.col[t]]);
    level[i] = lv + 1;
  }
  // reverse DAG: row i of L^T holds the k > i with L_ki != 0
  std::vector<std::vector<int32_t>> up(n);
  for (int64_t k = 0; k < n; ++k)
    for (int64_t t = L.ptr[k]; t < L.ptr[k + 1]; ++t)
      if (L.col[t] < k) up[L.col[t]].push_back((int32_t)k);
  rlevel.assign(n, 0);
  for (int64_t i = n - 1; i >= 0; --i) {
    int32_t lv = -1;
    for (int32_t k : up[i]) lv = std::max(lv, rlevel[k]);
    rlevel[i] = lv + 1;
  }
}

}  // namespace oracle
