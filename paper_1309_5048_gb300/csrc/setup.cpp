// setup.cpp -- device upload of the discrete spaces, sparsity patterns,
// ordering, IC(0) level sets and internal numbering (built on the host by
// pattern.cpp) and of the kernel layouts (SELL-32 here; staged and packed
// built by layouts.cpp).
#include <algorithm>
#include <cstring>

#include "gbs_internal.h"
#include "pattern.h"

namespace gbs {

namespace {

// Upload of the SELL-32 copy of a CSR pattern (layouts.h); lev_slice
// receives the slice range of every level.
void build_sell(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                const std::vector<int32_t>& lev_ptr, std::vector<int32_t>& lev_slice, Sell& S,
                cudaStream_t stream) {
  SellLayout h = sell_layout(ptr, col, lev_ptr);
  if (!h.ok) fail(GB_ERR_INVALID_ARG, "SELL copy exceeds 32-bit indexing");
  lev_slice = std::move(h.lev_slice);
  S.nslices = h.nslices;
  S.slots = h.slots;
  S.row0.upload(h.row0.data(), h.row0.size(), stream);
  S.off.upload(h.off.data(), h.off.size(), stream);
  S.rowlen.upload(h.rowlen.data(), h.rowlen.size(), stream);
  S.col.upload(h.col.data(), h.col.size(), stream);  // empty: one slot, no copy
  S.src.upload(h.src.data(), h.src.size(), stream);
  S.val.alloc(std::max<int64_t>(1, h.slots));
  S.val32.alloc(std::max<int64_t>(1, h.slots));
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
  S.col.upload(h.col.data(), h.col.size(), stream);  // empty: one slot, no copy
  S.src.upload(h.src.data(), h.src.size(), stream);
  S.val.alloc(std::max<int64_t>(1, S.slots));
  S.val32.alloc(std::max<int64_t>(1, S.slots));
}

}  // namespace

void setup_pattern(Ctx& c, const gb_problem& prob) {
  HostPattern P;
  try {
    P = build_pattern(prob.dim, prob.N, prob.p, prob.ordering);
  } catch (const PatternError& e) {
    fail(GB_ERR_INVALID_ARG, e.what());
  }
  c.prob = prob;
  c.dim = P.dim;
  c.N = P.N;
  c.p = P.p;
  c.n_u = P.n_u;
  c.n_p = P.n_p;
  c.ncolours = P.ncolours;
  c.nlev = P.nlev;
  c.nrlev = P.nrlev;
  c.nnzA = P.nnzA;
  c.nnzL = P.nnzL;
  c.nnzB = P.nnzB;
  c.nnzQ = P.nnzQ;
  c.perm = std::move(P.perm);
  c.level = std::move(P.level);
  c.rlevel = std::move(P.rlevel);
  c.lev_ptr = std::move(P.lev_ptr);
  c.int_to_pos = std::move(P.int_to_pos);
  c.order = std::move(P.order);
  c.hA_ptr = std::move(P.hA_ptr);
  c.hA_col = std::move(P.hA_col);
  c.hB_ptr = std::move(P.hB_ptr);
  c.hB_col = std::move(P.hB_col);
  const int64_t n = c.n_u, np = c.n_p;
  const std::vector<int32_t>& iorder = P.iorder;
  const std::vector<int32_t>& hdiag = P.A_diag;
  const std::vector<int32_t>& Lptr = P.L_ptr;
  const std::vector<int32_t>& Lcol = P.L_col;
  const std::vector<int32_t>& Uptr = P.U_ptr;
  const std::vector<int32_t>& Ucol = P.U_col;
  const std::vector<int32_t>& Umap = P.U_map;
  const std::vector<int32_t>& Btptr = P.Bt_ptr;
  const std::vector<int32_t>& Btcol = P.Bt_col;
  const std::vector<int32_t>& Btmap = P.Bt_map;
  const std::vector<int32_t>& Qptr = P.Q_ptr;
  const std::vector<int32_t>& Qcol = P.Q_col;

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
    const size_t band = (size_t)(c.N + c.p - 1) * c.p;
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
  c.lev_maxL.assign(c.nlev, 0);
  c.lev_maxU.assign(c.nlev, 0);
  for (int l = 0; l < c.nlev; ++l)
    for (int32_t r = c.lev_ptr[l]; r < c.lev_ptr[l + 1]; ++r) {
      c.lev_maxL[l] = std::max(c.lev_maxL[l], Lptr[r + 1] - Lptr[r]);
      c.lev_maxU[l] = std::max(c.lev_maxU[l], Uptr[r + 1] - Uptr[r]);
    }
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
  if (v == 10) return c.max_lrow <= 8 * kTmaPF;
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
