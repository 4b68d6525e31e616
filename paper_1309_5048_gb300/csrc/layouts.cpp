// layouts.cpp -- host construction of the SELL-32 copies and of the staged
// and packed block layouts of the IC(0) sweeps (layouts.h).  No CUDA: setup
// uploads the results.
#include "layouts.h"

#include <algorithm>
#include <climits>

namespace gbs {

namespace {

// Blocks for a level of R rows and E entries: enough for the caps, raised to
// the SM count, or rounded up to a multiple of it past one wave.
int64_t level_blocks(int64_t R, int64_t E, int64_t per_block, int n_sm) {
  int64_t nb = std::max<int64_t>((E + per_block - 1) / per_block, (R + kStagedRows - 1) / kStagedRows);
  return nb <= n_sm ? std::min<int64_t>(R, n_sm) : (nb + n_sm - 1) / n_sm * n_sm;
}

bool rows_fit(const std::vector<int32_t>& ptr, const std::vector<int32_t>& lev_ptr, int64_t limit) {
  const int nlev = (int)lev_ptr.size() - 1;
  for (int32_t r = lev_ptr[0]; r < lev_ptr[nlev]; ++r)
    if (ptr[r + 1] - ptr[r] > limit) return false;
  return true;
}

}  // namespace

SellLayout sell_layout(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                       const std::vector<int32_t>& lev_ptr) {
  SellLayout S;
  const int nlev = (int)lev_ptr.size() - 1;
  S.lev_slice.assign(nlev + 1, 0);
  int64_t slots = 0;
  for (int l = 0; l < nlev; ++l) {
    S.lev_slice[l] = (int32_t)S.row0.size();
    for (int32_t r = lev_ptr[l]; r < lev_ptr[l + 1]; r += 32) {
      const int32_t r1 = std::min(r + 32, lev_ptr[l + 1]);
      int32_t len = 0;
      for (int32_t q = r; q < r1; ++q) len = std::max(len, ptr[q + 1] - ptr[q]);
      S.row0.push_back(r);
      S.off.push_back((int32_t)std::min<int64_t>(slots, INT_MAX));
      slots += (int64_t)32 * len;
    }
  }
  S.lev_slice[nlev] = (int32_t)S.row0.size();
  if (slots >= INT_MAX) return SellLayout{false};
  S.nslices = (int)S.row0.size();
  S.row0.push_back(lev_ptr[nlev]);
  S.off.push_back((int32_t)slots);
  S.slots = slots;
  S.rowlen.assign(ptr.size() - 1, 0);
  S.col.assign(slots, 0);
  S.src.assign(slots, -1);
  for (int s = 0; s < S.nslices; ++s)
    for (int32_t q = S.row0[s]; q < S.row0[s + 1]; ++q) {
      const int lane = q - S.row0[s];
      S.rowlen[q] = ptr[q + 1] - ptr[q];
      for (int32_t k = 0; k < S.rowlen[q]; ++k) {
        const int64_t slot = S.off[s] + (int64_t)32 * k + lane;
        S.col[slot] = col[ptr[q] + k];
        S.src[slot] = ptr[q] + k;
      }
    }
  return S;
}

StagedLayout staged_layout(const std::vector<int32_t>& ptr, const std::vector<int32_t>& lev_ptr, int n_sm) {
  StagedLayout T;
  const int nlev = (int)lev_ptr.size() - 1;
  if (!rows_fit(ptr, lev_ptr, kStagedEntries)) {
    T.ok = false;
    return T;
  }
  T.lev_b.assign(nlev, 0);
  T.lev_nb.assign(nlev, 0);
  T.lev_ecap.assign(nlev, 0);
  T.lev_rcap.assign(nlev, 0);
  T.lev_mean.assign(nlev, 0.f);
  std::vector<int32_t> brow;
  for (int l = 0; l < nlev; ++l) {
    const int32_t r0 = lev_ptr[l], r1 = lev_ptr[l + 1];
    const int64_t R = r1 - r0, E = (int64_t)ptr[r1] - ptr[r0];
    const int64_t nb = level_blocks(R, E, kStagedEntries, n_sm);
    const double share = (double)(E + 4 * R) / (double)std::max<int64_t>(1, nb);
    T.lev_b[l] = (int32_t)(T.desc.size() / 4);
    T.lev_mean[l] = R ? (float)((double)E / (double)R) : 0.f;
    brow.assign(1, r0);
    int64_t acc = 0, ent = 0, rows = 0, cuts = 0;
    for (int32_t r = r0; r < r1; ++r) {
      const int64_t len = ptr[r + 1] - ptr[r];
      const bool full = ent + len > kStagedEntries || rows == kStagedRows;
      const bool due = rows > 0 && (double)(acc + len + 4) > share * (double)(cuts + 1);
      if (rows > 0 && (full || due)) {
        brow.push_back(r);
        T.lev_ecap[l] = std::max<int32_t>(T.lev_ecap[l], (int32_t)ent);
        T.lev_rcap[l] = std::max<int32_t>(T.lev_rcap[l], (int32_t)rows);
        ++cuts;
        ent = rows = 0;
      }
      acc += len + 4;
      ent += len;
      ++rows;
    }
    brow.push_back(r1);
    T.lev_ecap[l] = std::max<int32_t>(T.lev_ecap[l], (int32_t)ent);
    T.lev_rcap[l] = std::max<int32_t>(T.lev_rcap[l], (int32_t)rows);
    T.lev_nb[l] = (int32_t)(cuts + 1);
    T.ecap = std::max(T.ecap, T.lev_ecap[l]);
    T.rcap = std::max(T.rcap, T.lev_rcap[l]);
    for (size_t b = 0; b + 1 < brow.size(); ++b) {
      T.desc.push_back(brow[b]);
      T.desc.push_back(brow[b + 1]);
      T.desc.push_back(ptr[brow[b]]);
      T.desc.push_back(ptr[brow[b + 1]]);
    }
  }
  return T;
}

PackedLayout packed_layout(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                           const std::vector<int32_t>& lev_ptr, int n_sm, int split) {
  PackedLayout T;
  const int nlev = (int)lev_ptr.size() - 1;
  if (!rows_fit(ptr, lev_ptr, kPackedSlots)) {
    T.ok = false;
    return T;
  }
  std::vector<int32_t> lev_of;
  if (split) {
    lev_of.assign(lev_ptr[nlev], 0);
    for (int l = 0; l < nlev; ++l)
      for (int32_t r = lev_ptr[l]; r < lev_ptr[l + 1]; ++r) lev_of[r] = l;
  }
  T.lev_b.assign(nlev, 0);
  T.lev_nb.assign(nlev, 0);
  T.lev_mean.assign(nlev, 0.f);
  bool overflow = false;
  // entries of row r (in level l) in the second segment
  auto second = [&](int32_t r, int l) {
    int32_t m = 0;
    if (split)
      for (int32_t e = ptr[r]; e < ptr[r + 1]; ++e) m += lev_of[col[e]] == l - split;
    return m;
  };
  auto emit = [&](int l, int32_t rb, int32_t nr, int32_t lo, int32_t lr) {
    const int64_t off = (int64_t)T.col.size();
    const int64_t len = (int64_t)lo + lr;
    if (off + (int64_t)nr * len >= INT_MAX) {
      overflow = true;
      return;
    }
    T.desc.push_back(rb);
    T.desc.push_back(nr);
    T.desc.push_back((int32_t)off);
    T.desc.push_back(lo + (lr << 16));
    T.col.resize(off + (int64_t)nr * len, -1);
    T.src.resize(off + (int64_t)nr * len, -1);
    for (int32_t i = 0; i < nr; ++i) {
      int32_t ko = 0, kr = 0;
      for (int32_t e = ptr[rb + i]; e < ptr[rb + i + 1]; ++e) {
        const bool in_second = split && lev_of[col[e]] == l - split;
        const int64_t slot = in_second ? off + (int64_t)nr * lo + (int64_t)(kr++) * nr + i
                                       : off + (int64_t)(ko++) * nr + i;
        T.col[slot] = col[e];
        T.src[slot] = e;
      }
    }
    T.cap = std::max<int>(T.cap, (int)(nr * len));
    T.rcap = std::max(T.rcap, nr);
  };
  for (int l = 0; l < nlev && !overflow; ++l) {
    const int32_t r0 = lev_ptr[l], r1 = lev_ptr[l + 1];
    const int64_t R = r1 - r0, E = (int64_t)ptr[r1] - ptr[r0];
    const int64_t nb = level_blocks(R, E, kPackedSlots, n_sm);
    const double share = (double)(E + 4 * R) / (double)std::max<int64_t>(1, nb);
    T.lev_b[l] = (int32_t)(T.desc.size() / 4);
    int64_t first = 0;  // entries of the level in the first segment
    int32_t rb = r0, rows = 0, lo = 0, lr = 0, cuts = 0;
    int64_t acc = 0;
    for (int32_t r = r0; r < r1; ++r) {
      const int32_t len = ptr[r + 1] - ptr[r];
      const int32_t m = second(r, l);
      first += len - m;
      const bool full =
          (int64_t)(rows + 1) * (std::max(lo, len - m) + std::max(lr, m)) > kPackedSlots || rows == kStagedRows;
      const bool due = rows > 0 && (double)(acc + len + 4) > share * (double)(cuts + 1);
      if (rows > 0 && (full || due)) {
        emit(l, rb, rows, lo, lr);
        ++cuts;
        rb = r;
        rows = lo = lr = 0;
      }
      acc += len + 4;
      lo = std::max(lo, len - m);
      lr = std::max(lr, m);
      ++rows;
    }
    emit(l, rb, rows, lo, lr);
    T.lev_nb[l] = cuts + 1;
    T.lev_mean[l] = R ? (float)((double)first / (double)R) : 0.f;
  }
  if (overflow) {
    T = PackedLayout();
    T.ok = false;
  }
  return T;
}

}  // namespace gbs
