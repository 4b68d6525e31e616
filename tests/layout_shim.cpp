// Test-only C entry points around the host builders of the library: the
// sparsity patterns, ordering and level sets (pattern.h), the SELL-32 copies
// and the staged and packed layouts of the IC(0) sweeps (layouts.h), so that
// the CPU tests can
// check them without a GPU.  Compiled by tests/test_layouts.py and
// tests/test_pattern.py with g++.
#include <cstring>
#include <vector>

#include "layouts.h"
#include "pattern.h"

namespace {
gbs::StagedLayout g_staged;
gbs::PackedLayout g_packed;
gbs::HostPattern g_pattern;
gbs::SellLayout g_sell;

std::vector<int32_t> copy(const int32_t* p, int64_t n) { return std::vector<int32_t>(p, p + n); }
}  // namespace

extern "C" {

// SELL-32 copy; sizes[0..2] = ok, slices, slots.
void lt_sell(const int32_t* ptr, const int32_t* col, int32_t n, const int32_t* lev_ptr, int32_t nlev,
             int64_t* sizes) {
  std::vector<int32_t> p = copy(ptr, n + 1);
  g_sell = gbs::sell_layout(p, copy(col, p[n]), copy(lev_ptr, nlev + 1));
  sizes[0] = g_sell.ok;
  sizes[1] = g_sell.nslices;
  sizes[2] = g_sell.slots;
}

void lt_sell_fetch(int32_t* row0, int32_t* off, int32_t* rowlen, int32_t* col, int32_t* src, int32_t* lev_slice) {
  std::memcpy(row0, g_sell.row0.data(), g_sell.row0.size() * 4);
  std::memcpy(off, g_sell.off.data(), g_sell.off.size() * 4);
  std::memcpy(rowlen, g_sell.rowlen.data(), g_sell.rowlen.size() * 4);
  std::memcpy(col, g_sell.col.data(), g_sell.col.size() * 4);
  std::memcpy(src, g_sell.src.data(), g_sell.src.size() * 4);
  std::memcpy(lev_slice, g_sell.lev_slice.data(), g_sell.lev_slice.size() * 4);
}

// Builds the layout; sizes[0..2] = ok, blocks, slots (slots: packed only).
void lt_staged(const int32_t* ptr, int32_t n, const int32_t* lev_ptr, int32_t nlev, int32_t n_sm,
               int64_t* sizes) {
  g_staged = gbs::staged_layout(copy(ptr, n + 1), copy(lev_ptr, nlev + 1), n_sm);
  sizes[0] = g_staged.ok;
  sizes[1] = (int64_t)g_staged.desc.size() / 4;
  sizes[2] = 0;
}

void lt_staged_fetch(int32_t* desc, int32_t* lev_b, int32_t* lev_nb, int32_t* caps) {
  std::memcpy(desc, g_staged.desc.data(), g_staged.desc.size() * 4);
  std::memcpy(lev_b, g_staged.lev_b.data(), g_staged.lev_b.size() * 4);
  std::memcpy(lev_nb, g_staged.lev_nb.data(), g_staged.lev_nb.size() * 4);
  caps[0] = g_staged.ecap;
  caps[1] = g_staged.rcap;
}

void lt_packed(const int32_t* ptr, const int32_t* col, int32_t n, const int32_t* lev_ptr, int32_t nlev,
               int32_t n_sm, int32_t split, int64_t* sizes) {
  std::vector<int32_t> p = copy(ptr, n + 1);
  g_packed = gbs::packed_layout(p, copy(col, p[n]), copy(lev_ptr, nlev + 1), n_sm, split);
  sizes[0] = g_packed.ok;
  sizes[1] = (int64_t)g_packed.desc.size() / 4;
  sizes[2] = (int64_t)g_packed.col.size();
}

void lt_packed_fetch(int32_t* desc, int32_t* col, int32_t* src, int32_t* lev_b, int32_t* lev_nb,
                     float* lev_mean, int32_t* caps) {
  std::memcpy(desc, g_packed.desc.data(), g_packed.desc.size() * 4);
  std::memcpy(col, g_packed.col.data(), g_packed.col.size() * 4);
  std::memcpy(src, g_packed.src.data(), g_packed.src.size() * 4);
  std::memcpy(lev_b, g_packed.lev_b.data(), g_packed.lev_b.size() * 4);
  std::memcpy(lev_nb, g_packed.lev_nb.data(), g_packed.lev_nb.size() * 4);
  std::memcpy(lev_mean, g_packed.lev_mean.data(), g_packed.lev_mean.size() * 4);
  caps[0] = g_packed.cap;
  caps[1] = g_packed.rcap;
}

// Builds the pattern; returns 0, or 1 with the message in msg (size cap).
int lt_pattern(int32_t dim, int32_t N, int32_t p, int32_t ordering, int64_t* sizes, char* msg, int32_t cap) {
  try {
    g_pattern = gbs::build_pattern(dim, N, p, ordering);
  } catch (const gbs::PatternError& e) {
    std::strncpy(msg, e.what(), cap - 1);
    msg[cap - 1] = 0;
    return 1;
  }
  const gbs::HostPattern& P = g_pattern;
  const int64_t v[] = {P.n_u, P.n_p, P.nlev, P.nrlev, P.ncolours, P.nnzA, P.nnzL, P.nnzB, P.nnzQ,
                       (int64_t)P.L_col.size(), (int64_t)P.U_col.size()};
  std::memcpy(sizes, v, sizeof(v));
  return 0;
}

// Copies one array of the last pattern: 0 perm, 1 level, 2 rlevel, 3 lev_ptr,
// 4 int_to_pos, 5 order, 6 iorder, 7 A ptr, 8 A col, 9 A diag, 10 L ptr,
// 11 L col, 12 U ptr, 13 U col, 14 U map, 15 B ptr, 16 B col, 17 Bt ptr,
// 18 Bt col, 19 Bt map, 20 Q ptr, 21 Q col.  Returns its length.
int64_t lt_pattern_array(int32_t which, int32_t* out) {
  const gbs::HostPattern& P = g_pattern;
  const std::vector<int32_t>* a[] = {&P.perm,   &P.level,  &P.rlevel, &P.lev_ptr, &P.int_to_pos, &P.order,
                                     &P.iorder, &P.hA_ptr, &P.hA_col, &P.A_diag,  &P.L_ptr,      &P.L_col,
                                     &P.U_ptr,  &P.U_col,  &P.U_map,  &P.hB_ptr,  &P.hB_col,     &P.Bt_ptr,
                                     &P.Bt_col, &P.Bt_map, &P.Q_ptr,  &P.Q_col};
  if (which < 0 || which >= (int32_t)(sizeof(a) / sizeof(a[0]))) return -1;
  if (out) std::memcpy(out, a[which]->data(), a[which]->size() * 4);
  return (int64_t)a[which]->size();
}
}
