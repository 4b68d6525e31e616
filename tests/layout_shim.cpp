// Test-only C entry points around the host layout builders (layouts.h), so
// that the CPU tests can check the staged and packed layouts of the IC(0)
// sweeps without a GPU.  Compiled by tests/test_layouts.py with g++.
#include <cstring>
#include <vector>

#include "layouts.h"

namespace {
gbs::StagedLayout g_staged;
gbs::PackedLayout g_packed;

std::vector<int32_t> copy(const int32_t* p, int64_t n) { return std::vector<int32_t>(p, p + n); }
}  // namespace

extern "C" {

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
}
