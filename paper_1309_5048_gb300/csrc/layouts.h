// layouts.h -- host construction of the kernel layouts of the sparse
// operators: SELL-32 copies (inner SpMV and sweeps) and the block layouts of
// the IC(0) sweeps (Sec. 6.4, "PCG(A)": the forward and backward triangular
// solves of the IC(0) preconditioner, one launch per level of the factor's
// DAG).  Plain C++ without CUDA: setup uploads what these functions return.
//
// Input: a triangular factor as CSR over the internal numbering (rows sorted
// by level, so level l is the row range [lev_ptr[l], lev_ptr[l+1])), strict
// part only; the SM count sizes each level's grid.
#pragma once

#include <cstdint>
#include <vector>

namespace gbs {

// Blocks own at most kStagedRows rows of one level; the staged form holds at
// most kStagedEntries entries per block, the packed forms kPackedSlots padded
// slots.
constexpr int kStagedRows = 256;
constexpr int kStagedEntries = 2048;
constexpr int kPackedSlots = 2048;

// SELL-32 copy: rows cut into slices of 32 consecutive rows that never cross
// a level; slice s starts at row row0[s] (row0[nslices] = end) and slot
// off[s] (off[nslices] = slots); entry k of the row in lane i sits at
// off[s] + 32 k + i, with col the column and src its CSR position (padding
// past rowlen: col 0, src -1, never read).  Level l owns slices
// [lev_slice[l], lev_slice[l+1]).  ok is false (the rest empty) when the copy
// would exceed 32-bit slot indices.
struct SellLayout {
  bool ok = true;
  int nslices = 0;
  int64_t slots = 0;
  std::vector<int32_t> row0, off, rowlen, col, src, lev_slice;
};
SellLayout sell_layout(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                       const std::vector<int32_t>& lev_ptr);

// Staged partition: block b is desc[4b .. 4b+3] = {first row, end row, first
// entry, end entry} (CSR positions); level l owns blocks lev_b[l] ..
// lev_b[l] + lev_nb[l] - 1.  A level gets about max(entries / kStagedEntries,
// rows / kStagedRows) blocks, raised to the SM count (or a multiple of it),
// and rows are cut greedily at equal shares of entries + 4 per row.  ok is
// false (and everything else empty) when a row has more than kStagedEntries
// entries.
struct StagedLayout {
  bool ok = true;
  std::vector<int32_t> desc;
  std::vector<int32_t> lev_b, lev_nb;
  std::vector<int32_t> lev_ecap, lev_rcap;  // largest block of the level (entries, rows)
  std::vector<float> lev_mean;             // mean entries per row of the level
  int ecap = 0, rcap = 0;                  // over all levels
};
StagedLayout staged_layout(const std::vector<int32_t>& ptr, const std::vector<int32_t>& lev_ptr, int n_sm);

// Packed k-major copy: blocks cut as in staged_layout with the padded size
// rows * (longest row) as the cap; slot off + k * rows + i holds the k-th
// entry of the block's row i (col -1 and src -1 past the row's end); src maps
// slots to CSR positions.  desc[4b .. 4b+3] = {first row, rows, first slot,
// lo + (lr << 16)}.  With split = 0 every entry is in the first segment
// (lr = 0).  With split = +1 (forward sweep) or -1 (backward sweep) the
// entries whose column lies in level l - split, the level swept just before,
// form a second k-major segment of rows * lr slots after the first rows * lo,
// and lev_mean counts the first segment only.  ok is false (and everything
// else empty) when a row has more than kPackedSlots entries or the copy would
// exceed 32-bit slot indices.
struct PackedLayout {
  bool ok = true;
  std::vector<int32_t> desc, col, src;
  std::vector<int32_t> lev_b, lev_nb;
  std::vector<float> lev_mean;
  int cap = 0, rcap = 0;  // largest block (slots, rows)
};
PackedLayout packed_layout(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                           const std::vector<int32_t>& lev_ptr, int n_sm, int split);

}  // namespace gbs
