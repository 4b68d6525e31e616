// pattern.h -- host construction of the discrete spaces (Sec. 3.2), the
// sparsity patterns of A_h, B, B^T and Q, the velocity ordering, the level
// sets of the IC(0) factor's DAG (Sec. 6.4) and the internal numbering.
// Plain C++ without CUDA: setup uploads what build_pattern returns.
//
// Numberings: "natural" is component-major, then lexicographic with the last
// direction fastest; the ordering (natural, RCM or multicolour) gives each
// natural velocity index a position; "internal" sorts positions by level
// (stable), so every level is a contiguous range and the factor stays lower
// triangular.
#pragma once

#include <cstdint>
#include <stdexcept>
#include <vector>

namespace gbs {

// Invalid sizes or a pattern past 32-bit indexing.
struct PatternError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

struct HostPattern {
  int dim = 0, N = 0, p = 0;
  int64_t n_u = 0, n_p = 0;
  int ncolours = 0;        // colours of the multicolour ordering (0 otherwise)
  int nlev = 0, nrlev = 0;  // forward / backward levels
  std::vector<int32_t> perm;             // ordering position -> natural
  std::vector<int32_t> level, rlevel;    // by ordering position
  std::vector<int32_t> lev_ptr;          // level l = internal rows [lev_ptr[l], lev_ptr[l+1])
  std::vector<int32_t> int_to_pos;       // internal -> ordering position
  std::vector<int32_t> order, iorder;    // internal -> natural, natural -> internal
  int64_t nnzA = 0, nnzL = 0, nnzB = 0, nnzQ = 0;  // nnzL counts the diagonal
  std::vector<int32_t> hA_ptr, hA_col, A_diag;     // A (internal), position of each diagonal
  std::vector<int32_t> L_ptr, L_col;               // strict lower part (a prefix of each A row)
  std::vector<int32_t> U_ptr, U_col, U_map;        // strict upper = L^T; U_map: slot of L
  std::vector<int32_t> hB_ptr, hB_col;             // B: natural pressure rows, internal columns
  std::vector<int32_t> Bt_ptr, Bt_col, Bt_map;     // B^T; Bt_map: slot of B
  std::vector<int32_t> Q_ptr, Q_col;               // Q: natural pressure numbering
};

// ordering: 0 natural, 1 RCM, 2 multicolour.  Throws PatternError.
HostPattern build_pattern(int dim, int N, int p, int ordering);

}  // namespace gbs
