// gbs_internal.h -- private declarations of the gbstokes library.
//
// Device data layout
// ------------------
// Velocity unknowns are stored in an *internal* numbering: the rows of the
// chosen ordering (natural / RCM / multicolour) sorted by their level in the
// IC(0) factor's DAG (stable, so ties keep the ordering's order).  Sorting by
// level is a topological order of that DAG, so the IC(0) factor is unchanged
// (every coupled pair keeps its relative order) while each level becomes a
// contiguous row range.  Pressure unknowns keep the natural numbering.
//
//   A_h      CSR (int32 ptr/col, FP64 val, FP32 copy), rows/cols internal,
//            sorted columns; the strictly-lower part of row i is a prefix.
//   L        strict lower part of the IC(0) factor, CSR (internal numbering),
//            plus 1/L_ii; U = L^T strict upper part in CSR (row form of the
//            backward solve), values gathered from L through U_map.
//   B        CSR, rows = pressure (natural), cols = velocity (internal).
//   Bt       CSR of B^T, rows = velocity (internal), values from B via Bt_map.
//   vectors  [n][K] interleaved: entry (row, rhs) at row*K + rhs, K the padded
//            batch width (1, 8 or 32).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gbstokes.h"
#include "layouts.h"

namespace gbs {

// Error raised inside the library; converted to a status at the C boundary.
struct Error {
  int status;
  std::string msg;
};
[[noreturn]] void fail(int status, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define GBS_CUDA(call) ::gbs::cuda_check((call), #call)

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { free_(); }
  void alloc(size_t count);
  void free_();
  void upload(const T* host, size_t count, cudaStream_t s);
  void zero(cudaStream_t s);
};

// Per-RHS scalar state of the solver, structure of arrays [field][K].
enum ScalarField {
  // MINRES
  S_GAMMA, S_GAMMA_PREV, S_GAMMA1, S_ETA, S_C, S_C_PREV, S_S, S_S_PREV, S_DELTA,
  S_XCOEF, S_A1, S_A2, S_A3, S_BNORM, S_RELRES, S_OUTER_ACTIVE, S_OUTER_ITS, S_STATUS,
  // inner CG
  S_RHO, S_ALPHA, S_CG_BNORM, S_RNORM, S_CG_ITS, S_CG_ACTIVE, S_CG_TARGET,
  // statistics
  S_INNER_TOTAL, S_INNER_MAX, S_APPS, S_TRUE_RES, S_NONFINITE, S_PMEAN,
  // right-hand side whose pressure part violates 1^T g_p = 0
  S_INCONSISTENT,
  // pressure-block CG on Q (IC(0)-PCG pressure block)
  S_Q_RHO, S_Q_ALPHA, S_Q_BNORM, S_Q_RNORM, S_Q_ITS, S_Q_ACTIVE, S_Q_TARGET, S_Q_TOTAL, S_Q_MAX,
  S_NFIELDS
};

// Slots per lane and slice group of the TMA-staged SELL sweep: a level whose
// longest factor row exceeds 8 * kTmaPF has no group that fits a stage, so
// that layout is available only when every row of L and U is that short.
constexpr int kTmaPF = 11;

// SELL-32 copy of a CSR matrix (single right-hand-side kernels): rows are cut
// into slices of 32 consecutive rows that never cross a level of the IC(0)
// DAG; entry k of the row in lane i of slice s sits at off[s] + 32 k + i.
// rowlen[row] bounds each row (padding is never read); src maps every slot to
// the position of its value in the CSR value array (-1 for padding), so
// values are refilled after assembly / factorisation.
struct Sell {
  DevBuf<int32_t> off, row0, rowlen, col, src;
  DevBuf<double> val;
  DevBuf<float> val32;
  int64_t slots = 0;
  int nslices = 0;
};

// Block partition of the levels of one triangular sweep for the staged
// single-RHS kernels: every block owns a contiguous range of internal rows of
// one level, at most kStagedRows rows and kStagedEntries off-diagonal
// entries, and the blocks of a level are balanced by entries over a grid of
// (a multiple of) the SM count.  Block b of the sweep is described by
// desc[4b .. 4b+3] = {first row, end row, first entry, end entry} (CSR
// positions); level l owns blocks lev_b[l] ... lev_b[l] + lev_nb[l] - 1.
// A factor with a row of more than kStagedEntries off-diagonal entries (3D,
// velocity degree 5 or 6) gets no partition: ok is false and the staged
// layouts are unavailable for that problem.  Built by staged_layout
// (layouts.h, which holds the block caps).
struct Staged {
  bool ok = true;
  DevBuf<int32_t> desc;
  std::vector<int32_t> lev_b, lev_nb;
  std::vector<int32_t> lev_ecap, lev_rcap;  // largest block of the level (entries, rows)
  std::vector<float> lev_mean;             // mean off-diagonal entries per row
  int ecap = 0, rcap = 0;                  // over all levels
};

// Packed copy of the levels of one triangular sweep for the packed
// single-RHS kernels: the same kind of block partition as Staged (at most
// kStagedRows rows and kPackedSlots padded slots per block), but each block's
// entries are stored k-major -- slot k * rows + i holds the k-th entry of the
// block's row i (column -1 and value 0 past the row's end) -- so that a warp
// reading consecutive slots reads the same stencil entry of consecutive rows.
// desc[4b .. 4b+3] = {first row, rows, first slot, slots per row}; level l owns
// blocks lev_b[l] .. lev_b[l] + lev_nb[l] - 1.  data.src maps slots to CSR
// positions (-1 for padding) to refill values after factorisation.  The split
// copies (Ctx::qL, qU) put the entries whose column lies in the level swept
// just before in a second k-major segment of rows * lr slots after the first
// rows * lo; their desc.w is lo + (lr << 16) and lev_mean counts the first
// segment only.  As for Staged, a row longer than kPackedSlots (or a copy past
// 32-bit slot indices) leaves the copy empty with ok false.  Built by
// packed_layout (layouts.h).
struct Packed {
  bool ok = true;
  Sell data;  // col, src, val, val32, slots (off / row0 / rowlen unused)
  DevBuf<int32_t> desc;
  std::vector<int32_t> lev_b, lev_nb;
  std::vector<float> lev_mean;  // mean entries per row of the level
  int cap = 0, rcap = 0;        // largest block (slots, rows)
};

struct Workspace {
  int K = 0;          // padded batch width
  int k = 0;          // capacity (right-hand sides) of the staging buffers
  int last_k = 0;     // right-hand sides of the most recent solve (0: none)
  int precision = -1;
  size_t n = 0;       // n_u + n_p
  // MINRES (FP64): x, three Lanczos vectors, two z buffers, three w buffers, q
  double* x = nullptr;
  double* V[3] = {nullptr, nullptr, nullptr};
  double* Z[2] = {nullptr, nullptr};
  double* W[3] = {nullptr, nullptr, nullptr};
  double* q = nullptr;
  double* b = nullptr;  // right-hand side, internal layout
  double* R = nullptr;  // residual b - K x_j (2-norm stopping rule)
  double* lz = nullptr;  // Lanczos tridiagonal record [2][K][lz_cap]
  int lz_cap = 0;
  double* KW[3] = {nullptr, nullptr, nullptr};  // K w_j, rotating like W
  // inner CG, element type T (double or float) stored as raw bytes
  void* cg_x = nullptr;
  void* cg_r = nullptr;
  void* cg_z = nullptr;
  void* cg_y = nullptr;
  void* cg_p = nullptr;
  void* cg_q = nullptr;
  // pressure-block CG on Q (element type T, [n_p][K])
  void* qcg_x = nullptr;
  void* qcg_r = nullptr;
  void* qcg_z = nullptr;
  void* qcg_p = nullptr;
  void* qcg_q = nullptr;
  int32_t* forced_q = nullptr;  // device replay counts of the pressure CG
  int64_t nforced_q = 0;
  size_t forced_q_cap = 0;
  double* S = nullptr;          // scalars [S_NFIELDS][K]
  double* S_host = nullptr;     // pinned mirror
  int* flag = nullptr;          // device: [0] any outer active, [1] any inner active,
                                // [2] MINRES step j, [3] any pressure CG active
  int* flag_host = nullptr;     // pinned
  int32_t* forced = nullptr;    // device replay counts
  int64_t nforced = 0;
  size_t forced_cap = 0;
  double* partial = nullptr;    // reduction partials [blocks][K][<=4]
  unsigned* counter = nullptr;  // completion counter of the reduction kernels
  double* aux = nullptr;        // small scratch (adjoint coefficients, dnu partials)
  double* rhs_tmp = nullptr;    // adjoint right-hand side [k][n]
  double* host_in = nullptr;    // device staging for gb_solve_host
  double* host_out = nullptr;
  // CUDA graph of the whole solve (device-side loop control)
  cudaGraphExec_t graph = nullptr;
  std::vector<double> graph_key;
  bool graph_valid = false;
};

struct Ctx {
  gb_problem prob{};
  // All device work runs on `stream`, a non-blocking stream owned by the
  // context (graphs cannot be captured on the legacy default stream); every
  // API call orders it after the caller's stream on entry and the caller's
  // stream after it on exit, with events.
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int dim = 2, N = 1, p = 2;
  int64_t n_u = 0, n_p = 0, nnzA = 0, nnzB = 0, nnzL = 0, nnzQ = 0;
  int nlev = 0, nrlev = 0, ncolours = 0;
  // host copies
  std::vector<int32_t> order;    // internal -> natural velocity index
  std::vector<int32_t> perm;     // ordering position -> natural
  std::vector<int32_t> int_to_pos;  // internal -> ordering position
  std::vector<int32_t> level, rlevel;  // by ordering position
  std::vector<int32_t> lev_ptr;  // forward level l = internal rows [lev_ptr[l], lev_ptr[l+1])
  std::vector<int32_t> hA_ptr, hA_col;  // internal CSR pattern of A
  std::vector<int32_t> hB_ptr, hB_col;  // B pattern (cols internal)
  // device arrays
  DevBuf<int32_t> order_d, iorder_d, pos_d;  // pos_d: internal -> ordering position
  DevBuf<int32_t> A_ptr, A_col, A_diag;  // A_diag[i]: position of the diagonal
  DevBuf<double> A_val;
  DevBuf<float> A_val32;
  DevBuf<int32_t> L_ptr, L_col;
  DevBuf<double> L_val, L_diag, L_inv;
  DevBuf<float> L_val32, L_inv32;
  DevBuf<int32_t> U_ptr, U_col, U_map;
  DevBuf<double> U_val;
  DevBuf<float> U_val32;
  DevBuf<int32_t> B_ptr, B_col, Bt_ptr, Bt_col, Bt_map;
  DevBuf<double> B_val, Bt_val;
  DevBuf<double> Qdiag, wmean;
  DevBuf<double> tab1d;  // 1D integral tables (assembly)
  // Pressure mass matrix Q, natural numbering, for the IC(0)-PCG pressure
  // block.  Q is the Kronecker product of the 1D mass matrix Q1 of the
  // degree p-1 B-splines (m = N + p - 1 functions, half-bandwidth p - 1) over
  // the directions; in the natural (lexicographic) order the exact Cholesky
  // factor L1 x L1 [x L1] lies inside the lower pattern of Q, so IC(0) of Q
  // is that factor, kept as the band of L1: l1[a * p + o] = L1[a][a - o].
  DevBuf<int32_t> Q_ptr, Q_col;
  DevBuf<double> Q_val;
  DevBuf<float> Q_val32;
  DevBuf<double> q1;   // band of Q1, same layout as l1
  DevBuf<double> l1;
  DevBuf<float> l1_32;
  bool q_factored = false;
  Sell sA, sL, sU;                 // SELL-32 copies of A, L, U
  std::vector<int32_t> lev_slice;  // level l = slices [lev_slice[l], lev_slice[l+1])
  std::vector<int32_t> lev_maxL, lev_maxU;  // longest off-diagonal row of L, U in level l
  Staged tL, tU;                   // staged-sweep partitions of L and U = L^T
  Packed pL, pU;                   // packed (k-major) copies of L and U
  Packed qL, qU;                   // the same, each row split by the level of its columns
  int n_sm = 0;                    // streaming multiprocessors of the device
  // kernel layout per precision (index 0 FP64, 1 mixed) for single-RHS
  // solves: SpMV 0 CSR with 8 lanes per row, 1 SELL-32 one thread per row,
  // 2/3 SELL-32 with 2/4 warps per slice;
  // triangular sweeps 0 CSR, 1 SELL-32, 2/3/4 staged with about 4/12/32
  // entries per lane, 5/6 packed with about 12/32 entries per lane, 7/8 split
  // packed, 9 and 11-18 SELL-32 with W warps per slice (9: 12 slots loaded
  // before the dependency wait; 11-17 light forms; 18 the hybrid of 14 and
  // 9), 10 TMA-staged SELL-32; -1 not chosen yet (chosen at the first
  // single-RHS solve by autotune_single)
  int var_spmv[2] = {-1, -1}, var_trsv[2] = {-1, -1};
  // batched sweeps per precision and width (index 0: K = 8, 1: K = 32): 0 the
  // warp-per-row kernel, 1 the staged batched kernel, -1 not chosen yet
  int var_trsv_batch[2][2] = {{-1, -1}, {-1, -1}};
  int max_lrow = 0;  // longest off-diagonal row of L and U
  DevBuf<int> status_d;  // device error flags: [0] IC(0) breakdown row, [1] band Cholesky, [2] sweep wait timeout
  DevBuf<int32_t> tune_forced;  // replay counts of the in-graph layout tuning solve
  int tma_bps[2] = {0, 0};  // resident blocks per SM of the TMA sweep (FP64, FP32), 0: not yet known
  double nu = 1.0, cpen = 0.0;
  bool assembled = false, factored = false;
  Workspace ws;
};

// setup.cpp
void setup_pattern(Ctx& c, const gb_problem& prob);
// Device bytes of the context's operators, factors and kernel layouts.
size_t held_bytes(const Ctx& c);
// Whether single-RHS sweep layout v (gb_set_kernel_variants) exists for this
// problem: the staged (2-4), packed (5-6) and split packed (7-8) forms need
// every row of L and U to fit one block.
bool trsv_available(const Ctx& c, int v);
// assemble.cu
void assemble(Ctx& c, double nu, double cpen);
void load_fourier(Ctx& c, int nmodes, const int32_t* kappa, const double* amp, double* f_dev);
void load_manufactured(Ctx& c, double* f_dev);
void load_cavity(Ctx& c, double* f_dev);
// factor.cu
int64_t factor_ic0(Ctx& c);
void sell_refill(Ctx& c, Sell& S, const double* csr_val);
// solver.cu
int solve(Ctx& c, const double* rhs_dev, double* x_dev, int k, const gb_solve_opts& o,
          gb_info* info, bool adjoint);
int solve_host(Ctx& c, const double* rhs_host, double* x_host, int k, const gb_solve_opts& o,
               gb_info* info);
void apply_operator(Ctx& c, int which, const double* x, double* y);
double time_kernel(Ctx& c, int which, int reps);
void dnu(Ctx& c, const double* lam, const double* x, int k, double* out);
void dnu_noalloc(Ctx& c, const double* lam, const double* x, int k, double* out);
void release_workspace(Ctx& c);
int lanczos_coeffs(Ctx& c, int rhs, double* delta, double* gamma, int cap);
void ritz_extremes(Ctx& c, int rhs, int exclude_one, double* out);

// Velocity DOF decoding shared by host setup code.
struct Space {
  int dim, N, p;
  int64_t voff[4];
  int deg(int c, int k) const { return k == c ? p : p - 1; }
  int vlen(int c, int k) const { return k == c ? N + p - 2 : N + p - 1; }
  int plen() const { return N + p - 1; }
};

}  // namespace gbs
