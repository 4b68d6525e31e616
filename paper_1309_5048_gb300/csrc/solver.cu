// solver.cu -- host driver of the preconditioned MINRES solve (Sec. 5).
//
// The kernel sequence of one solve (see solver_kernels.cuh) is
//   gather, z_1 = M^{-1} b (Lanczos j=0, inner CG), gamma_1,
//   repeat { K z_j, Lanczos, inner CG, Givens, w/x update } while any RHS live,
//   true residual, zero-mean filter and scatter.
// Loop control is on the device: the last block of the CG and MINRES step
// kernels decides whether any RHS is still active.  Two drivers run the same
// sequence: a host loop that reads that flag (one synchronisation per inner
// iteration), and a CUDA graph whose loops are WHILE conditional nodes set by
// those kernels (no host round trip during the solve).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <type_traits>
#include <vector>

#include "solver_kernels.cuh"

namespace gbs {

namespace {

void* dmalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(GB_ERR_OOM, "cudaMalloc failed for workspace");
  }
  return p;
}

// Allocates the solve workspace for batch width K and the precision's inner
// CG element size (called on an empty workspace).
void alloc_workspace(Ctx& c, int K, int precision, size_t n) {
  Workspace& w = c.ws;
  w.K = K;
  w.precision = precision;
  w.n = n;
  const size_t esz = precision == GB_PREC_MIXED ? 4 : 8;
  const size_t vb = n * K * sizeof(double), cb = (size_t)c.n_u * K * esz;
  w.x = (double*)dmalloc(vb);
  for (int i = 0; i < 3; ++i) w.V[i] = (double*)dmalloc(vb);
  for (int i = 0; i < 2; ++i) w.Z[i] = (double*)dmalloc(vb);
  for (int i = 0; i < 3; ++i) w.W[i] = (double*)dmalloc(vb);
  w.q = (double*)dmalloc(vb);
  w.b = (double*)dmalloc(vb);
  w.R = (double*)dmalloc(vb);
  for (int i = 0; i < 3; ++i) w.KW[i] = (double*)dmalloc(vb);
  w.cg_x = dmalloc(cb);
  w.cg_r = dmalloc(cb);
  w.cg_z = dmalloc(cb);
  w.cg_y = dmalloc(cb);
  w.cg_p = dmalloc(cb);
  w.cg_q = dmalloc(cb);
  const size_t qb = (size_t)c.n_p * K * esz;
  w.qcg_x = dmalloc(qb);
  w.qcg_r = dmalloc(qb);
  w.qcg_z = dmalloc(qb);
  w.qcg_p = dmalloc(qb);
  w.qcg_q = dmalloc(qb);
  w.S = (double*)dmalloc(sizeof(double) * S_NFIELDS * K);
  GBS_CUDA(cudaMallocHost((void**)&w.S_host, sizeof(double) * S_NFIELDS * K));
  w.flag = (int*)dmalloc(sizeof(int) * 8);
  GBS_CUDA(cudaMallocHost((void**)&w.flag_host, sizeof(int) * 8));
  w.partial = (double*)dmalloc(sizeof(double) * kRB * 32 * 4);
  w.counter = (unsigned*)dmalloc(64);
  w.aux = (double*)dmalloc(sizeof(double) * kRB * 32);
  GBS_CUDA(cudaMemsetAsync(w.counter, 0, 64, c.stream));
  GBS_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int) * 8, c.stream));
  GBS_CUDA(cudaMemsetAsync(w.S, 0, sizeof(double) * S_NFIELDS * K, c.stream));
  w.graph_valid = false;
}

void ensure_workspace(Ctx& c, int K, int precision, int k_io) {
  Workspace& w = c.ws;
  const size_t n = (size_t)(c.n_u + c.n_p);
  if (!(w.K == K && w.precision == precision && w.n == n && w.x)) {
    release_workspace(c);
    // an allocation that fails part way releases everything, so that a
    // half-built workspace never passes the check above
    try {
      alloc_workspace(c, K, precision, n);
    } catch (...) {
      release_workspace(c);
      throw;
    }
  }
  if (k_io > 0 && w.k < k_io) {
    w.graph_valid = false;
    for (double** b : {&w.rhs_tmp, &w.host_in, &w.host_out}) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    w.k = 0;
    w.rhs_tmp = (double*)dmalloc(sizeof(double) * n * k_io);
    w.host_in = (double*)dmalloc(sizeof(double) * n * k_io);
    w.host_out = (double*)dmalloc(sizeof(double) * n * k_io);
    w.k = k_io;
  }
}

Args make_args(Ctx& c, const gb_solve_opts* o, int k) {
  Workspace& w = c.ws;
  Args a;
  std::memset(&a, 0, sizeof(a));
  a.n_u = (int)c.n_u;
  a.n_p = (int)c.n_p;
  a.k = k;
  a.A_ptr = c.A_ptr.p;
  a.A_col = c.A_col.p;
  a.A_val = c.A_val.p;
  a.A_val32 = c.A_val32.p;
  a.L_ptr = c.L_ptr.p;
  a.L_col = c.L_col.p;
  a.L_val = c.L_val.p;
  a.L_inv = c.L_inv.p;
  a.L_val32 = c.L_val32.p;
  a.L_inv32 = c.L_inv32.p;
  a.U_ptr = c.U_ptr.p;
  a.U_col = c.U_col.p;
  a.U_val = c.U_val.p;
  a.U_val32 = c.U_val32.p;
  a.B_ptr = c.B_ptr.p;
  a.B_col = c.B_col.p;
  a.B_val = c.B_val.p;
  a.Bt_ptr = c.Bt_ptr.p;
  a.Bt_col = c.Bt_col.p;
  a.Bt_val = c.Bt_val.p;
  a.Qdiag = c.Qdiag.p;
  a.wmean = c.wmean.p;
  a.order = c.order_d.p;
  a.nu = c.nu;
  a.x = w.x;
  a.V0 = w.V[0];
  a.V1 = w.V[1];
  a.V2 = w.V[2];
  a.Z0 = w.Z[0];
  a.Z1 = w.Z[1];
  a.W0 = w.W[0];
  a.W1 = w.W[1];
  a.W2 = w.W[2];
  a.q = w.q;
  a.b = w.b;
  a.cg_x = w.cg_x;
  a.cg_r = w.cg_r;
  a.cg_z = w.cg_z;
  a.cg_y = w.cg_y;
  a.cg_p = w.cg_p;
  a.cg_q = w.cg_q;
  a.S = w.S;
  a.flag = w.flag;
  a.jcur = w.flag + 2;
  a.partial = w.partial;
  a.counter = w.counter;
  auto view = [](const Sell& S) {
    SellView v;
    v.off = S.off.p;
    v.row0 = S.row0.p;
    v.rowlen = S.rowlen.p;
    v.col = S.col.p;
    v.val = S.val.p;
    v.val32 = S.val32.p;
    v.nslices = S.nslices;
    return v;
  };
  a.sA = view(c.sA);
  a.sL = view(c.sL);
  a.sU = view(c.sU);
  a.dim = c.dim;
  a.qm = c.N + c.p - 1;
  a.qp = c.p;
  a.Q_ptr = c.Q_ptr.p;
  a.Q_col = c.Q_col.p;
  a.Q_val = c.Q_val.p;
  a.Q_val32 = c.Q_val32.p;
  a.l1 = c.l1.p;
  a.l1_32 = c.l1_32.p;
  a.qcg_x = w.qcg_x;
  a.qcg_r = w.qcg_r;
  a.qcg_z = w.qcg_z;
  a.qcg_p = w.qcg_p;
  a.qcg_q = w.qcg_q;
  a.pressure_block = GB_PRESSURE_DIAG;
  a.velocity_block = GB_VELOCITY_IC0_PCG;
  a.stop_rule = GB_STOP_RESIDUAL;
  a.A_diag = c.A_diag.p;
  a.R = w.R;
  a.lz = w.lz;
  a.lz_cap = w.lz_cap;
  a.dev_status = c.status_d.p + 2;
  a.KW0 = w.KW[0];
  a.KW1 = w.KW[1];
  a.KW2 = w.KW[2];
  if (o) {
    a.pressure_block = o->pressure_block;
    a.velocity_block = o->velocity_block;
    a.stop_rule = o->stop_rule;
    a.forced_q = o->forced_q_host ? w.forced_q : nullptr;
    a.nforced_q = o->forced_q_host ? (int)o->nforced_q : 0;
    a.tol = o->tol;
    a.inner_tol = o->inner_tol;
    a.max_outer = o->max_outer;
    a.max_inner = o->max_inner;
    a.forced = o->forced_inner_host ? w.forced : nullptr;
    a.nforced = o->forced_inner_host ? (int)o->nforced : 0;
  }
  return a;
}

// Dynamic shared memory of k_trsv_level_staged for a block of at most ecap
// entries and rcap rows.
size_t staged_smem_bytes(int ecap, int rcap, size_t tsize) {
  return (size_t)(2 * ecap + 2 * rcap) * tsize + (size_t)(ecap + rcap + 1) * 4;
}

template <class T, bool FWD, int G>
void staged_allow_smem_one(size_t bytes) {
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_staged<T, FWD, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes));
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_staged<T, FWD, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
}

template <class T, bool FWD, int G>
void packed_allow_smem_one(size_t bytes) {
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_packed<T, FWD, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes));
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_packed<T, FWD, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
}

template <class T, bool FWD>
void packed_allow_smem(size_t bytes) {
  packed_allow_smem_one<T, FWD, 1>(bytes);
  packed_allow_smem_one<T, FWD, 2>(bytes);
  packed_allow_smem_one<T, FWD, 4>(bytes);
  packed_allow_smem_one<T, FWD, 8>(bytes);
  packed_allow_smem_one<T, FWD, 16>(bytes);
  packed_allow_smem_one<T, FWD, 32>(bytes);
}

template <class T, bool FWD, int G>
void split_allow_smem_one(size_t bytes) {
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_split<T, FWD, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes));
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_split<T, FWD, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
}

template <class T, bool FWD>
void split_allow_smem(size_t bytes) {
  split_allow_smem_one<T, FWD, 1>(bytes);
  split_allow_smem_one<T, FWD, 2>(bytes);
  split_allow_smem_one<T, FWD, 4>(bytes);
  split_allow_smem_one<T, FWD, 8>(bytes);
  split_allow_smem_one<T, FWD, 16>(bytes);
  split_allow_smem_one<T, FWD, 32>(bytes);
}

// Dynamic shared memory of k_trsv_level_packed (one size for every launch).
size_t packed_smem_bytes(int cap, int rcap, size_t tsize) {
  return (size_t)(2 * cap + 2 * rcap) * tsize + (size_t)cap * 4;
}

template <class T>
size_t packed_bytes(const Ctx& c) {
  return packed_smem_bytes(std::max(c.pL.cap, c.pU.cap), std::max(c.pL.rcap, c.pU.rcap), sizeof(T));
}

// Dynamic shared memory of k_trsv_level_split (one size for every launch):
// values and solution entries per slot, partial sum and inverse diagonal per row.
template <class T>
size_t split_bytes(const Ctx& c) {
  return (size_t)(2 * std::max(c.qL.cap, c.qU.cap) + 2 * std::max(c.qL.rcap, c.qU.rcap)) * sizeof(T);
}

template <class T, bool FWD>
void staged_allow_smem(size_t bytes) {
  staged_allow_smem_one<T, FWD, 1>(bytes);
  staged_allow_smem_one<T, FWD, 2>(bytes);
  staged_allow_smem_one<T, FWD, 4>(bytes);
  staged_allow_smem_one<T, FWD, 8>(bytes);
  staged_allow_smem_one<T, FWD, 16>(bytes);
  staged_allow_smem_one<T, FWD, 32>(bytes);
}

// Shared memory of every staged launch of this problem: one size for all
// levels and both sweeps, with the carve-out fixed at its shared-memory
// maximum, so consecutive levels never ask the SMs for a different L1 /
// shared split (a change that cannot overlap the previous level).
template <class T>
size_t staged_bytes(const Ctx& c) {
  return staged_smem_bytes(std::max(c.tL.ecap, c.tU.ecap), std::max(c.tL.rcap, c.tU.rcap), sizeof(T));
}

// Shared memory and row capacity of k_trsv_level_batch.
int batch_capr(const Ctx& c) { return std::max(1, std::min(c.max_lrow, 512)); }
template <int K, class T>
size_t batch_bytes(const Ctx& c) {
  return (size_t)(kBlock / K) * batch_capr(c) * (sizeof(T) + 4);
}
template <int K, class T>
void batch_allow_smem(const Ctx& c) {
  const int b = (int)batch_bytes<K, T>(c);
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_batch<K, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_batch<K, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
}

// Dynamic shared memory of k_trsv_level_tma: two stages of values and column
// indices, then two mbarriers (one size for every launch).
template <class T>
size_t tma_bytes() {
  return (size_t)2 * kTmaCap * (sizeof(T) + 4) + 2 * sizeof(uint64_t);
}

template <class T, bool FWD, int W>
void tma_allow_smem_one() {
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_tma<T, FWD, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tma_bytes<T>()));
  GBS_CUDA(cudaFuncSetAttribute(k_trsv_level_tma<T, FWD, W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
}

template <class T>
void tma_prepare(Ctx& c) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  if (c.tma_bps[pi] > 0) return;
  tma_allow_smem_one<T, true, 1>();
  tma_allow_smem_one<T, true, 2>();
  tma_allow_smem_one<T, true, 4>();
  tma_allow_smem_one<T, true, 8>();
  tma_allow_smem_one<T, false, 1>();
  tma_allow_smem_one<T, false, 2>();
  tma_allow_smem_one<T, false, 4>();
  tma_allow_smem_one<T, false, 8>();
  int bps = 0;  // the forward W = 8 form has the largest static shared memory
  GBS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_trsv_level_tma<T, true, 8>, kBlock,
                                                         tma_bytes<T>()));
  c.tma_bps[pi] = std::max(1, bps);
}

// Raise the dynamic shared-memory limits of the sweep kernels that stage in
// shared memory to what the layouts of this problem need (outside any graph
// capture).
template <class T>
void staged_prepare(Ctx& c) {
  tma_prepare<T>(c);
  batch_allow_smem<8, T>(c);
  batch_allow_smem<32, T>(c);
  staged_allow_smem<T, true>(staged_bytes<T>(c));
  staged_allow_smem<T, false>(staged_bytes<T>(c));
  packed_allow_smem<T, true>(packed_bytes<T>(c));
  packed_allow_smem<T, false>(packed_bytes<T>(c));
  split_allow_smem<T, true>(split_bytes<T>(c));
  split_allow_smem<T, false>(split_bytes<T>(c));
}

template <class T>
const T* pick_host(const double* d, const float* f);
template <>
const double* pick_host<double>(const double* d, const float*) {
  return d;
}
template <>
const float* pick_host<float>(const double*, const float* f) {
  return f;
}

int grid_cap(int64_t threads) {
  int64_t g = (threads + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kRB));
}

template <int K, class T>
struct Run {
  Ctx& c;
  Args a;
  cudaStream_t s;
  int vspmv = 0, vtrsv = 0;  // single-RHS layouts (Ctx::var_spmv, Ctx::var_trsv)
  int vbatch = 0;            // batched sweep (Ctx::var_trsv_batch)
  static constexpr int G = Map<K>::G;
  Run(Ctx& cc, Args aa) : c(cc), a(aa), s(cc.stream) {
    const int pi = std::is_same<T, float>::value ? 1 : 0;
    vspmv = K == 1 ? std::max(0, c.var_spmv[pi]) : 0;
    vtrsv = K == 1 ? std::max(0, c.var_trsv[pi]) : 0;
    vbatch = K == 1 ? 0 : std::max(0, c.var_trsv_batch[pi][K == 8 ? 0 : 1]);
  }
  int64_t n() const { return c.n_u + c.n_p; }

  void gather(const double* rhs) { k_gather<K><<<grid_cap(n() * K), kBlock, 0, s>>>(a, rhs); }
  void lanczos() { k_lanczos<K, T><<<grid_cap(n() * K), kBlock, 0, s>>>(a); }
  void stokes() { k_stokes_apply<K><<<grid_cap(n() * G), kBlock, 0, s>>>(a); }
  void gamma() { k_gamma<K, T><<<grid_cap(n() * K), kBlock, 0, s>>>(a); }
  void update() { k_update<K><<<grid_cap(n() * K), kBlock, 0, s>>>(a); }
  // One kernel per level, launched with programmatic dependent launch so a
  // level's independent loads overlap the previous level (k_trsv_level).
  template <bool FWD, int GG>
  void staged_level(cudaLaunchConfig_t& cfg, const Staged& st, int l) {
    GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_staged<T, FWD, GG>, a, (const int4*)st.desc.p + st.lev_b[l],
                                std::max(c.tL.ecap, c.tU.ecap), std::max(c.tL.rcap, c.tU.rcap)));
  }
  template <bool FWD, int GG>
  void packed_level(cudaLaunchConfig_t& cfg, const Packed& pk, int l) {
    GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_packed<T, FWD, GG>, a, (const int4*)pk.desc.p + pk.lev_b[l],
                                (const int32_t*)pk.data.col.p, pick_host<T>(pk.data.val.p, pk.data.val32.p),
                                std::max(c.pL.cap, c.pU.cap), std::max(c.pL.rcap, c.pU.rcap)));
  }
  template <bool FWD, int GG>
  void split_level(cudaLaunchConfig_t& cfg, const Packed& pk, int l) {
    const int ln = FWD ? l + 1 : l - 1;  // next level of the sweep
    const bool has = ln >= 0 && ln < c.nlev;
    GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_split<T, FWD, GG>, a, (const int4*)pk.desc.p + pk.lev_b[l],
                                (const int32_t*)pk.data.col.p, pick_host<T>(pk.data.val.p, pk.data.val32.p),
                                std::max(c.qL.cap, c.qU.cap), std::max(c.qL.rcap, c.qU.rcap),
                                (const int4*)pk.desc.p + (has ? pk.lev_b[ln] : 0), has ? pk.lev_nb[ln] : 0));
  }
  // SELL-32 sweeps with W warps per slice (k_trsv_level_sellw): W from the
  // level's longest row; with `resident` a grid of at most the resident
  // blocks, each taking several slice groups.
  template <bool FWD, int W, int PF>
  void sellw_level(cudaLaunchConfig_t& cfg, int l, bool resident = false) {
    const int s0 = c.lev_slice[l], s1 = c.lev_slice[l + 1];
    constexpr int SPB = kBlock / (32 * W);
    int grid = std::max(1, (s1 - s0 + SPB - 1) / SPB);
    if (resident) grid = std::min(grid, c.n_sm * 5);  // the resident blocks of 256 threads (launch bounds: 5 per SM)
    cfg.gridDim = dim3((unsigned)grid);
    GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_sellw<T, FWD, W, PF>, a, s0, s1));
  }
  // TMA-staged SELL sweep: W from the level's longest row, a grid of at
  // most the resident blocks, each taking groups of 8 / W slices in turn.
  template <bool FWD, int W>
  void tma_level(cudaLaunchConfig_t& cfg, int l) {
    const int s0 = c.lev_slice[l], s1 = c.lev_slice[l + 1];
    constexpr int SPB = kBlock / (32 * W);
    const int groups = std::max(1, (s1 - s0 + SPB - 1) / SPB);
    const int pi = std::is_same<T, float>::value ? 1 : 0;
    const int grid = std::min(groups, c.n_sm * std::max(1, c.tma_bps[pi]));
    cfg.gridDim = dim3((unsigned)grid);
    cfg.dynamicSmemBytes = tma_bytes<T>();
    GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_tma<T, FWD, W>, a, s0, s1));
  }
  template <bool FWD>
  void level(int l) {
    if (K == 1 && vtrsv >= 9) {
      const int len = FWD ? c.lev_maxL[l] : c.lev_maxU[l];
      cudaLaunchConfig_t cfg = {};
      cfg.blockDim = dim3(kBlock);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (vtrsv == 9) {
        if (len <= kSellwPF) sellw_level<FWD, 1, kSellwPF>(cfg, l);
        else if (len <= 2 * kSellwPF) sellw_level<FWD, 2, kSellwPF>(cfg, l);
        else if (len <= 4 * kSellwPF) sellw_level<FWD, 4, kSellwPF>(cfg, l);
        else sellw_level<FWD, 8, kSellwPF>(cfg, l);
      } else if (vtrsv == 10) {
        if (len <= kTmaPF) tma_level<FWD, 1>(cfg, l);
        else if (len <= 2 * kTmaPF) tma_level<FWD, 2>(cfg, l);
        else if (len <= 4 * kTmaPF) tma_level<FWD, 4>(cfg, l);
        else tma_level<FWD, 8>(cfg, l);
      } else if (vtrsv == 18) {  // about 32 slots per lane; levels of one warp per slice prefetch 12 slots
        if (len <= 32) sellw_level<FWD, 1, kSellwPF>(cfg, l);
        else if (len <= 64) sellw_level<FWD, 2, kSellwLitePF>(cfg, l);
        else if (len <= 128) sellw_level<FWD, 4, kSellwLitePF>(cfg, l);
        else sellw_level<FWD, 8, kSellwLitePF>(cfg, l);
      } else if (vtrsv == 15) {  // lightest form: two slots before the wait, about 16 per lane
        if (len <= 16) sellw_level<FWD, 1, kSellwLite2PF>(cfg, l);
        else if (len <= 32) sellw_level<FWD, 2, kSellwLite2PF>(cfg, l);
        else if (len <= 64) sellw_level<FWD, 4, kSellwLite2PF>(cfg, l);
        else sellw_level<FWD, 8, kSellwLite2PF>(cfg, l);
      } else {  // light form: about 16 (11, 13), 8 (12), 32 (14), 24 (16) or 48 (17) slots per lane;
                // 13 on a resident grid
        const int per = vtrsv == 12 ? 8 : vtrsv == 14 ? 32 : vtrsv == 16 ? 24 : vtrsv == 17 ? 48 : 16;
        const bool res = vtrsv == 13;
        if (len <= per) sellw_level<FWD, 1, kSellwLitePF>(cfg, l, res);
        else if (len <= 2 * per) sellw_level<FWD, 2, kSellwLitePF>(cfg, l, res);
        else if (len <= 4 * per) sellw_level<FWD, 4, kSellwLitePF>(cfg, l, res);
        else sellw_level<FWD, 8, kSellwLitePF>(cfg, l, res);
      }
      return;
    }
    if (K == 1 && vtrsv >= 7) {
      const Packed& pk = FWD ? c.qL : c.qU;
      const float per_lane = vtrsv == 7 ? 12.f : 32.f;
      int lanes = 1;
      while (lanes < 32 && pk.lev_mean[l] > per_lane * (float)lanes) lanes *= 2;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)pk.lev_nb[l]);
      cfg.blockDim = dim3(kBlock);
      cfg.dynamicSmemBytes = split_bytes<T>(c);
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      switch (lanes) {
        case 1: split_level<FWD, 1>(cfg, pk, l); break;
        case 2: split_level<FWD, 2>(cfg, pk, l); break;
        case 4: split_level<FWD, 4>(cfg, pk, l); break;
        case 8: split_level<FWD, 8>(cfg, pk, l); break;
        case 16: split_level<FWD, 16>(cfg, pk, l); break;
        default: split_level<FWD, 32>(cfg, pk, l); break;
      }
      return;
    }
    if (K == 1 && vtrsv >= 5) {
      const Packed& pk = FWD ? c.pL : c.pU;
      const float per_lane = vtrsv == 5 ? 12.f : 32.f;
      int lanes = 1;
      while (lanes < 32 && pk.lev_mean[l] > per_lane * (float)lanes) lanes *= 2;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)pk.lev_nb[l]);
      cfg.blockDim = dim3(kBlock);
      cfg.dynamicSmemBytes = packed_bytes<T>(c);
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      switch (lanes) {
        case 1: packed_level<FWD, 1>(cfg, pk, l); break;
        case 2: packed_level<FWD, 2>(cfg, pk, l); break;
        case 4: packed_level<FWD, 4>(cfg, pk, l); break;
        case 8: packed_level<FWD, 8>(cfg, pk, l); break;
        case 16: packed_level<FWD, 16>(cfg, pk, l); break;
        default: packed_level<FWD, 32>(cfg, pk, l); break;
      }
      return;
    }
    if (K == 1 && vtrsv >= 2) {
      const Staged& st = FWD ? c.tL : c.tU;
      const float per_lane = vtrsv == 2 ? 4.f : (vtrsv == 3 ? 12.f : 32.f);
      int lanes = 1;
      while (lanes < 32 && st.lev_mean[l] > per_lane * (float)lanes) lanes *= 2;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)st.lev_nb[l]);
      cfg.blockDim = dim3(kBlock);
      cfg.dynamicSmemBytes = staged_bytes<T>(c);
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      switch (lanes) {
        case 1: staged_level<FWD, 1>(cfg, st, l); break;
        case 2: staged_level<FWD, 2>(cfg, st, l); break;
        case 4: staged_level<FWD, 4>(cfg, st, l); break;
        case 8: staged_level<FWD, 8>(cfg, st, l); break;
        case 16: staged_level<FWD, 16>(cfg, st, l); break;
        default: staged_level<FWD, 32>(cfg, st, l); break;
      }
      return;
    }
    if (K > 1 && vbatch == 1) {
      constexpr int KB = K > 1 ? K : 8;  // (K == 1 never reaches here)
      const int r0 = c.lev_ptr[l], r1 = c.lev_ptr[l + 1];
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)((r1 - r0 + kBlock / KB - 1) / (kBlock / KB)));
      cfg.blockDim = dim3(kBlock);
      cfg.dynamicSmemBytes = batch_bytes<KB, T>(c);
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_batch<KB, T, FWD>, a, r0, r1, batch_capr(c)));
      return;
    }
    const bool sell = (K == 1 && vtrsv == 1);
    const int r0 = sell ? c.lev_slice[l] : c.lev_ptr[l];
    const int r1 = sell ? c.lev_slice[l + 1] : c.lev_ptr[l + 1];
    const int64_t th = (int64_t)(r1 - r0) * (sell ? 32 : G);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((th + kBlock - 1) / kBlock));
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (sell) GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level_sell<T, FWD>, a, r0, r1));
    else GBS_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_level<K, T, FWD>, a, r0, r1));
  }
  void spmv() {
    if (K == 1 && vspmv == 2) k_cg_spmv_sellw<T, 2><<<grid_cap((int64_t)c.sA.nslices * 64), kBlock, 0, s>>>(a);
    else if (K == 1 && vspmv == 3) k_cg_spmv_sellw<T, 4><<<grid_cap((int64_t)c.sA.nslices * 128), kBlock, 0, s>>>(a);
    else if (K == 1 && vspmv == 1) k_cg_spmv_sell<T><<<grid_cap((int64_t)c.sA.nslices * 32), kBlock, 0, s>>>(a);
    else k_cg_spmv<K, T><<<grid_cap(c.n_u * G), kBlock, 0, s>>>(a);
  }
  void trsv_fwd() {
    for (int l = 0; l < c.nlev; ++l) level<true>(l);
  }
  void trsv_bwd() {
    for (int l = c.nlev - 1; l >= 0; --l) level<false>(l);
  }
  // M^{-1} r of the velocity CG: the IC(0) sweeps, or the diagonal
  bool vel_cg() const { return a.velocity_block != GB_VELOCITY_DIAG; }
  void vel_precond() {
    if (a.velocity_block == GB_VELOCITY_JACOBI_PCG) {
      k_jacobi<K, T, 0><<<grid_cap(c.n_u * K), kBlock, 0, s>>>(a);
    } else {
      trsv_fwd();
      trsv_bwd();
    }
  }
  void cg_prologue() {
    vel_precond();
    k_cg_rho<K, T><<<grid_cap(c.n_u * K), kBlock, 0, s>>>(a, 1);
  }
  void cg_head() {
    spmv();
    k_cg_axpy<K, T><<<grid_cap(c.n_u * K), kBlock, 0, s>>>(a);
  }
  void cg_tail() {
    vel_precond();
    k_cg_rho<K, T><<<grid_cap(c.n_u * K), kBlock, 0, s>>>(a, 0);
    k_cg_pupdate<K, T><<<grid_cap(c.n_u * K), kBlock, 0, s>>>(a);
  }
  // Pressure-block CG on Q (GB_PRESSURE_PCG): the IC(0) application is one
  // pass of banded line solves per direction, alternating between the
  // z and q buffers so that the last pass lands in z.
  bool pcg_q() const { return a.pressure_block != GB_PRESSURE_DIAG; }
  void q_precond() {
    if (a.pressure_block == GB_PRESSURE_JACOBI_PCG) k_jacobi<K, T, 1><<<grid_cap(c.n_p * K), kBlock, 0, s>>>(a);
    else q_lines();
  }
  void q_lines() {
    const int64_t threads = (int64_t)c.n_p / (c.N + c.p - 1) * K;
    const int grid = (int)((threads + 127) / 128);
    const T* src = (const T*)a.qcg_r;
    for (int axis = 0; axis < c.dim; ++axis) {
      T* dst = (T*)(((c.dim - 1 - axis) % 2 == 0) ? a.qcg_z : a.qcg_q);
      k_q_lines<K, T><<<grid, 128, 0, s>>>(a, axis, src, dst);
      src = dst;
    }
  }
  void qcg_prologue() {
    q_precond();
    k_cg_rho<K, T, 1><<<grid_cap(c.n_p * K), kBlock, 0, s>>>(a, 1);
  }
  void qcg_head() {
    k_cg_spmv<K, T, 1><<<grid_cap(c.n_p * G), kBlock, 0, s>>>(a);
    k_cg_axpy<K, T, 1><<<grid_cap(c.n_p * K), kBlock, 0, s>>>(a);
  }
  void qcg_tail() {
    q_precond();
    k_cg_rho<K, T, 1><<<grid_cap(c.n_p * K), kBlock, 0, s>>>(a, 0);
    k_cg_pupdate<K, T, 1><<<grid_cap(c.n_p * K), kBlock, 0, s>>>(a);
  }
  void finish(double* out) {
    k_residual<K><<<grid_cap(n() * G), kBlock, 0, s>>>(a);
    k_scatter<K><<<grid_cap(n() * K), kBlock, 0, s>>>(a, out);
  }

  int read_flag(int i) {
    GBS_CUDA(cudaMemcpyAsync(c.ws.flag_host, c.ws.flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    GBS_CUDA(cudaStreamSynchronize(s));
    return c.ws.flag_host[i];
  }
  void cg_loop_host() {
    for (; vel_cg();) {
      cg_head();
      if (!read_flag(1)) break;
      cg_tail();
    }
    if (!pcg_q()) return;
    qcg_prologue();
    for (;;) {
      qcg_head();
      if (!read_flag(3)) break;
      qcg_tail();
    }
  }
  void run_host(const double* rhs, double* out) {
    a.use_handles = 0;
    gather(rhs);
    lanczos();
    if (vel_cg()) cg_prologue();
    cg_loop_host();
    gamma();
    while (read_flag(0)) {
      stokes();
      lanczos();
      if (vel_cg()) cg_prologue();
      cg_loop_host();
      gamma();
      update();
    }
    finish(out);
    GBS_CUDA(cudaGetLastError());
  }

  // --- CUDA graph with device-side loop control
  cudaGraph_t add_while(cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    GBS_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, &ed, &nd));
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};  // aggregate init (no default ctor)
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    GBS_CUDA(cudaGraphAddNode(&node, cg, deps, ed, nd, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    GBS_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return body;
  }
  template <class F>
  void capture_into(cudaGraph_t g, F fn) {
    GBS_CUDA(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    fn();
    cudaGraph_t out = nullptr;
    GBS_CUDA(cudaStreamEndCapture(s, &out));
  }
  cudaGraphExec_t build_graph(const double* rhs, double* out) {
    cudaGraph_t g;
    GBS_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h_out, h_in0 = 0, h_in = 0, h_q0 = 0, h_q = 0;
    GBS_CUDA(cudaGraphConditionalHandleCreate(&h_out, g, 0, 0));
    if (vel_cg()) GBS_CUDA(cudaGraphConditionalHandleCreate(&h_in0, g, 0, 0));
    if (pcg_q()) GBS_CUDA(cudaGraphConditionalHandleCreate(&h_q0, g, 0, 0));
    const Args base = a;
    a.use_handles = 1;
    a.h_outer = h_out;
    a.h_inner = h_in0;
    a.h_qinner = h_q0;
    cudaGraph_t body0 = nullptr, bodyO = nullptr, bodyI = nullptr, bodyQ0 = nullptr, bodyQ = nullptr;
    capture_into(g, [&] {
      gather(rhs);
      lanczos();
      if (vel_cg()) {
        cg_prologue();
        body0 = add_while(h_in0);
      }
      if (pcg_q()) {
        qcg_prologue();
        bodyQ0 = add_while(h_q0);
      }
      gamma();
      bodyO = add_while(h_out);
      finish(out);
    });
    if (vel_cg())
      capture_into(body0, [&] {
        cg_head();
        cg_tail();
      });
    if (pcg_q())
      capture_into(bodyQ0, [&] {
        qcg_head();
        qcg_tail();
      });
    if (vel_cg()) GBS_CUDA(cudaGraphConditionalHandleCreate(&h_in, bodyO, 0, 0));
    if (pcg_q()) GBS_CUDA(cudaGraphConditionalHandleCreate(&h_q, bodyO, 0, 0));
    a.h_inner = h_in;
    a.h_qinner = h_q;
    capture_into(bodyO, [&] {
      stokes();
      lanczos();
      if (vel_cg()) {
        cg_prologue();
        bodyI = add_while(h_in);
      }
      if (pcg_q()) {
        qcg_prologue();
        bodyQ = add_while(h_q);
      }
      gamma();
      update();
    });
    if (vel_cg())
      capture_into(bodyI, [&] {
        cg_head();
        cg_tail();
      });
    if (pcg_q())
      capture_into(bodyQ, [&] {
        qcg_head();
        qcg_tail();
      });
    a = base;
    cudaGraphExec_t exec = nullptr;
    GBS_CUDA(cudaGraphInstantiate(&exec, g, 0));
    GBS_CUDA(cudaGraphDestroy(g));
    return exec;
  }
};

// In-graph time of one single-RHS layout pair: a solve of one MINRES step
// whose two preconditioner applications are forced (replay mode) to
// kTuneInner inner iterations each, captured as the CUDA graph a solve runs --
// SpMV, CG vector kernels, sweeps and MINRES kernels in their graph order,
// each finding the L2 contents the previous one left -- launched once to warm
// up, then timed over two launches.  rhs / out are the solve's own buffers
// (out is overwritten by the solve that follows).
constexpr int kTuneInner = 12;

template <class T>
float time_layouts_in_graph(Ctx& c, const double* rhs, double* out, int vspmv, int vtrsv) {
  if (!c.tune_forced.p) {
    const int32_t h[2] = {kTuneInner, kTuneInner};
    c.tune_forced.upload(h, 2, c.stream);
  }
  gb_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.tol = 0.0;
  o.inner_tol = 1e-2;
  o.precision = std::is_same<T, float>::value ? GB_PREC_MIXED : GB_PREC_FP64;
  o.max_outer = 1;
  o.max_inner = 1000;
  o.use_graph = 1;
  o.pressure_block = GB_PRESSURE_DIAG;
  o.stop_rule = GB_STOP_RESIDUAL;
  o.velocity_block = GB_VELOCITY_IC0_PCG;
  Args a = make_args(c, &o, 1);
  a.forced = c.tune_forced.p;
  a.nforced = 2;
  Run<1, T> run(c, a);
  run.vspmv = vspmv;
  run.vtrsv = vtrsv;
  cudaGraphExec_t g = run.build_graph(rhs, out);
  cudaEvent_t e0, e1;
  GBS_CUDA(cudaEventCreate(&e0));
  GBS_CUDA(cudaEventCreate(&e1));
  GBS_CUDA(cudaGraphLaunch(g, c.stream));
  GBS_CUDA(cudaEventRecord(e0, c.stream));
  GBS_CUDA(cudaGraphLaunch(g, c.stream));
  GBS_CUDA(cudaGraphLaunch(g, c.stream));
  GBS_CUDA(cudaEventRecord(e1, c.stream));
  GBS_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  GBS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(g);
  return ms / 2;
}

// Layout tuning for single-RHS solves, once per precision, outside any
// graph capture, at the first solve (with its right-hand side):
// * the inner SpMV: CSR (8 lanes per row) and SELL-32 (thread per row; 2 or
//   4 warps per slice), each timed alone;
// * the IC(0) sweeps: every available form (CSR, SELL-32, three staged, two
//   packed, two split packed, SELL-32 with W warps per slice in nine forms,
//   TMA-staged SELL-32), each timed inside the graph of a short replayed solve
//   (time_layouts_in_graph) with the chosen SpMV, so that the sweep is judged
//   with the L2 contents and launch overlap it has in a solve (timed alone, a
//   sweep finds much of the factor in L2 and the forms that prefetch least
//   look best).
// A form replaces the best so far only when it is 3 % faster.  The choice
// only changes the summation order inside a row.
template <class T>
void autotune_single(Ctx& c, const double* rhs, double* out) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  staged_prepare<T>(c);
  if (c.var_spmv[pi] >= 0 && c.var_trsv[pi] >= 0) return;
  Workspace& w = c.ws;
  if (c.var_spmv[pi] < 0) {
    k_fill_value<T><<<grid_cap(c.n_u), kBlock, 0, c.stream>>>((T*)w.cg_p, c.n_u, T(1));
    const double live[2] = {1.0, 1.0};
    GBS_CUDA(cudaMemcpyAsync(w.S + S_CG_ACTIVE, &live[0], sizeof(double), cudaMemcpyHostToDevice, c.stream));
    GBS_CUDA(cudaMemcpyAsync(w.S + S_RHO, &live[1], sizeof(double), cudaMemcpyHostToDevice, c.stream));
    Args a = make_args(c, nullptr, 1);
    cudaEvent_t e0, e1;
    GBS_CUDA(cudaEventCreate(&e0));
    GBS_CUDA(cudaEventCreate(&e1));
    auto time_spmv = [&](int variant) {
      Run<1, T> run(c, a);
      run.vspmv = variant;
      const int reps = 20;
      run.spmv();
      GBS_CUDA(cudaEventRecord(e0, c.stream));
      for (int r = 0; r < reps; ++r) run.spmv();
      GBS_CUDA(cudaEventRecord(e1, c.stream));
      GBS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      GBS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms;
    };
    float best = time_spmv(0);
    int choice = 0;
    for (int v = 1; v <= 3; ++v) {
      const float t = time_spmv(v);
      if (t < 0.97f * best) {
        best = t;
        choice = v;
      }
    }
    c.var_spmv[pi] = choice;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (c.var_trsv[pi] < 0) {
    float best = time_layouts_in_graph<T>(c, rhs, out, c.var_spmv[pi], 0);
    int choice = 0;
    for (int v = 1; v <= 18; ++v) {
      if (!trsv_available(c, v)) continue;
      const float t = time_layouts_in_graph<T>(c, rhs, out, c.var_spmv[pi], v);
      if (t < 0.97f * best) {
        best = t;
        choice = v;
      }
    }
    c.var_trsv[pi] = choice;
  }
  GBS_CUDA(cudaGetLastError());
}

// Batched sweep tuning: time one IC(0) application of the warp-per-row and
// the staged batched kernels at width K and keep the faster (3 % margin).
template <int K, class T>
void autotune_batch(Ctx& c) {
  const int pi = std::is_same<T, float>::value ? 1 : 0, ki = K == 8 ? 0 : 1;
  staged_prepare<T>(c);
  if (c.var_trsv_batch[pi][ki] >= 0) return;
  Workspace& w = c.ws;
  k_fill_value<T><<<grid_cap(c.n_u * K), kBlock, 0, c.stream>>>((T*)w.cg_r, c.n_u * K, T(1));
  std::vector<double> live(K, 1.0);
  GBS_CUDA(cudaMemcpyAsync(w.S + S_CG_ACTIVE * K, live.data(), sizeof(double) * K, cudaMemcpyHostToDevice, c.stream));
  Args a = make_args(c, nullptr, K);
  cudaEvent_t e0, e1;
  GBS_CUDA(cudaEventCreate(&e0));
  GBS_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](int variant) {
    Run<K, T> run(c, a);
    run.vbatch = variant;
    run.trsv_fwd();
    run.trsv_bwd();
    GBS_CUDA(cudaEventRecord(e0, c.stream));
    for (int r = 0; r < 3; ++r) {
      run.trsv_fwd();
      run.trsv_bwd();
    }
    GBS_CUDA(cudaEventRecord(e1, c.stream));
    GBS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    GBS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  const float t0 = time_it(0), t1 = time_it(1);
  c.var_trsv_batch[pi][ki] = t1 < 0.97f * t0 ? 1 : 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GBS_CUDA(cudaGetLastError());
}

template <int K, class T>
void dispatch_solve(Ctx& c, const double* rhs, double* out, int k, const gb_solve_opts& o) {
  if (K == 1) autotune_single<T>(c, rhs, out);
  if (K > 1) autotune_batch<K, T>(c);
  Args a = make_args(c, &o, k);
  Run<K, T> run(c, a);
  Workspace& w = c.ws;
  if (!o.use_graph) {
    run.run_host(rhs, out);
    return;
  }
  std::vector<double> key = {(double)(uintptr_t)rhs, (double)(uintptr_t)out, (double)k, o.tol, o.inner_tol,
                             (double)o.max_outer, (double)o.max_inner, (double)K, (double)o.precision,
                             (double)a.nforced, c.nu, (double)run.vspmv, (double)run.vtrsv,
                             (double)o.pressure_block, (double)a.nforced_q, (double)o.stop_rule,
                             (double)o.velocity_block, (double)run.vbatch};
  if (!w.graph_valid || w.graph_key != key) {
    if (w.graph) {
      cudaGraphExecDestroy(w.graph);
      w.graph = nullptr;
    }
    w.graph = run.build_graph(rhs, out);
    w.graph_key = key;
    w.graph_valid = true;
  }
  GBS_CUDA(cudaGraphLaunch(w.graph, c.stream));
}

int collect_info(Ctx& c, int k, gb_info* info) {
  Workspace& w = c.ws;
  const int K = w.K;
  int timeout = 0;
  GBS_CUDA(cudaMemcpyAsync(w.S_host, w.S, sizeof(double) * S_NFIELDS * K, cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaMemcpyAsync(&timeout, c.status_d.p + 2, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  if (timeout) {  // a bounded wait of a sweep gave up: the solution is not valid
    GBS_CUDA(cudaMemsetAsync(c.status_d.p + 2, 0, sizeof(int), c.stream));
    for (int t = 0; t < k; ++t) info[t].status = GB_ERR_DEVICE_TIMEOUT;
    GBS_CUDA(cudaStreamSynchronize(c.stream));
    return GB_ERR_DEVICE_TIMEOUT;
  }
  int worst = GB_OK;
  for (int t = 0; t < k; ++t) {
    auto f = [&](int field) { return w.S_host[field * K + t]; };
    gb_info& I = info[t];
    I.outer_its = (int)f(S_OUTER_ITS);
    I.precond_apps = (int)f(S_APPS);
    I.inner_its_total = (int64_t)f(S_INNER_TOTAL);
    I.inner_its_max = (int)f(S_INNER_MAX);
    I.relres_est = f(S_RELRES);
    I.relres_true = f(S_TRUE_RES);
    I.q_inner_its_total = (int64_t)f(S_Q_TOTAL);
    I.q_inner_its_max = (int)f(S_Q_MAX);
    int st = GB_OK;
    if (f(S_NONFINITE) != 0.0) st = GB_ERR_NONFINITE;
    else if (f(S_INCONSISTENT) != 0.0) st = GB_ERR_INVALID_ARG;
    else if (f(S_STATUS) != 0.0) st = GB_ERR_NOT_CONVERGED;
    I.status = st;
    // severity: nonfinite > invalid argument > not converged (a device
    // timeout has returned above for every column)
    auto rank = [](int v) {
      return v == GB_ERR_NONFINITE ? 3 : v == GB_ERR_INVALID_ARG ? 2 : v == GB_ERR_NOT_CONVERGED ? 1 : 0;
    };
    if (rank(st) > rank(worst)) worst = st;
  }
  return worst;
}

// Timing of one kernel family with the last solve's configuration.
template <int K, class T>
double time_family(Ctx& c, int which, int reps) {
  Workspace& w = c.ws;
  Args a = make_args(c, nullptr, w.last_k);
  Run<K, T> run(c, a);
  std::vector<double> saved(S_NFIELDS * K), act;
  GBS_CUDA(cudaMemcpyAsync(saved.data(), w.S, sizeof(double) * saved.size(), cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  act = saved;
  for (int t = 0; t < w.last_k; ++t) {
    act[S_CG_ACTIVE * K + t] = 1.0;
    act[S_OUTER_ACTIVE * K + t] = 1.0;
    if (act[S_GAMMA * K + t] == 0.0) act[S_GAMMA * K + t] = 1.0;
    if (act[S_RHO * K + t] == 0.0) act[S_RHO * K + t] = 1.0;
  }
  GBS_CUDA(cudaMemcpyAsync(w.S, act.data(), sizeof(double) * act.size(), cudaMemcpyHostToDevice, c.stream));
  auto launch = [&] {
    switch (which) {
      case 0: run.spmv(); break;
      case 1: run.trsv_fwd(); run.trsv_bwd(); break;
      case 2: run.stokes(); break;
      default: run.trsv_fwd(); break;
    }
  };
  launch();
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev) GBS_CUDA(cudaEventCreate(&e));
  for (int r = 0; r < reps; ++r) {
    // sweeps: the inner SpMV runs untimed before each one and streams A_h
    // through L2, as it does before every preconditioner application of a solve
    if (which == 1 || which == 3) run.spmv();
    GBS_CUDA(cudaEventRecord(ev[2 * r], c.stream));
    launch();
    GBS_CUDA(cudaEventRecord(ev[2 * r + 1], c.stream));
  }
  GBS_CUDA(cudaEventSynchronize(ev.back()));
  double ms = 0.0;
  for (int r = 0; r < reps; ++r) {
    float m = 0.f;
    GBS_CUDA(cudaEventElapsedTime(&m, ev[2 * r], ev[2 * r + 1]));
    ms += m;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaMemcpyAsync(w.S, saved.data(), sizeof(double) * saved.size(), cudaMemcpyHostToDevice, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  return ms / reps;
}

}  // namespace

double time_kernel(Ctx& c, int which, int reps) {
  Workspace& w = c.ws;
  if (w.last_k < 1 || !w.x) fail(GB_ERR_INVALID_ARG, "time_kernel needs a completed solve");
  if (which < 0 || which > 3 || reps < 1 || reps > 100000) fail(GB_ERR_INVALID_ARG, "bad time_kernel request");
  const bool mixed = w.precision == GB_PREC_MIXED;
  switch (w.K) {
    case 1: return mixed ? time_family<1, float>(c, which, reps) : time_family<1, double>(c, which, reps);
    case 8: return mixed ? time_family<8, float>(c, which, reps) : time_family<8, double>(c, which, reps);
    default: return mixed ? time_family<32, float>(c, which, reps) : time_family<32, double>(c, which, reps);
  }
}

void release_workspace(Ctx& c) {
  Workspace& w = c.ws;
  if (w.graph) cudaGraphExecDestroy(w.graph);
  void* ptrs[] = {w.x, w.V[0], w.V[1], w.V[2], w.Z[0], w.Z[1], w.W[0], w.W[1], w.W[2], w.q, w.b,
                  w.cg_x, w.cg_r, w.cg_z, w.cg_y, w.cg_p, w.cg_q, w.S, w.flag, w.forced, w.partial,
                  w.counter, w.aux, w.rhs_tmp, w.host_in, w.host_out, w.qcg_x, w.qcg_r, w.qcg_z,
                  w.qcg_p, w.qcg_q, w.forced_q, w.R, w.KW[0], w.KW[1], w.KW[2], w.lz};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (w.S_host) cudaFreeHost(w.S_host);
  if (w.flag_host) cudaFreeHost(w.flag_host);
  w = Workspace();
}

int solve(Ctx& c, const double* rhs_dev, double* x_dev, int k, const gb_solve_opts& o, gb_info* info,
          bool adjoint) {
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "assemble before solve");
  if (o.velocity_block == GB_VELOCITY_IC0_PCG && !c.factored)
    fail(GB_ERR_INVALID_ARG, "factor_ic0 must succeed before an IC(0) velocity block");
  if (k < 1 || k > 32) fail(GB_ERR_INVALID_ARG, "k must be in [1, 32]");
  if (!rhs_dev || !x_dev || !info) fail(GB_ERR_INVALID_ARG, "null pointer argument");
  if (!(o.tol >= 0.0) || !(o.inner_tol > 0.0) || o.max_outer < 1 || o.max_inner < 1)
    fail(GB_ERR_INVALID_ARG, "bad solver options");
  if (o.precision != GB_PREC_FP64 && o.precision != GB_PREC_MIXED) fail(GB_ERR_INVALID_ARG, "bad precision");
  if (o.forced_inner_host && (k != 1 || o.nforced < 1 || o.nforced > (1 << 24)))
    fail(GB_ERR_INVALID_ARG, "replay mode needs k == 1 and 1 <= nforced <= 2^24");
  if (o.pressure_block < GB_PRESSURE_DIAG || o.pressure_block > GB_PRESSURE_JACOBI_PCG)
    fail(GB_ERR_INVALID_ARG, "bad pressure block");
  if (o.velocity_block < GB_VELOCITY_IC0_PCG || o.velocity_block > GB_VELOCITY_JACOBI_PCG)
    fail(GB_ERR_INVALID_ARG, "bad velocity block");
  if (o.stop_rule != GB_STOP_RESIDUAL && o.stop_rule != GB_STOP_ESTIMATE) fail(GB_ERR_INVALID_ARG, "bad stop rule");
  if (o.forced_q_host && (o.pressure_block == GB_PRESSURE_DIAG || k != 1 || o.nforced_q < 1 ||
                          o.nforced_q > (1 << 24)))
    fail(GB_ERR_INVALID_ARG, "pressure replay needs a CG pressure block, k == 1, 1 <= nforced_q <= 2^24");
  if (o.forced_inner_host && o.velocity_block == GB_VELOCITY_DIAG)
    fail(GB_ERR_INVALID_ARG, "velocity replay needs a CG velocity block");
  if (o.pressure_block == GB_PRESSURE_PCG && !c.q_factored)
    fail(GB_ERR_IC0_BREAKDOWN, "IC(0) of the pressure mass matrix failed");
  const int K = (k == 1) ? 1 : (k <= 8 ? 8 : 32);
  ensure_workspace(c, K, o.precision, k);
  Workspace& w = c.ws;
  {
    // Lanczos record: max_outer steps (and gamma_{max_outer+1}), capped
    const int cap = std::min(o.max_outer, 1 << 20) + 1;
    if (!w.lz || w.lz_cap < cap) {
      if (w.lz) cudaFree(w.lz);
      w.lz = nullptr;
      w.lz_cap = 0;
      w.graph_valid = false;
      w.lz = (double*)dmalloc(sizeof(double) * 2 * (size_t)K * cap);
      w.lz_cap = cap;
      w.graph_valid = false;
    }
  }
  if (o.forced_q_host) {
    if ((size_t)o.nforced_q > w.forced_q_cap) {
      if (w.forced_q) cudaFree(w.forced_q);
      w.forced_q = nullptr;
      w.forced_q_cap = 0;
      w.graph_valid = false;
      w.forced_q = (int32_t*)dmalloc(sizeof(int32_t) * o.nforced_q);
      w.forced_q_cap = o.nforced_q;
      w.graph_valid = false;
    }
    GBS_CUDA(cudaMemcpyAsync(w.forced_q, o.forced_q_host, sizeof(int32_t) * o.nforced_q,
                             cudaMemcpyHostToDevice, c.stream));
  }
  if (o.forced_inner_host) {
    if ((size_t)o.nforced > w.forced_cap) {
      if (w.forced) cudaFree(w.forced);
      w.forced = nullptr;
      w.forced_cap = 0;
      w.graph_valid = false;
      w.forced = (int32_t*)dmalloc(sizeof(int32_t) * o.nforced);
      w.forced_cap = o.nforced;
      w.graph_valid = false;
    }
    GBS_CUDA(cudaMemcpyAsync(w.forced, o.forced_inner_host, sizeof(int32_t) * o.nforced,
                             cudaMemcpyHostToDevice, c.stream));
  }
  const double* rhs = rhs_dev;
  if (adjoint) {
    k_adjoint_coef<<<k, kBlock, 0, c.stream>>>((int)c.n_u, (int)c.n_p, k, rhs_dev, c.wmean.p, w.aux);
    k_adjoint_rhs<<<grid_cap((c.n_u + c.n_p) * k), kBlock, 0, c.stream>>>((int)c.n_u, (int)c.n_p, k, rhs_dev,
                                                                         c.wmean.p, w.aux, w.rhs_tmp);
    GBS_CUDA(cudaGetLastError());
    rhs = w.rhs_tmp;
  }
  const bool mixed = o.precision == GB_PREC_MIXED;
  switch (K) {
    case 1:
      mixed ? dispatch_solve<1, float>(c, rhs, x_dev, k, o) : dispatch_solve<1, double>(c, rhs, x_dev, k, o);
      break;
    case 8:
      mixed ? dispatch_solve<8, float>(c, rhs, x_dev, k, o) : dispatch_solve<8, double>(c, rhs, x_dev, k, o);
      break;
    default:
      mixed ? dispatch_solve<32, float>(c, rhs, x_dev, k, o) : dispatch_solve<32, double>(c, rhs, x_dev, k, o);
      break;
  }
  GBS_CUDA(cudaGetLastError());
  w.last_k = k;
  return collect_info(c, k, info);
}

int solve_host(Ctx& c, const double* rhs_host, double* x_host, int k, const gb_solve_opts& o, gb_info* info) {
  if (k < 1 || k > 32 || !rhs_host || !x_host) fail(GB_ERR_INVALID_ARG, "bad host solve arguments");
  const int K = (k == 1) ? 1 : (k <= 8 ? 8 : 32);
  ensure_workspace(c, K, o.precision, k);
  const size_t bytes = sizeof(double) * (size_t)(c.n_u + c.n_p) * k;
  GBS_CUDA(cudaMemcpyAsync(c.ws.host_in, rhs_host, bytes, cudaMemcpyHostToDevice, c.stream));
  int st = solve(c, c.ws.host_in, c.ws.host_out, k, o, info, false);
  GBS_CUDA(cudaMemcpyAsync(x_host, c.ws.host_out, bytes, cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  return st;
}

// ---- Ritz values (spectral diagnostics) --------------------------------------
// MINRES is the Lanczos process on M^{-1} K in the M-inner product (Sec. 5):
// after j steps the tridiagonal T_j (diagonal delta_1..delta_j, off-diagonal
// gamma_2..gamma_j) represents M^{-1} K on the Krylov space, and its
// eigenvalues (Ritz values) approximate the eigenvalues of M^{-1} K, the
// extremal ones first.  The record is written by k_gamma.
int lanczos_coeffs(Ctx& c, int rhs, double* delta, double* gamma, int cap) {
  Workspace& w = c.ws;
  if (!w.lz || w.last_k < 1) fail(GB_ERR_INVALID_ARG, "no completed solve");
  if (rhs < 0 || rhs >= w.last_k) fail(GB_ERR_INVALID_ARG, "rhs out of range");
  const int j = std::min((int)w.S_host[S_OUTER_ITS * w.K + rhs], w.lz_cap - 1);
  const int n = std::min(j, std::max(cap, 0));
  if (delta && n > 0)
    GBS_CUDA(cudaMemcpyAsync(delta, w.lz + (size_t)rhs * w.lz_cap, sizeof(double) * n, cudaMemcpyDeviceToHost,
                             c.stream));
  const int ng = std::min(j + 1, cap + 1);
  if (gamma && ng > 0)
    GBS_CUDA(cudaMemcpyAsync(gamma, w.lz + (size_t)(w.K + rhs) * w.lz_cap, sizeof(double) * ng,
                             cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  return j;
}

namespace {
// Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm
// sequence of the LDL^T pivots of T - x I).
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double off = i ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// The i-th smallest eigenvalue (0-based) by bisection inside [lo, hi].
double kth_eigenvalue(const std::vector<double>& d, const std::vector<double>& e, int i, double lo, double hi) {
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(d, e, mid) > i) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}
}  // namespace

void ritz_extremes(Ctx& c, int rhs, int exclude_one, double* out) {
  std::vector<double> d(c.ws.lz_cap > 0 ? c.ws.lz_cap : 1), g(d.size() + 1);
  const int j = lanczos_coeffs(c, rhs, d.data(), g.data(), (int)d.size());
  const double nan = std::nan("");
  for (int i = 0; i < 4; ++i) out[i] = nan;
  if (j < 1) return;
  d.resize(j);
  std::vector<double> e(g.begin() + 1, g.begin() + j);  // gamma_2 .. gamma_j
  double lo = d[0], hi = d[0];
  for (int i = 0; i < j; ++i) {  // Gershgorin bounds
    const double r = (i ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < j ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  lo -= 1e-12 * (std::fabs(lo) + 1.0);
  hi += 1e-12 * (std::fabs(hi) + 1.0);
  const int neg = sturm_count(d, e, 0.0);
  if (neg > 0) {
    out[0] = kth_eigenvalue(d, e, 0, lo, 0.0);
    out[1] = kth_eigenvalue(d, e, neg - 1, lo, 0.0);
  }
  // positive side, optionally without the Ritz values within 1e-6 of 1
  int first = neg, last = j - 1;
  if (exclude_one) {
    const int c1 = sturm_count(d, e, 1.0 - 1e-6), c2 = sturm_count(d, e, 1.0 + 1e-6);
    if (first >= c1 && first < c2) first = c2;
    if (last >= c1 && last < c2) last = c1 - 1;
  }
  if (first <= last && first < j) {
    out[2] = kth_eigenvalue(d, e, first, 0.0, hi);
    out[3] = kth_eigenvalue(d, e, last, 0.0, hi);
  }
}

void apply_operator(Ctx& c, int which, const double* x, double* y) {
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "assemble first");
  if (which < 0 || which > 4 || !x || !y) fail(GB_ERR_INVALID_ARG, "bad operator request");
  Args a = make_args(c, nullptr, 1);
  const int64_t rows = which == 0 ? c.n_u + c.n_p : ((which == 2 || which == 4) ? c.n_p : c.n_u);
  k_apply_natural<<<grid_cap(rows * 8), kBlock, 0, c.stream>>>(a, which, x, y);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaStreamSynchronize(c.stream));
}

void dnu(Ctx& c, const double* lam, const double* x, int k, double* out) {
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "assemble first");
  if (k < 1 || k > 32 || !lam || !x || !out) fail(GB_ERR_INVALID_ARG, "bad dnu arguments");
  ensure_workspace(c, c.ws.K > 0 ? c.ws.K : 1, c.ws.precision >= 0 ? c.ws.precision : 0, 0);
  Args a = make_args(c, nullptr, 1);
  const int grid = grid_cap(c.n_u * 8);
  double* res = c.ws.aux + (size_t)kRB * 32 - 32;  // k results after the partials
  k_dnu<<<grid, kBlock, 0, c.stream>>>(a, k, lam, x, c.ws.partial, c.ws.counter, res);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaMemcpyAsync(out, res, sizeof(double) * k, cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
}

// ---- dL/dnu without allocating device memory --------------------------------
// gb_dnu may allocate the context's workspace (cudaMalloc) on first use.  Some
// callers cannot allow that: programs whose device memory is handed out by
// their own pool or framework, which forbids raw allocations beside it, and
// callers that have used up a fixed memory budget.  dnu_noalloc computes the
// same quantity with the same kernel (k_dnu, same launch) but takes its
// reduction scratch -- the per-block partial sums, the completion counter and
// the k results -- from the static device array below, whose size is fixed at
// build time: 64 + 1216 * 32 doubles (about 304 KiB), enough for the largest
// launch (1216 blocks) and k <= 32.  Every GPU that loads this library holds
// the array until the process exits.  All calls share it, so calls that
// overlap on the GPU race; each call clears the counter before its launch.
// The call ends by copying the k results to host memory and waiting for them.
constexpr int kNoAllocMaxK = 32;
constexpr size_t kNoAllocDoubles = 64 + (size_t)kRB * kNoAllocMaxK;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_addr[64] = {};  // device address of g_noalloc_scratch, per device

// The host-side name g_noalloc_scratch is only a stand-in for the symbol; the
// kernel needs its device address, looked up once per device with that
// device current (the first call on a device does this lookup, so it should
// come before any stream capture).
double* noalloc_scratch() {
  int dev = 0;
  GBS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(GB_ERR_INVALID_ARG, "gb_dnu_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      fail(GB_ERR_CUDA, std::string("gb_dnu_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    }
    g_noalloc_addr[dev] = (double*)p;
  }
  return g_noalloc_addr[dev];
}
}  // namespace

void dnu_noalloc(Ctx& c, const double* lam, const double* x, int k, double* out) {
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "gb_dnu_noalloc: assemble first");
  if (k < 1 || k > kNoAllocMaxK)
    fail(GB_ERR_INVALID_ARG, "gb_dnu_noalloc: k must be in [1, 32], the size of its static scratch");
  if (!lam || !x || !out) fail(GB_ERR_INVALID_ARG, "gb_dnu_noalloc: null pointer argument");
  const int grid = grid_cap(c.n_u * 8);
  if ((size_t)grid * k + 64 > kNoAllocDoubles) fail(GB_ERR_INVALID_ARG, "gb_dnu_noalloc: launch exceeds static scratch");
  double* scratch = noalloc_scratch();
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);  // scratch[0]
  double* res = scratch + 32;                                 // scratch[32 .. 32+k)
  double* partial = scratch + 64;                             // [k][grid] partial sums
  Args a = make_args(c, nullptr, 1);
  GBS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), c.stream));
  k_dnu<<<grid, kBlock, 0, c.stream>>>(a, k, lam, x, partial, counter, res);
  GBS_CUDA(cudaGetLastError());
  GBS_CUDA(cudaMemcpyAsync(out, res, sizeof(double) * k, cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace gbs
