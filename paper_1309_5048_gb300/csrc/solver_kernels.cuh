// solver_kernels.cuh -- kernels of the preconditioned MINRES solve (included by solver.cu only).
//
// Sec. 5: MINRES on K x = b, K = [A_h B^T; B 0], with the block-diagonal
// preconditioner M = diag(M_A, M_Q) (eq. general_precond_M): M_A^{-1} r is a
// relaxed inner conjugate-gradient solve with A_h preconditioned by IC(0)
// (Sec. 6.4, "PCG(A)") or by its diagonal, or Diag(A_h); M_Q = Diag(Q_nu)
// with Q_nu = Q / (2 nu) (Sec. 5.1), or a CG solve with Q_nu preconditioned by
// the exact IC(0) factor of Q or by its diagonal.
// MINRES is the Lanczos process in the M^{-1} inner product with a QR
// factorisation of the tridiagonal matrix by Givens rotations (eq.
// opt_condition, eq. linsys_precond); |eta| tracks ||r||_{M^{-1}}.
//
// All arithmetic runs in the kernels below; the host only launches them.
// Every reduction is written as per-block partials plus a last-block
// epilogue that sums them in a fixed order and performs the scalar part of
// the recurrence, so no scalar ever travels to the host inside a solve and
// results do not depend on timing.  k right-hand sides run together in an
// interleaved [n][K] layout; each keeps its own scalars and stops on its own
// (masked), so every column follows the arithmetic of its own solve.
#include <cmath>
#include <cstring>
#include <vector>

#include "gbs_device.cuh"
#include "gbs_internal.h"

namespace gbs {

namespace {

constexpr int kRB = 1216;  // max blocks of the reduction kernels: 152 SMs x 8 blocks of 256 threads
constexpr int kSellwPF = 12;      // slots per lane loaded before the wait by k_trsv_level_sellw (layout 9; 18 on one-warp levels)
constexpr int kSellwLitePF = 4;   // the same, light forms (layouts 11-14, 16, 17; 18 on the other levels)
constexpr int kSellwLite2PF = 2;  // the same, lightest form (layout 15)
constexpr int kTmaCap = (kBlock / 32) * 32 * kTmaPF;      // slots of one TMA stage (8 slices x 32 rows x kTmaPF)
constexpr long long kTmaWaitPolls = 1LL << 26;            // bound on the polls of one stage wait
constexpr unsigned long long kTmaWaitNs = 2000000000ULL;  // and on its wall time (2 s)

// Device view of a SELL-32 matrix copy (see Sell in gbs_internal.h).
struct SellView {
  const int32_t *off, *row0, *rowlen, *col;
  const double* val;
  const float* val32;
  int nslices;
};

struct Args {
  int n_u, n_p, k;
  // matrices (internal numbering)
  const int32_t *A_ptr, *A_col;
  const double* A_val;
  const float* A_val32;
  const int32_t *L_ptr, *L_col;
  const double *L_val, *L_inv;
  const float *L_val32, *L_inv32;
  const int32_t *U_ptr, *U_col;
  const double* U_val;
  const float* U_val32;
  const int32_t *B_ptr, *B_col, *Bt_ptr, *Bt_col;
  const double *B_val, *Bt_val;
  const double *Qdiag, *wmean;
  const int32_t* order;
  double nu;
  // workspace
  double *x, *V0, *V1, *V2, *Z0, *Z1, *W0, *W1, *W2, *q, *b;
  void *cg_x, *cg_r, *cg_z, *cg_y, *cg_p, *cg_q;
  double* S;
  int* flag;
  int* jcur;
  const int32_t* forced;
  int nforced;
  double tol, inner_tol;
  int max_outer, max_inner;
  double* partial;
  unsigned* counter;
  cudaGraphConditionalHandle h_outer, h_inner;
  int use_handles;
  SellView sA, sL, sU;  // SELL-32 copies used by the single-RHS variants
  // pressure block: GB_PRESSURE_DIAG or GB_PRESSURE_PCG (CG on Q with the
  // exact IC(0) factor L1 x L1 [x L1] of Q, natural numbering)
  int pressure_block;
  int dim, qm, qp;  // pressure functions per direction m = N + p - 1; band p of L1
  const int32_t *Q_ptr, *Q_col;
  const double* Q_val;
  const float* Q_val32;
  const double* l1;
  const float* l1_32;
  void *qcg_x, *qcg_r, *qcg_z, *qcg_p, *qcg_q;
  const int32_t* forced_q;
  int nforced_q;
  cudaGraphConditionalHandle h_qinner;
  // velocity block (GB_VELOCITY_*), diagonal positions of A (internal rows)
  int velocity_block;
  const int32_t* A_diag;
  // stopping rule (GB_STOP_*): the 2-norm residual r_j and the products
  // K w_j (three rotating buffers, like w) of its recurrence
  int stop_rule;
  double *R, *KW0, *KW1, *KW2;
  // Lanczos tridiagonal record, per RHS t: delta_j at lz[t * lz_cap + j - 1],
  // gamma_j at lz[(K + t) * lz_cap + j - 1]
  double* lz;
  int lz_cap;
  // device error word: set to 1 by a kernel whose bounded wait ran out
  int* dev_status;
};

// The two inner CG solves: SYS 0 on A_h (velocity block, Sec. 5.1 "PCG(A)"),
// SYS 1 on Q (pressure block, Sec. 6.4 "PCG(Q)"): scalar fields, vectors,
// matrix, replay counts and loop control of each.
template <int SYS>
struct CgSys {
  static constexpr int RHO = SYS ? S_Q_RHO : S_RHO;
  static constexpr int ALPHA = SYS ? S_Q_ALPHA : S_ALPHA;
  static constexpr int BNORM = SYS ? S_Q_BNORM : S_CG_BNORM;
  static constexpr int RNORM = SYS ? S_Q_RNORM : S_RNORM;
  static constexpr int ITS = SYS ? S_Q_ITS : S_CG_ITS;
  static constexpr int ACTIVE = SYS ? S_Q_ACTIVE : S_CG_ACTIVE;
  static constexpr int TARGET = SYS ? S_Q_TARGET : S_CG_TARGET;
  static constexpr int TOTAL = SYS ? S_Q_TOTAL : S_INNER_TOTAL;
  static constexpr int MAX = SYS ? S_Q_MAX : S_INNER_MAX;
  static constexpr int FLAG = SYS ? 3 : 1;  // index in Args::flag of "any active"
  __device__ static int n(const Args& a) { return SYS ? a.n_p : a.n_u; }
  __device__ static void* x(const Args& a) { return SYS ? a.qcg_x : a.cg_x; }
  __device__ static void* r(const Args& a) { return SYS ? a.qcg_r : a.cg_r; }
  __device__ static void* z(const Args& a) { return SYS ? a.qcg_z : a.cg_z; }
  __device__ static void* p(const Args& a) { return SYS ? a.qcg_p : a.cg_p; }
  __device__ static void* q(const Args& a) { return SYS ? a.qcg_q : a.cg_q; }
  __device__ static const int32_t* ptr(const Args& a) { return SYS ? a.Q_ptr : a.A_ptr; }
  __device__ static const int32_t* col(const Args& a) { return SYS ? a.Q_col : a.A_col; }
  __device__ static const double* val(const Args& a) { return SYS ? a.Q_val : a.A_val; }
  __device__ static const float* val32(const Args& a) { return SYS ? a.Q_val32 : a.A_val32; }
  __device__ static cudaGraphConditionalHandle handle(const Args& a) { return SYS ? a.h_qinner : a.h_inner; }
};

template <int K>
struct Map {
  static constexpr int G = (K == 1) ? 8 : K;  // lanes per row
  static constexpr int RPW = 32 / G;          // rows per warp
};

__device__ __forceinline__ double& SF(const Args& a, int f, int t, int K) { return a.S[f * K + t]; }

__device__ __forceinline__ double* Vbuf(const Args& a, int i) {
  i %= 3;
  return i == 0 ? a.V0 : (i == 1 ? a.V1 : a.V2);
}
__device__ __forceinline__ double* Wbuf(const Args& a, int i) {
  i %= 3;
  return i == 0 ? a.W0 : (i == 1 ? a.W1 : a.W2);
}
__device__ __forceinline__ double* Zbuf(const Args& a, int i) { return (i % 2) == 0 ? a.Z0 : a.Z1; }
__device__ __forceinline__ double* KWbuf(const Args& a, int i) {
  i %= 3;
  return i == 0 ? a.KW0 : (i == 1 ? a.KW1 : a.KW2);
}

template <class T>
__device__ __forceinline__ const T* pick(const double* d, const float* f);
template <>
__device__ __forceinline__ const double* pick<double>(const double* d, const float*) {
  return d;
}
template <>
__device__ __forceinline__ const float* pick<float>(const double*, const float* f) {
  return f;
}

// ---------------------------------------------------------------- gather --
// b (internal layout) from rhs [k][n] (natural numbering); zero the MINRES
// vectors; ||b||^2, a finiteness check and the consistency condition
// 1^T g_p = 0 per RHS (K is singular with kernel [0; 1]: B^T 1 = 0 because
// the pressure B-splines sum to one and the velocity has zero normal trace);
// scalar initialisation.  A RHS with |1^T g_p| > 1e-10 sqrt(n_p) ||g_p|| is
// not solved and reports an invalid argument.
template <int K>
__global__ void k_gather(Args a, const double* __restrict__ rhs) {
  const int n = a.n_u + a.n_p;
  double vals[4] = {0.0, 0.0, 0.0, 0.0};  // ||b||^2, nonfinite count, 1^T g_p, ||g_p||^2
  const int t = threadIdx.x % K;
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) / K; r < n; r += stride) {
    double v = 0.0;
    if (t < a.k) {
      const int nat = r < a.n_u ? a.order[r] : r;
      v = rhs[(size_t)t * n + nat];
    }
    const size_t idx = (size_t)r * K + t;
    a.b[idx] = v;
    a.x[idx] = 0.0;
    a.V0[idx] = 0.0;
    a.W0[idx] = 0.0;
    a.W1[idx] = 0.0;
    if (a.stop_rule == GB_STOP_RESIDUAL) {
      a.R[idx] = v;  // r_0 = b - K x_0 with x_0 = 0
      a.KW0[idx] = 0.0;
      a.KW1[idx] = 0.0;
    }
    vals[0] += v * v;
    if (!isfinite(v)) vals[1] += 1.0;
    if (r >= a.n_u) {
      vals[2] += v;
      vals[3] += v * v;
    }
  }
  block_partials<K, 4>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K * 4];
    finalize_partials<K, 4>(a.partial, gridDim.x, tot);
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      for (int f = 0; f < S_NFIELDS; ++f) SF(a, f, s, K) = 0.0;
      const double bn = sqrt(tot[s * 4 + 0]);
      SF(a, S_BNORM, s, K) = bn;
      SF(a, S_NONFINITE, s, K) = tot[s * 4 + 1] > 0 ? 1.0 : 0.0;
      const bool bad_p = fabs(tot[s * 4 + 2]) > 1e-10 * sqrt((double)a.n_p) * sqrt(tot[s * 4 + 3]);
      SF(a, S_INCONSISTENT, s, K) = (s < a.k && bad_p) ? 1.0 : 0.0;
      const bool live = s < a.k && bn > 0.0 && tot[s * 4 + 1] == 0.0 && !bad_p;
      SF(a, S_OUTER_ACTIVE, s, K) = live ? 1.0 : 0.0;
      SF(a, S_C, s, K) = 1.0;
      SF(a, S_C_PREV, s, K) = 1.0;
      SF(a, S_GAMMA_PREV, s, K) = 1.0;
    }
    if (threadIdx.x == 0) {
      *a.jcur = 0;
      *a.counter = 0;
    }
  }
}

// ------------------------------------------------------------ K-apply ----
// y = K z_j for the live RHS, q = y / gamma_j (= K times the normalised z_j),
// delta_j = q^T (z_j / gamma_j) = y^T z_j / gamma_j^2.
template <int K>
__global__ void k_stokes_apply(Args a) {
  using M = Map<K>;
  const int j = *a.jcur;
  const double* __restrict__ z = Zbuf(a, j);
  const int n = a.n_u + a.n_p;
  const int lane = threadIdx.x & 31;
  const int g = lane % M::G;
  const int t = (K == 1) ? 0 : g;
  const bool live = SF(a, S_OUTER_ACTIVE, t, K) != 0.0;
  const double ig = live ? 1.0 / SF(a, S_GAMMA, t, K) : 0.0;
  double vals[1] = {0.0};
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / M::G;
  const int ng = (gridDim.x * blockDim.x) / M::G;
  for (int r = gid; r < n; r += ng) {
    double y = 0.0;
    if (r < a.n_u) {
      if (K == 1) {
        for (int e = a.A_ptr[r] + g; e < a.A_ptr[r + 1]; e += M::G) y += a.A_val[e] * z[a.A_col[e]];
        for (int e = a.Bt_ptr[r] + g; e < a.Bt_ptr[r + 1]; e += M::G)
          y += a.Bt_val[e] * z[a.n_u + a.Bt_col[e]];
      } else {
        for (int e = a.A_ptr[r]; e < a.A_ptr[r + 1]; ++e) y += a.A_val[e] * z[(size_t)a.A_col[e] * K + t];
        for (int e = a.Bt_ptr[r]; e < a.Bt_ptr[r + 1]; ++e)
          y += a.Bt_val[e] * z[(size_t)(a.n_u + a.Bt_col[e]) * K + t];
      }
    } else {
      const int kr = r - a.n_u;
      if (K == 1) {
        for (int e = a.B_ptr[kr] + g; e < a.B_ptr[kr + 1]; e += M::G) y += a.B_val[e] * z[a.B_col[e]];
      } else {
        for (int e = a.B_ptr[kr]; e < a.B_ptr[kr + 1]; ++e) y += a.B_val[e] * z[(size_t)a.B_col[e] * K + t];
      }
    }
    if (K == 1) y = group_sum<M::G>(y);
    if (live && (K > 1 || g == 0)) {
      const size_t idx = (size_t)r * K + t;
      a.q[idx] = y * ig;
      vals[0] += y * z[idx];
    }
  }
  block_partials<K, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K];
    finalize_partials<K, 1>(a.partial, gridDim.x, tot);
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      if (SF(a, S_OUTER_ACTIVE, s, K) != 0.0) {
        const double gm = SF(a, S_GAMMA, s, K);
        SF(a, S_DELTA, s, K) = tot[s] / (gm * gm);
      }
    }
    if (threadIdx.x == 0) *a.counter = 0;
  }
}

// ----------------------------------------------------------- Lanczos -----
// v_{j+1} = q - (delta_j/gamma_j) v_j - (gamma_j/gamma_{j-1}) v_{j-1}
// (j = 0: v_1 = b).  The velocity block of z_{j+1} = M^{-1} v_{j+1} is
// v_u / diag(A_h) (Diag(A) block), or starts the inner CG with b = r =
// v_{j+1,u}, x = 0.  The pressure block is 2 nu v_p / diag(Q) (Diag(Q_nu)),
// or starts the pressure CG on Q with b = r = v_{j+1,p}, x = 0 (CG blocks;
// z_p = 2 nu x is taken in k_gamma).  Epilogue: ||b|| and the CG state of
// each block per RHS.
template <int K, class T>
__global__ void k_lanczos(Args a) {
  const int j = *a.jcur;
  const int n = a.n_u + a.n_p;
  double* __restrict__ vn = Vbuf(a, j + 1);
  const double* __restrict__ vc = Vbuf(a, j);
  const double* __restrict__ vp = Vbuf(a, j + 2);  // (j - 1) mod 3
  double* __restrict__ zn = Zbuf(a, j + 1);
  T* __restrict__ r_cg = (T*)a.cg_r;
  T* __restrict__ x_cg = (T*)a.cg_x;
  T* __restrict__ r_q = (T*)a.qcg_r;
  T* __restrict__ x_q = (T*)a.qcg_x;
  const bool pcg_q = a.pressure_block != GB_PRESSURE_DIAG;
  const int t = threadIdx.x % K;
  const bool live = SF(a, S_OUTER_ACTIVE, t, K) != 0.0;
  double c1 = 0.0, c2 = 0.0;
  if (live && j > 0) {
    const double gm = SF(a, S_GAMMA, t, K);
    c1 = SF(a, S_DELTA, t, K) / gm;
    c2 = gm / SF(a, S_GAMMA_PREV, t, K);
  }
  double vals[2] = {0.0, 0.0};  // ||v_u||^2, ||v_p||^2
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) / K; r < n; r += stride) {
    if (!live) continue;
    const size_t idx = (size_t)r * K + t;
    const double v = (j == 0) ? a.b[idx] : a.q[idx] - c1 * vc[idx] - c2 * vp[idx];
    vn[idx] = v;
    if (r < a.n_u) {
      if (a.velocity_block == GB_VELOCITY_DIAG) {
        zn[idx] = v / a.A_val[a.A_diag[r]];
      } else {
        r_cg[idx] = (T)v;
        x_cg[idx] = (T)0;
        vals[0] += v * v;
      }
    } else if (pcg_q) {
      const size_t iq = (size_t)(r - a.n_u) * K + t;
      r_q[iq] = (T)v;
      x_q[iq] = (T)0;
      vals[1] += v * v;
    } else {
      zn[idx] = 2.0 * a.nu * v / a.Qdiag[r - a.n_u];
    }
  }
  block_partials<K, 2>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K * 2];
    finalize_partials<K, 2>(a.partial, gridDim.x, tot);
    int any = 0, anyq = 0;
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      SF(a, S_CG_ACTIVE, s, K) = 0.0;
      SF(a, S_Q_ACTIVE, s, K) = 0.0;
      if (SF(a, S_OUTER_ACTIVE, s, K) != 0.0) {
        const int app = (int)SF(a, S_APPS, s, K);
        const double bn = sqrt(tot[s * 2 + 0]);
        SF(a, S_CG_BNORM, s, K) = bn;
        SF(a, S_CG_ITS, s, K) = 0.0;
        double target = -1.0;
        if (a.forced) target = app < a.nforced ? (double)a.forced[app] : 0.0;
        SF(a, S_CG_TARGET, s, K) = target;
        SF(a, S_APPS, s, K) += 1.0;
        const bool act = bn > 0.0 && target != 0.0;
        SF(a, S_CG_ACTIVE, s, K) = act ? 1.0 : 0.0;
        any = act;
        if (pcg_q) {
          const double bq = sqrt(tot[s * 2 + 1]);
          SF(a, S_Q_BNORM, s, K) = bq;
          SF(a, S_Q_ITS, s, K) = 0.0;
          double tq = -1.0;
          if (a.forced_q) tq = app < a.nforced_q ? (double)a.forced_q[app] : 0.0;
          SF(a, S_Q_TARGET, s, K) = tq;
          const bool actq = bq > 0.0 && tq != 0.0;
          SF(a, S_Q_ACTIVE, s, K) = actq ? 1.0 : 0.0;
          anyq = actq;
        }
      }
    }
    any = __syncthreads_or(any);
    anyq = __syncthreads_or(anyq);
    if (threadIdx.x == 0) {
      a.flag[1] = any;
      a.flag[3] = anyq;
      if (a.use_handles) {
        if (a.velocity_block != GB_VELOCITY_DIAG) cudaGraphSetConditional(a.h_inner, any ? 1u : 0u);
        if (pcg_q) cudaGraphSetConditional(a.h_qinner, anyq ? 1u : 0u);
      }
      *a.counter = 0;
    }
  }
}

// ---------------------------------------------------------- gamma/Givens --
// z_{j+1,u} = x_cg (the inner CG result), z_{j+1,p} = 2 nu x_q with the
// IC(0)-PCG pressure block; gamma_{j+1}^2 = z_{j+1}^T v_{j+1}.
// j = 0: initial recurrence values.  j >= 1: Givens rotation of the new
// column of the tridiagonal matrix, coefficient of the x update, new eta,
// the record of T_j, and with the estimate stopping rule the convergence test
// |eta| / gamma_1 <= tol (the 2-norm rule is tested in k_update).
template <int K, class T>
__global__ void k_gamma(Args a) {
  const int j = *a.jcur;
  const int n = a.n_u + a.n_p;
  const double* __restrict__ vn = Vbuf(a, j + 1);
  double* __restrict__ zn = Zbuf(a, j + 1);
  const T* __restrict__ x_cg = (const T*)a.cg_x;
  const int t = threadIdx.x % K;
  const bool live = SF(a, S_OUTER_ACTIVE, t, K) != 0.0;
  double vals[1] = {0.0};
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) / K; r < n; r += stride) {
    if (!live) continue;
    const size_t idx = (size_t)r * K + t;
    double z;
    if (r < a.n_u) {
      if (a.velocity_block == GB_VELOCITY_DIAG) {
        z = zn[idx];
      } else {
        z = (double)x_cg[idx];
        zn[idx] = z;
      }
    } else if (a.pressure_block != GB_PRESSURE_DIAG) {
      z = 2.0 * a.nu * (double)((const T*)a.qcg_x)[(size_t)(r - a.n_u) * K + t];
      zn[idx] = z;
    } else {
      z = zn[idx];
    }
    vals[0] += z * vn[idx];
  }
  block_partials<K, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K];
    finalize_partials<K, 1>(a.partial, gridDim.x, tot);
    int any = 0;
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      if (SF(a, S_OUTER_ACTIVE, s, K) != 0.0) {
        const double gg = tot[s];
        bool stop = false;
        if (!isfinite(gg)) {
          SF(a, S_NONFINITE, s, K) = 1.0;
          stop = true;
        } else if (gg < 0.0) {
          SF(a, S_STATUS, s, K) = 2.0;  // preconditioner not positive
          stop = true;
        }
        const double gnext = stop ? 0.0 : sqrt(gg);
        if (j == 0) {
          SF(a, S_GAMMA, s, K) = gnext;
          SF(a, S_GAMMA1, s, K) = gnext;
          SF(a, S_ETA, s, K) = gnext;
          SF(a, S_XCOEF, s, K) = 0.0;
          if (a.lz && a.lz_cap > 0) a.lz[(size_t)(K + s) * a.lz_cap] = gnext;  // gamma_1
          if (stop || gnext == 0.0) {
            SF(a, S_OUTER_ACTIVE, s, K) = 0.0;
          }
        } else {
          const double gm = SF(a, S_GAMMA, s, K), gp = SF(a, S_GAMMA_PREV, s, K);
          const double dl = SF(a, S_DELTA, s, K);
          const double c = SF(a, S_C, s, K), cp = SF(a, S_C_PREV, s, K);
          const double sn = SF(a, S_S, s, K), sp = SF(a, S_S_PREV, s, K);
          (void)gp;
          if (a.lz && j < a.lz_cap) {  // T_j: delta_j, gamma_{j+1}
            a.lz[(size_t)s * a.lz_cap + j - 1] = dl;
            a.lz[(size_t)(K + s) * a.lz_cap + j] = gnext;
          }
          const double a0 = c * dl - cp * sn * gm;
          const double a1 = sqrt(a0 * a0 + gnext * gnext);
          const double a2 = sn * dl + cp * c * gm;
          const double a3 = sp * gm;
          const double cn = a0 / a1, snn = gnext / a1;
          const double eta = SF(a, S_ETA, s, K);
          SF(a, S_A1, s, K) = a1;
          SF(a, S_A2, s, K) = a2;
          SF(a, S_A3, s, K) = a3;
          SF(a, S_XCOEF, s, K) = cn * eta;
          SF(a, S_ETA, s, K) = -snn * eta;
          SF(a, S_C_PREV, s, K) = c;
          SF(a, S_C, s, K) = cn;
          SF(a, S_S_PREV, s, K) = sn;
          SF(a, S_S, s, K) = snn;
          SF(a, S_GAMMA_PREV, s, K) = gm;
          SF(a, S_GAMMA, s, K) = gnext;
          SF(a, S_OUTER_ITS, s, K) = j;
          const double rel = fabs(-snn * eta) / SF(a, S_GAMMA1, s, K);
          SF(a, S_RELRES, s, K) = rel;
          // S_OUTER_ACTIVE stays set until k_update has applied this step; with
          // the residual rule k_update decides convergence
          const bool est_conv = a.stop_rule == GB_STOP_ESTIMATE && rel <= a.tol;
          SF(a, S_STATUS, s, K) = stop ? SF(a, S_STATUS, s, K) : (est_conv ? 0.0 : 1.0);
          if (!isfinite(a1) || !isfinite(rel)) SF(a, S_NONFINITE, s, K) = 1.0;
        }
      }
      any = SF(a, S_OUTER_ACTIVE, s, K) != 0.0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
      if (j == 0) {
        *a.jcur = 1;
        a.flag[0] = any;
        if (a.use_handles) cudaGraphSetConditional(a.h_outer, any ? 1u : 0u);
      }
      *a.counter = 0;
    }
  }
}

// w_{j+1} = (z_j / gamma_j - a3 w_{j-1} - a2 w_j) / a1;  x += (c_{j+1} eta_j) w_{j+1}.
// gamma_j here is the value before k_gamma advanced it, i.e. S_GAMMA_PREV.
// With the residual rule the same recurrence runs on K w (q = K z_j / gamma_j
// from k_stokes_apply): K w_{j+1} = (q - a3 K w_{j-1} - a2 K w_j) / a1, and
// r_j = r_{j-1} - (c_{j+1} eta_j) K w_{j+1} = b - K x_j; ||r_j||^2 is reduced.
// Epilogue: retire converged RHS (||r_j|| <= tol ||b|| or the estimate test
// of k_gamma), advance j, set the outer loop condition.
template <int K>
__global__ void k_update(Args a) {
  const int j = *a.jcur;
  const int n = a.n_u + a.n_p;
  const double* __restrict__ zc = Zbuf(a, j);
  const double* __restrict__ wp = Wbuf(a, j + 2);  // w_{j-1}
  const double* __restrict__ wc = Wbuf(a, j);      // w_j
  double* __restrict__ wn = Wbuf(a, j + 1);        // w_{j+1}
  const int t = threadIdx.x % K;
  const bool live = SF(a, S_OUTER_ACTIVE, t, K) != 0.0;
  double ig = 0, a1i = 0, a2 = 0, a3 = 0, xc = 0;
  if (live) {
    ig = 1.0 / SF(a, S_GAMMA_PREV, t, K);
    a1i = 1.0 / SF(a, S_A1, t, K);
    a2 = SF(a, S_A2, t, K);
    a3 = SF(a, S_A3, t, K);
    xc = SF(a, S_XCOEF, t, K);
  }
  const bool resid = a.stop_rule == GB_STOP_RESIDUAL;
  const double* __restrict__ kwp = KWbuf(a, j + 2);
  const double* __restrict__ kwc = KWbuf(a, j);
  double* __restrict__ kwn = KWbuf(a, j + 1);
  double vals[1] = {0.0};
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) / K; r < n; r += stride) {
    if (!live) continue;
    const size_t idx = (size_t)r * K + t;
    const double w = (zc[idx] * ig - a3 * wp[idx] - a2 * wc[idx]) * a1i;
    wn[idx] = w;
    a.x[idx] += xc * w;
    if (resid) {
      const double kw = (a.q[idx] - a3 * kwp[idx] - a2 * kwc[idx]) * a1i;
      kwn[idx] = kw;
      const double rv = a.R[idx] - xc * kw;
      a.R[idx] = rv;
      vals[0] += rv * rv;
    }
  }
  if (resid) block_partials<K, 1>(vals, a.partial);  // uniform over the grid
  if (last_block(a.counter)) {
    __shared__ double tot[K];
    if (resid) finalize_partials<K, 1>(a.partial, gridDim.x, tot);
    int any = 0;
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      if (SF(a, S_OUTER_ACTIVE, s, K) != 0.0) {
        if (resid && SF(a, S_STATUS, s, K) == 1.0) {
          const double rel2 = sqrt(tot[s]) / SF(a, S_BNORM, s, K);
          if (rel2 <= a.tol) SF(a, S_STATUS, s, K) = 0.0;
          if (!isfinite(rel2)) SF(a, S_NONFINITE, s, K) = 1.0;
        }
        const bool conv = SF(a, S_STATUS, s, K) != 1.0;
        const bool cap = j >= a.max_outer;
        const bool bad = SF(a, S_NONFINITE, s, K) != 0.0;
        if (conv || cap || bad) SF(a, S_OUTER_ACTIVE, s, K) = 0.0;
      }
      any = SF(a, S_OUTER_ACTIVE, s, K) != 0.0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
      *a.jcur = j + 1;
      a.flag[0] = any;
      if (a.use_handles) cudaGraphSetConditional(a.h_outer, any ? 1u : 0u);
      *a.counter = 0;
    }
  }
}

// ------------------------------------------------------------- inner CG --
// q = A p (SYS 0) or q = Q p (SYS 1) and p^T q; epilogue alpha = rho / p^T q.
template <int K, class T, int SYS = 0>
__global__ void k_cg_spmv(Args a) {
  using M = Map<K>;
  using C = CgSys<SYS>;
  const T* __restrict__ val = pick<T>(C::val(a), C::val32(a));
  const int32_t* __restrict__ mptr = C::ptr(a);
  const int32_t* __restrict__ mcol = C::col(a);
  const int nrows = C::n(a);
  const T* __restrict__ p = (const T*)C::p(a);
  T* __restrict__ q = (T*)C::q(a);
  const int lane = threadIdx.x & 31;
  const int g = lane % M::G;
  const int t = (K == 1) ? 0 : g;
  const bool live = SF(a, C::ACTIVE, t, K) != 0.0;
  double vals[1] = {0.0};
  if (K == 1 && !live) {
    // nothing to do for this RHS; still take part in the reduction
  } else {
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / M::G;
    const int ng = (gridDim.x * blockDim.x) / M::G;
    for (int r = gid; r < nrows; r += ng) {
      T y = 0;
      if (K == 1) {
        for (int e = mptr[r] + g; e < mptr[r + 1]; e += M::G) y += val[e] * p[mcol[e]];
        if (sizeof(T) == 8) y = (T)group_sum<M::G>((double)y);
        else y = (T)group_sumf<M::G>((float)y);
      } else {
        for (int e = mptr[r]; e < mptr[r + 1]; ++e) y += val[e] * p[(size_t)mcol[e] * K + t];
      }
      if (live && (K > 1 || g == 0)) {
        const size_t idx = (size_t)r * K + t;
        q[idx] = y;
        vals[0] += (double)y * (double)p[idx];
      }
    }
  }
  block_partials<K, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K];
    finalize_partials<K, 1>(a.partial, gridDim.x, tot);
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      if (SF(a, C::ACTIVE, s, K) != 0.0) SF(a, C::ALPHA, s, K) = SF(a, C::RHO, s, K) / tot[s];
    }
    if (threadIdx.x == 0) *a.counter = 0;
  }
}

// x += alpha p, r -= alpha q, ||r||^2; epilogue: stopping test
// ||r|| <= inner_tol ||b|| or its == max_inner (or the replayed count).
template <int K, class T, int SYS = 0>
__global__ void k_cg_axpy(Args a) {
  using C = CgSys<SYS>;
  const T* __restrict__ p = (const T*)C::p(a);
  const T* __restrict__ q = (const T*)C::q(a);
  T* __restrict__ x = (T*)C::x(a);
  T* __restrict__ r = (T*)C::r(a);
  const int t = threadIdx.x % K;
  const bool live = SF(a, C::ACTIVE, t, K) != 0.0;
  const T alpha = live ? (T)SF(a, C::ALPHA, t, K) : (T)0;
  double vals[1] = {0.0};
  T acc = 0;
  const int stride = (gridDim.x * blockDim.x) / K;
  if (live) {
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / K; i < C::n(a); i += stride) {
      const size_t idx = (size_t)i * K + t;
      x[idx] += alpha * p[idx];
      const T rv = r[idx] - alpha * q[idx];
      r[idx] = rv;
      acc += rv * rv;
    }
  }
  vals[0] = (double)acc;
  block_partials<K, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K];
    finalize_partials<K, 1>(a.partial, gridDim.x, tot);
    int any = 0;
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      if (SF(a, C::ACTIVE, s, K) != 0.0) {
        const double its = SF(a, C::ITS, s, K) + 1.0;
        SF(a, C::ITS, s, K) = its;
        SF(a, C::TOTAL, s, K) += 1.0;
        const double rn = sqrt(tot[s]);
        SF(a, C::RNORM, s, K) = rn;
        const double target = SF(a, C::TARGET, s, K);
        bool stop;
        if (target >= 0.0) stop = its >= target;
        else stop = rn <= a.inner_tol * SF(a, C::BNORM, s, K) || its >= a.max_inner || !isfinite(rn);
        if (stop) {
          SF(a, C::ACTIVE, s, K) = 0.0;
          if (its > SF(a, C::MAX, s, K)) SF(a, C::MAX, s, K) = its;
        }
      }
      any = SF(a, C::ACTIVE, s, K) != 0.0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
      a.flag[C::FLAG] = any;
      if (a.use_handles) cudaGraphSetConditional(C::handle(a), any ? 1u : 0u);
      *a.counter = 0;
    }
  }
}

// One level of a triangular solve, internal rows [r0, r1):
//   forward  (L):   y_i = (r_i - sum_{j<i} L_ij y_j) / L_ii
//   backward (L^T): z_i = (y_i - sum_{j>i} L_ji z_j) / L_ii
// The rows of a level depend only on rows of earlier (forward) or later
// (backward) levels.  Levels are launched back to back with programmatic
// dependent launch: each level kernel lets the next one start at once; the
// next one loads what does not depend on earlier kernels (row pointers,
// column indices, factor values, 1/L_ii) and then waits for its predecessor
// grid (cudaGridDependencySynchronize) before it reads the right-hand side,
// the CG state and the solution entries it depends on.  A level then costs
// about one memory round trip for those entries plus its stores, instead of
// a launch and three dependent round trips.
template <int K, class T, bool FWD>
__global__ void __launch_bounds__(kBlock) k_trsv_level(Args a, int r0, int r1) {
  using M = Map<K>;
  constexpr int PF = 6;  // entries per lane fetched before the wait
  constexpr int STEP = (K == 1) ? M::G : 1;
  cudaTriggerProgrammaticLaunchCompletion();
  const int32_t* __restrict__ ptr = FWD ? a.L_ptr : a.U_ptr;
  const int32_t* __restrict__ col = FWD ? a.L_col : a.U_col;
  const T* __restrict__ val = FWD ? pick<T>(a.L_val, a.L_val32) : pick<T>(a.U_val, a.U_val32);
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  const int lane = threadIdx.x & 31;
  const int g = lane % M::G;
  const int t = (K == 1) ? 0 : g;
  const int row = r0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) / M::G);
  const bool act = row < r1;  // uniform over a lane group
  int eb = 0, ee = 0;
  int cc[PF];
  T v[PF];
  T ii = T(0);
  if (act) {
    eb = ptr[row] + ((K == 1) ? g : 0);
    ee = ptr[row + 1];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int e = eb + u * STEP;
      cc[u] = e < ee ? col[e] : 0;
      v[u] = e < ee ? val[e] : T(0);
    }
    ii = inv[row];
  }
  cudaGridDependencySynchronize();
  if (!act) return;  // uniform over a lane group
  // the CG state flag is loaded together with the solution entries and only
  // decides the store (uniform over a lane group)
  const bool live = SF(a, S_CG_ACTIVE, t, K) != 0.0;
  T s = 0;
#pragma unroll
  for (int u = 0; u < PF; ++u)
    if (eb + u * STEP < ee) s += v[u] * __ldcg(out + ((K == 1) ? (size_t)cc[u] : (size_t)cc[u] * K + t));
  for (int e = eb + PF * STEP; e < ee; e += STEP)
    s += val[e] * __ldcg(out + ((K == 1) ? (size_t)col[e] : (size_t)col[e] * K + t));
  if (K == 1) {
    if (sizeof(T) == 8) s = (T)group_sum<M::G>((double)s);
    else s = (T)group_sumf<M::G>((float)s);
  }
  const size_t ridx = (K == 1) ? (size_t)row : (size_t)row * K + t;
  if (live && (K > 1 || g == 0)) out[ridx] = (__ldcg(rhs + ridx) - s) * ii;
}

// ---- staged batched variant (K = 8 or 32 right-hand sides) ---------------
// One level for k right-hand sides (same recurrences as k_trsv_level), K lanes
// per row (lane t = right-hand side t).  Before the wait for the previous
// level each row's column indices and factor values (up to capr of them) are
// copied to shared memory, so that after the wait every lane can issue the
// loads of its solution entries x[col * K + t] -- one coalesced K-wide segment
// per entry -- 16 at a time without waiting for the indices; entries past
// capr are read from global memory.  Same summation order as k_trsv_level.
// Dynamic shared memory: T val[kBlock / K][capr], int col[kBlock / K][capr].
template <int K, class T, bool FWD>
__global__ void __launch_bounds__(kBlock) k_trsv_level_batch(Args a, int r0, int r1, int capr) {
  constexpr int RPB = kBlock / K;  // rows per block
  constexpr int CH = 16;           // solution loads in flight per lane
  extern __shared__ __align__(16) unsigned char batch_smem[];
  cudaTriggerProgrammaticLaunchCompletion();
  const int32_t* __restrict__ ptr = FWD ? a.L_ptr : a.U_ptr;
  const int32_t* __restrict__ col = FWD ? a.L_col : a.U_col;
  const T* __restrict__ val = FWD ? pick<T>(a.L_val, a.L_val32) : pick<T>(a.U_val, a.U_val32);
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  T* sv = (T*)batch_smem;
  int* sc = (int*)(sv + RPB * capr);
  const int t = threadIdx.x % K, lr = threadIdx.x / K;
  const int row = r0 + blockIdx.x * RPB + lr;
  const bool act = row < r1;  // uniform over a lane group
  int eb = 0, ee = 0, n = 0;
  T ii = T(0);
  T* rv = sv + lr * capr;
  int* rc = sc + lr * capr;
  if (act) {
    eb = ptr[row];
    ee = ptr[row + 1];
    n = min(ee - eb, capr);
    for (int j = t; j < n; j += K) {
      rc[j] = col[eb + j];
      rv[j] = val[eb + j];
    }
    ii = inv[row];
  }
  cudaGridDependencySynchronize();
  __syncthreads();
  if (!act) return;  // uniform over a lane group, after the barrier
  const bool live = SF(a, S_CG_ACTIVE, t, K) != 0.0;  // decides the store only
  T s = 0;
  int j = 0;
  for (; j + CH <= n; j += CH) {
    T xv[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) xv[u] = __ldcg(out + (size_t)rc[j + u] * K + t);
#pragma unroll
    for (int u = 0; u < CH; ++u) s += rv[j + u] * xv[u];
  }
  for (; j < n; ++j) s += rv[j] * __ldcg(out + (size_t)rc[j] * K + t);
  for (int e = eb + n; e < ee; ++e) s += val[e] * __ldcg(out + (size_t)col[e] * K + t);
  const size_t ridx = (size_t)row * K + t;
  if (live) out[ridx] = (__ldcg(rhs + ridx) - s) * ii;
}

// ---- SELL-32 variants (single right-hand side, one thread per row) --------
// The 32 lanes of a warp read 32 consecutive slots, so every load of values
// and column indices is coalesced and no cross-lane reduction is needed (on
// GB300 the shuffle-tree DADDs of the 8-lane CSR form cost as much FP64 issue
// as the useful FMAs).  Each row sums its entries in order.

// q = A p and p^T q; epilogue alpha = rho / p^T q (as k_cg_spmv).
template <class T>
__global__ void __launch_bounds__(kBlock) k_cg_spmv_sell(Args a) {
  const SellView m = a.sA;
  const T* __restrict__ val = pick<T>(m.val, m.val32);
  const T* __restrict__ p = (const T*)a.cg_p;
  T* __restrict__ q = (T*)a.cg_q;
  double vals[1] = {0.0};
  if (SF(a, S_CG_ACTIVE, 0, 1) != 0.0) {
    const int total = m.nslices * 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
      const int s = i >> 5, lane = i & 31;
      const int row = m.row0[s] + lane;
      if (row >= m.row0[s + 1]) continue;
      const int base = m.off[s] + lane, len = m.rowlen[row];
      T y = 0;
      for (int k = 0; k < len; ++k) y += val[base + 32 * k] * p[m.col[base + 32 * k]];
      q[row] = y;
      vals[0] += (double)y * (double)p[row];
    }
  }
  block_partials<1, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[1];
    finalize_partials<1, 1>(a.partial, gridDim.x, tot);
    if (threadIdx.x == 0) {
      if (SF(a, S_CG_ACTIVE, 0, 1) != 0.0) SF(a, S_ALPHA, 0, 1) = SF(a, S_RHO, 0, 1) / tot[0];
      *a.counter = 0;
    }
  }
}

// q = A p and p^T q on the SELL-32 copy with W warps per 32-row slice: warp h
// of a slice sums the slots k = h, h + W, ... of its rows (coalesced loads of
// the same stencil entry of 32 rows), the W partial sums are added in a fixed
// order in shared memory.  More warps in flight than one thread per row when
// rows are long and slices few.  Epilogue as k_cg_spmv.
template <class T, int W>
__global__ void __launch_bounds__(kBlock) k_cg_spmv_sellw(Args a) {
  constexpr int SPB = kBlock / (32 * W);  // slices per block
  static_assert(SPB * 32 * W == kBlock, "block shape");
  __shared__ T part[W][SPB][32];
  const SellView m = a.sA;
  const T* __restrict__ val = pick<T>(m.val, m.val32);
  const T* __restrict__ p = (const T*)a.cg_p;
  T* __restrict__ q = (T*)a.cg_q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = warp % W, ls = warp / W;
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;
  double vals[1] = {0.0};
  for (int s0 = blockIdx.x * SPB; s0 < m.nslices; s0 += gridDim.x * SPB) {  // uniform over the block
    const int s = s0 + ls;
    int row = -1;
    T y = 0;
    if (live && s < m.nslices) {
      row = m.row0[s] + lane;
      if (row < m.row0[s + 1]) {
        const int base = m.off[s] + lane, len = m.rowlen[row];
        for (int k = h; k < len; k += W) y += val[base + 32 * k] * p[m.col[base + 32 * k]];
      } else {
        row = -1;
      }
    }
    part[h][ls][lane] = y;
    __syncthreads();
    if (h == 0 && row >= 0) {
      T t = part[0][ls][lane];
#pragma unroll
      for (int u = 1; u < W; ++u) t += part[u][ls][lane];
      q[row] = t;
      vals[0] += (double)t * (double)p[row];
    }
    __syncthreads();
  }
  block_partials<1, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[1];
    finalize_partials<1, 1>(a.partial, gridDim.x, tot);
    if (threadIdx.x == 0) {
      if (SF(a, S_CG_ACTIVE, 0, 1) != 0.0) SF(a, S_ALPHA, 0, 1) = SF(a, S_RHO, 0, 1) / tot[0];
      *a.counter = 0;
    }
  }
}

// One level of a triangular solve over the slices [s0, s1) of that level
// (same recurrences and the same programmatic-dependent-launch structure as
// k_trsv_level).
template <class T, bool FWD>
__global__ void __launch_bounds__(kBlock) k_trsv_level_sell(Args a, int s0, int s1) {
  constexpr int PF = 8;  // entries per row fetched before the wait
  cudaTriggerProgrammaticLaunchCompletion();
  const SellView m = FWD ? a.sL : a.sU;
  const T* __restrict__ val = pick<T>(m.val, m.val32);
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + (i >> 5), lane = i & 31;
  int row = 0, base = 0, len = 0;
  bool act = s < s1;
  if (act) {
    row = m.row0[s] + lane;
    act = row < m.row0[s + 1];
  }
  int cc[PF];
  T v[PF];
  T ii = T(0);
  if (act) {
    base = m.off[s] + lane;
    len = m.rowlen[row];
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      cc[k] = k < len ? m.col[base + 32 * k] : 0;
      v[k] = k < len ? val[base + 32 * k] : T(0);
    }
    ii = inv[row];
  }
  cudaGridDependencySynchronize();
  if (!act) return;
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;  // decides the store only
  T sum = 0;
#pragma unroll
  for (int k = 0; k < PF; ++k)
    if (k < len) sum += v[k] * __ldcg(out + cc[k]);
  for (int k = PF; k < len; ++k) sum += val[base + 32 * k] * __ldcg(out + m.col[base + 32 * k]);
  if (live) out[row] = (__ldcg(rhs + row) - sum) * ii;
}

// One level of a triangular solve on the SELL-32 copy with W warps per
// 32-row slice (same recurrences as k_trsv_level).  Warp h of a slice owns the
// stencil slots k = h, h + W, ... of its 32 rows; a lane reads the column
// indices and factor values of its slots coalesced (a warp reads one slot of
// 32 neighbouring rows) with the streaming cache hint, so that the factor,
// read once per sweep, does not push the solution vector out of L2, and sums
// value * entry in slot order; the W partial sums of a row are added in warp
// order in shared memory.  One thread per row and lane keeps the FP64 issue
// at one DFMA per entry plus W - 1 DADDs per row, and the prefetched slots'
// FMAs stop at the warp's longest lane (a predicated, fully unrolled loop would issue
// every DFMA, and the FP64 pipe, 2 lanes per clock and SM, is as scarce as HBM
// bandwidth here).  A lane loads its first PF slots before the wait for the
// previous level (the factor does not depend on it), gathers their solution
// entries at once after it, and reads any further slots in a loop.  Three
// prefetch depths: PF = 12 (layout 9, W chosen so that 12 slots cover the
// level's longest row); the light form PF = 4 (layouts 11-14, 16, 17), which
// loops like the SELL SpMV with few registers and many warps per SM, W for
// about 16 (11, 13), 8 (12), 32 (14), 24 (16) or 48 (17) slots per lane;
// PF = 2 (layout 15), fewer registers still, W for about 16 slots per lane.
// The hybrid layout 18 is 14 with PF = 12 on its one-warp levels (rows of at
// most 32 entries).  (A software-pipelined light form -- the next four slots
// loaded while the current four are gathered -- needed more registers and
// was 15 % slower at 2D 1024^2.)
// A block takes the slice groups g = blockIdx.x, blockIdx.x + gridDim.x, ...
// of the level: one each when the grid covers every group (all but 13), or
// several in turn on a grid of the resident blocks (13), so that a level a
// little larger than one wave runs without a ragged second wave.
template <class T, bool FWD, int W, int PF>
__global__ void __launch_bounds__(kBlock, PF <= 2 ? 6 : (PF <= 4 ? 5 : 3)) k_trsv_level_sellw(Args a, int s0, int s1) {
  constexpr int SPB = kBlock / (32 * W);  // slices per group
  static_assert(SPB * 32 * W == kBlock, "block shape");
  __shared__ T part[W > 1 ? W - 1 : 1][SPB][32];
  cudaTriggerProgrammaticLaunchCompletion();
  const SellView m = FWD ? a.sL : a.sU;
  const T* __restrict__ val = pick<T>(m.val, m.val32);
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = warp % W, ls = warp / W;
  const int ngroups = (s1 - s0 + SPB - 1) / SPB;
  constexpr int SW = 32 * W;  // stride of a lane's consecutive slots
  int row = -1, n = 0, base = 0;
  T ii = T(0);
  int cc[PF];
  T v[PF];
  // the lane's row and its first PF slots in group g (constant arrays only)
#define GBS_SELLW_LANE(g)                                                  \
  do {                                                                     \
    row = -1;                                                              \
    n = 0;                                                                 \
    base = 0;                                                              \
    ii = T(0);                                                             \
    const int s_ = s0 + (g) * SPB + ls;                                    \
    if ((g) < ngroups && s_ < s1) {                                        \
      const int r_ = m.row0[s_] + lane;                                    \
      if (r_ < m.row0[s_ + 1]) {                                           \
        row = r_;                                                          \
        const int len_ = m.rowlen[r_];                                     \
        n = len_ > h ? (len_ - h + W - 1) / W : 0;                         \
        base = m.off[s_] + 32 * h + lane;                                  \
        if (h == 0) ii = inv[r_];                                          \
      }                                                                    \
    }                                                                      \
    _Pragma("unroll") for (int u = 0; u < PF; ++u) {                       \
      cc[u] = u < n ? __ldcs(m.col + base + SW * u) : 0;                   \
      v[u] = u < n ? __ldcs(val + base + SW * u) : T(0);                   \
    }                                                                      \
  } while (0)
  int g = blockIdx.x;
  GBS_SELLW_LANE(g);
  cudaGridDependencySynchronize();
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;  // decides the stores only
  for (bool first = true; g < ngroups; g += gridDim.x, first = false) {  // uniform over the block
    if (!first) GBS_SELLW_LANE(g);
    const int nw = __reduce_max_sync(0xffffffffu, n);  // the warp's longest lane
    T xg[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) xg[u] = u < n ? __ldcg(out + cc[u]) : T(0);
    T sum = 0;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      if (u >= nw) break;
      sum += v[u] * xg[u];
    }
    for (int u = PF; u < n; ++u) sum += __ldcs(val + base + SW * u) * __ldcg(out + __ldcs(m.col + base + SW * u));
    if (W > 1) {
      if (h > 0) part[h - 1][ls][lane] = sum;
      __syncthreads();
      if (h == 0) {
#pragma unroll
        for (int u = 0; u < W - 1; ++u) sum += part[u][ls][lane];
      }
    }
    if (h == 0 && row >= 0 && live) out[row] = (__ldcg(rhs + row) - sum) * ii;
    if (W > 1) __syncthreads();  // part[] is reused by the next group
  }
#undef GBS_SELLW_LANE
}

// ---- TMA-staged SELL-32 variant (single right-hand side) ------------------
// One level of a triangular solve (same recurrences as k_trsv_level) on the
// SELL-32 copy, with the factor streamed into shared memory by the Tensor
// Memory Accelerator.  The level's slices are cut into groups of 8 / W
// consecutive slices (W warps per 32-row slice, chosen by the host from the
// level's longest row so that W * kTmaPF slots cover it); the slots of a
// group are contiguous in the SELL copy, so one bulk copy (cp.async.bulk,
// completion counted in bytes on an mbarrier) moves its values and one its
// column indices.  Each block takes groups g = blockIdx.x, blockIdx.x +
// gridDim.x, ... through two shared-memory stages: the copies of its first
// two groups are issued before the wait for the previous level (the factor
// does not depend on it), and the copy of group i + 2 is issued as soon as
// group i has been consumed.  The gathers of group i + 1's solution entries
// are issued before the FMAs of group i, so the HBM stream of the factor, the
// L2 gathers and the FP64 work overlap.  Warp h of a slice sums the slots h,
// h + W, ... of its rows; the W partial sums of a row are added in warp order
// in shared memory.  Every wait on a stage is bounded: after kTmaWaitNs (2 s)
// the kernel sets *a.dev_status, skips the stage, waits (bounded again) for
// its own copies in flight and returns.
// Dynamic shared memory: 2 stages of kTmaCap values (T) and column indices,
// then two 8-byte mbarriers.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_arrive(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// true once the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for a stage: gives up after kTmaWaitNs of wall time (or kTmaWaitPolls
// polls, whichever comes first) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (long long i = 0; i < kTmaWaitPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && global_ns() - t0 > kTmaWaitNs) return false;
  }
  return false;
}

// bulk copy global -> shared (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <class T, bool FWD, int W>
__global__ void __launch_bounds__(kBlock) k_trsv_level_tma(Args a, int s0, int s1) {
  constexpr int SPB = kBlock / (32 * W);  // slices per group
  static_assert(SPB * 32 * W == kBlock, "block shape");
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ T part[W > 1 ? W - 1 : 1][SPB][32];
  __shared__ int oversize;
  T* sval = reinterpret_cast<T*>(tma_smem);                                        // [2][kTmaCap]
  int32_t* scol = reinterpret_cast<int32_t*>(tma_smem + 2 * kTmaCap * sizeof(T));  // [2][kTmaCap]
  uint64_t* bar = reinterpret_cast<uint64_t*>(tma_smem + 2 * kTmaCap * (sizeof(T) + 4));
  cudaTriggerProgrammaticLaunchCompletion();
  const SellView m = FWD ? a.sL : a.sU;
  const T* __restrict__ val = pick<T>(m.val, m.val32);
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = warp % W, ls = warp / W;
  const int ngroups = (s1 - s0 + SPB - 1) / SPB;
  // the copy of group g into stage st (thread 0 only); a group larger than a
  // stage (the host never launches one) is not copied and fails the block
  auto issue = [&](int g, int st) {
    const int sa = s0 + g * SPB, sb = min(sa + SPB, s1);
    const int first = m.off[sa], slots = m.off[sb] - first;
    if (slots > kTmaCap) {
      oversize = 1;
      mbar_arrive(&bar[st]);
    } else if (slots > 0) {
      mbar_expect_arrive(&bar[st], (unsigned)(slots * (sizeof(T) + 4)));
      bulk_g2s(sval + st * kTmaCap, val + first, (unsigned)(slots * sizeof(T)), &bar[st]);
      bulk_g2s(scol + st * kTmaCap, m.col + first, (unsigned)(slots * 4), &bar[st]);
    } else {
      mbar_arrive(&bar[st]);
    }
  };
  if (threadIdx.x == 0) {
    oversize = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if ((int)blockIdx.x < ngroups) issue(blockIdx.x, 0);
    if ((int)blockIdx.x + (int)gridDim.x < ngroups) issue(blockIdx.x + gridDim.x, 1);
  }
  cudaGridDependencySynchronize();
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;  // decides the stores only
  struct Lane {
    int row, n, base;
    T ii, rv;
  };
  auto lane_of = [&](int g) {
    Lane L = {-1, 0, 0, T(0), T(0)};
    const int sa = s0 + g * SPB, sb = min(sa + SPB, s1);
    const int s = sa + ls;
    if (s < sb) {
      const int r = m.row0[s] + lane;
      if (r < m.row0[s + 1]) {
        L.row = r;
        const int len = m.rowlen[r];
        L.n = len > h ? (len - h + W - 1) / W : 0;
        L.base = m.off[s] - m.off[sa] + 32 * h + lane;
        if (h == 0) {
          L.ii = inv[r];
          L.rv = __ldcg(rhs + r);
        }
      }
    }
    return L;
  };
  bool failed = false;
  // a stage is read only after its wait succeeded and its group was copied
  // (an oversize group is not copied and leaves the stage's contents stale)
  auto stage_ready = [&](int st, unsigned parity) {
    const bool ok = mbar_wait_bounded(&bar[st], parity) && *(volatile int*)&oversize == 0;
    if (!ok) failed = true;
    return ok;
  };
  int it = 0;
  T xa[kTmaPF], xb[kTmaPF];
  Lane cur = {-1, 0, 0, T(0), T(0)};
  int g = blockIdx.x;
  if (g < ngroups) {
    cur = lane_of(g);
    if (!stage_ready(0, 0u)) cur.n = 0;
    const int32_t* sc = scol;
#pragma unroll
    for (int u = 0; u < kTmaPF; ++u) xa[u] = u < cur.n ? __ldcg(out + sc[cur.base + 32 * W * u]) : T(0);
  }
  for (; g < ngroups; g += gridDim.x, ++it) {  // uniform over the block
    if (__syncthreads_or(failed || oversize)) break;
    const int st = it & 1;
    // start the next group: its lane data, its stage, its gathers
    const int gn = g + gridDim.x;
    Lane nxt = {-1, 0, 0, T(0), T(0)};
    if (gn < ngroups) {
      nxt = lane_of(gn);
      if (!stage_ready(st ^ 1, (unsigned)(((it + 1) >> 1) & 1))) nxt.n = 0;
      const int32_t* sc = scol + (st ^ 1) * kTmaCap;
#pragma unroll
      for (int u = 0; u < kTmaPF; ++u) xb[u] = u < nxt.n ? __ldcg(out + sc[nxt.base + 32 * W * u]) : T(0);
    }
    // this group's sums (uniform exit at the warp's longest lane; shorter
    // lanes add 0 * 0)
    const T* sv = sval + st * kTmaCap;
    const int32_t* sc = scol + st * kTmaCap;
    const int nw = __reduce_max_sync(0xffffffffu, cur.n);
    T sum = 0;
#pragma unroll
    for (int u = 0; u < kTmaPF; ++u) {
      if (u >= nw) break;
      sum += (u < cur.n ? sv[cur.base + 32 * W * u] : T(0)) * xa[u];
    }
    for (int u = kTmaPF; u < cur.n; ++u) sum += sv[cur.base + 32 * W * u] * __ldcg(out + sc[cur.base + 32 * W * u]);
    if (W > 1 && h > 0) part[h - 1][ls][lane] = sum;
    __syncthreads();  // stage st and part[] fully read / written
    if (W > 1 && h == 0) {
#pragma unroll
      for (int u = 0; u < W - 1; ++u) sum += part[u][ls][lane];
    }
    if (h == 0 && cur.row >= 0 && live) out[cur.row] = (cur.rv - sum) * cur.ii;
    if (threadIdx.x == 0 && g + 2 * (int)gridDim.x < ngroups) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // reads of stage st before its refill
      issue(g + 2 * gridDim.x, st);
    }
    if (W > 1) __syncthreads();  // part[] is reused by the next group
    cur = nxt;
#pragma unroll
    for (int u = 0; u < kTmaPF; ++u) xa[u] = xb[u];
  }
  if ((failed || oversize) && threadIdx.x == 0) {
    atomicExch(a.dev_status, 1);
    // let the copies this block issued land before it exits (bounded)
    for (int k = 0; k < 2; ++k) {
      const int g2 = (int)blockIdx.x + (it + k) * (int)gridDim.x;
      if (g2 < ngroups) mbar_wait_bounded(&bar[(it + k) & 1], (unsigned)(((it + k) >> 1) & 1));
    }
  }
}

// ---- staged variant (single right-hand side) ------------------------------
// One level of a triangular solve (same recurrences as k_trsv_level) over a
// block partition of the level (build_staged): block b owns the contiguous
// rows [desc[4b], desc[4b+1]), whose off-diagonal entries are the contiguous
// CSR positions [desc[4b+2], desc[4b+3]).  Before the wait for the previous level the block copies the
// rows' column indices, factor values, row offsets and 1/L_ii into shared
// memory with coalesced loads (this overlaps the previous level).  After the
// wait all threads gather the needed solution entries at once -- one
// memory round trip per level, whatever the row lengths -- and then G lanes
// per row sum value * entry from shared memory, G chosen by the host from
// the level's mean row length.  Dynamic shared memory: T val[ecap], T
// xg[ecap], T rhs[rcap], T inv[rcap], int col[ecap], int off[rcap + 1].
template <class T, bool FWD, int G>
__global__ void __launch_bounds__(kBlock) k_trsv_level_staged(Args a, const int4* __restrict__ desc, int ecap,
                                                              int rcap) {
  constexpr int EPT = kStagedEntries / kBlock;  // entries per thread
  static_assert(EPT * kBlock == kStagedEntries && kStagedRows <= kBlock, "staged block shape");
  extern __shared__ __align__(16) unsigned char staged_smem[];
  cudaTriggerProgrammaticLaunchCompletion();
  const int32_t* __restrict__ ptr = FWD ? a.L_ptr : a.U_ptr;
  const int32_t* __restrict__ col = FWD ? a.L_col : a.U_col;
  const T* __restrict__ val = FWD ? pick<T>(a.L_val, a.L_val32) : pick<T>(a.U_val, a.U_val32);
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  T* sv = (T*)staged_smem;
  T* sx = sv + ecap;
  T* sr = sx + ecap;
  T* si = sr + rcap;
  int* sc = (int*)(si + rcap);
  int* so = sc + ecap;
  const int tid = threadIdx.x;
  const int4 d = desc[blockIdx.x];
  const int rb = d.x, nr = d.y - d.x;
  const int eb = d.z, ne = d.w - d.z;
  {
    // all loads first (one round trip), then the shared-memory stores
    int cv[EPT];
    T vv[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = tid + u * kBlock;
      cv[u] = e < ne ? col[eb + e] : 0;
      vv[u] = e < ne ? val[eb + e] : T(0);
    }
    const int o = tid < nr ? ptr[rb + tid] - eb : 0;
    const T iv = tid < nr ? inv[rb + tid] : T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = tid + u * kBlock;
      if (e < ne) {
        sc[e] = cv[u];
        sv[e] = vv[u];
      }
    }
    if (tid < nr) {
      so[tid] = o;
      si[tid] = iv;
    }
    if (tid == 0) so[nr] = ne;
  }
  cudaGridDependencySynchronize();
  __syncthreads();
  // the CG state flag is read together with the gathers; it only decides the
  // stores (uniform over the grid)
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;
  {
    T xv[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = tid + u * kBlock;
      xv[u] = e < ne ? __ldcg(out + sc[e]) : T(0);
    }
    const T rv = tid < nr ? __ldcg(rhs + rb + tid) : T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = tid + u * kBlock;
      if (e < ne) sx[e] = xv[u];
    }
    if (tid < nr) sr[tid] = rv;
  }
  __syncthreads();
  if (!live) return;
  const int g = tid % G;
  for (int i = tid / G; i < nr; i += kBlock / G) {  // uniform over a lane group
    const int e1 = so[i + 1];
    int e = so[i] + g;
    T s0 = 0, s1 = 0;
    for (; e + G < e1; e += 2 * G) {
      s0 += sv[e] * sx[e];
      s1 += sv[e + G] * sx[e + G];
    }
    if (e < e1) s0 += sv[e] * sx[e];
    T s = s0 + s1;
    if (G > 1) {
      if (sizeof(T) == 8) s = (T)group_sum<G>((double)s);
      else s = (T)group_sumf<G>((float)s);
    }
    if (g == 0) out[rb + i] = (sr[i] - s) * si[i];
  }
}

// ---- packed variant (single right-hand side) ------------------------------
// One level of a triangular solve (same recurrences as k_trsv_level) over the
// packed k-major copy of the level (build_packed): block b owns rows
// [desc.x, desc.x + desc.y) and slots [desc.z, desc.z + desc.y * desc.w),
// slot k * rows + i holding the k-th entry of row i (column -1, value 0 past
// its end).  The slots are staged in shared memory before the wait for the
// previous level; after it, consecutive threads gather the solution entries
// of consecutive slots -- the same stencil entry of neighbouring rows, so a
// warp touches few memory sectors -- and G lanes per row sum value * entry
// over k (padding contributes exact zeros).  Shared memory: T val[cap],
// T xg[cap], T rhs[rcap], T inv[rcap], int col[cap].
template <class T, bool FWD, int G>
__global__ void __launch_bounds__(kBlock) k_trsv_level_packed(Args a, const int4* __restrict__ desc,
                                                              const int32_t* __restrict__ pcol,
                                                              const T* __restrict__ pval, int cap, int rcap) {
  constexpr int EPT = kPackedSlots / kBlock;  // slots per thread
  static_assert(EPT * kBlock == kPackedSlots && kStagedRows <= kBlock, "packed block shape");
  extern __shared__ __align__(16) unsigned char packed_smem[];
  cudaTriggerProgrammaticLaunchCompletion();
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  T* sv = (T*)packed_smem;
  T* sx = sv + cap;
  T* sr = sx + cap;
  T* si = sr + rcap;
  int* sc = (int*)(si + rcap);
  const int tid = threadIdx.x;
  const int4 d = desc[blockIdx.x];
  const int rb = d.x, nr = d.y, off = d.z, len = d.w;
  const int ns = nr * len;
  {
    int cv[EPT];
    T vv[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      cv[u] = q < ns ? pcol[off + q] : -1;
      vv[u] = q < ns ? pval[off + q] : T(0);
    }
    const T iv = tid < nr ? inv[rb + tid] : T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      if (q < ns) {
        sc[q] = cv[u];
        sv[q] = vv[u];
      }
    }
    if (tid < nr) si[tid] = iv;
  }
  cudaGridDependencySynchronize();
  __syncthreads();
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;  // read with the gathers; decides the stores
  {
    T xv[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      const int cc = q < ns ? sc[q] : -1;
      xv[u] = cc >= 0 ? __ldcg(out + cc) : T(0);
    }
    const T rv = tid < nr ? __ldcg(rhs + rb + tid) : T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      if (q < ns) sx[q] = xv[u];
    }
    if (tid < nr) sr[tid] = rv;
  }
  __syncthreads();
  if (!live) return;
  const int g = tid % G;
  for (int i = tid / G; i < nr; i += kBlock / G) {  // uniform over a lane group
    T s0 = 0, s1 = 0;
    int k = g;
    for (; k + G < len; k += 2 * G) {
      s0 += sv[k * nr + i] * sx[k * nr + i];
      s1 += sv[(k + G) * nr + i] * sx[(k + G) * nr + i];
    }
    if (k < len) s0 += sv[k * nr + i] * sx[k * nr + i];
    T s = s0 + s1;
    if (G > 1) {
      if (sizeof(T) == 8) s = (T)group_sum<G>((double)s);
      else s = (T)group_sumf<G>((float)s);
    }
    if (g == 0) out[rb + i] = (sr[i] - s) * si[i];
  }
}

// Packed sweep level on the split copy (Packed, Ctx::qL / qU): each row's
// entries whose column lies two or more levels back in the sweep come first,
// those of the level just before it in a second segment.  The launch signals
// its dependent level only after its own wait has returned, i.e. after the
// level before it has completed.  So when a level's blocks start, every level
// two or more steps back has completed and its stores are visible at device
// scope: the blocks gather those solution entries (L2 loads) and sum the first
// segment before they wait, and after the wait gather only the second segment
// and finish the rows (Sec. 6.4, "PCG(A)": the IC(0) application).  The
// wait is the programmatic dependency on the preceding launch alone.  Only
// two levels are in flight at a time, so each launch first asks L2 to fetch
// the columns and values of the next level of the sweep (next[0 .. nnext)),
// whose blocks start after this level's wait.
template <class T, bool FWD, int G>
__global__ void __launch_bounds__(kBlock) k_trsv_level_split(Args a, const int4* __restrict__ desc,
                                                             const int32_t* __restrict__ pcol,
                                                             const T* __restrict__ pval, int cap, int rcap,
                                                             const int4* __restrict__ next, int nnext) {
  constexpr int EPT = kPackedSlots / kBlock;  // slots per thread
  static_assert(EPT * kBlock == kPackedSlots && kStagedRows <= kBlock, "packed block shape");
  extern __shared__ __align__(16) unsigned char split_smem[];
  const T* __restrict__ inv = pick<T>(a.L_inv, a.L_inv32);
  const T* rhs = (const T*)(FWD ? a.cg_r : a.cg_y);
  T* out = (T*)(FWD ? a.cg_y : a.cg_z);
  T* sv = (T*)split_smem;  // first segment: values
  T* sx = sv + cap;        // first segment: solution entries; second: products
  T* ss = sx + cap;        // per row: sum over the first segment
  T* si = ss + rcap;       // per row: inverse diagonal
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < nnext; b += gridDim.x) {
    const int4 e = next[b];
    const int n2 = e.y * ((e.w & 0xffff) + (e.w >> 16));  // slots of that block
    constexpr int VL = 128 / (int)sizeof(T);               // values per 128-byte line
    const int lc = (n2 + 31) / 32, lv = (n2 + VL - 1) / VL;
    for (int t = tid; t < lc + lv; t += kBlock) {
      const void* p = t < lc ? (const void*)(pcol + e.z + 32 * t) : (const void*)(pval + e.z + VL * (t - lc));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
    }
  }
  const int4 d = desc[blockIdx.x];
  const int rb = d.x, nr = d.y, off = d.z, lo = d.w & 0xffff, lr = d.w >> 16;
  const int no = nr * lo, ns = no + nr * lr;
  int cv[EPT];
  T vv[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int q = tid + u * kBlock;
    cv[u] = q < ns ? pcol[off + q] : -1;
    vv[u] = q < ns ? pval[off + q] : T(0);
  }
  {
    T xv[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      xv[u] = (q < no && cv[u] >= 0) ? __ldcg(out + cv[u]) : T(0);
    }
    const T iv = tid < nr ? inv[rb + tid] : T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      if (q < no) {
        sv[q] = vv[u];
        sx[q] = xv[u];
      }
    }
    if (tid < nr) si[tid] = iv;
  }
  __syncthreads();
  const int g = tid % G;
  for (int i = tid / G; i < nr; i += kBlock / G) {  // uniform over a lane group
    T s0 = 0, s1 = 0;
    int k = g;
    for (; k + G < lo; k += 2 * G) {
      s0 += sv[k * nr + i] * sx[k * nr + i];
      s1 += sv[(k + G) * nr + i] * sx[(k + G) * nr + i];
    }
    if (k < lo) s0 += sv[k * nr + i] * sx[k * nr + i];
    T s = s0 + s1;
    if (G > 1) {
      if (sizeof(T) == 8) s = (T)group_sum<G>((double)s);
      else s = (T)group_sumf<G>((float)s);
    }
    if (g == 0) ss[i] = s;
  }
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  const bool live = SF(a, S_CG_ACTIVE, 0, 1) != 0.0;  // read with the gathers; decides the stores
  {
    T xv[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      xv[u] = (q >= no && q < ns && cv[u] >= 0) ? __ldcg(out + cv[u]) : T(0);
    }
    const T rv = tid < nr ? __ldcg(rhs + rb + tid) : T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int q = tid + u * kBlock;
      if (q >= no && q < ns) sx[q] = vv[u] * xv[u];
    }
    __syncthreads();
    if (!live) return;
    if (tid < nr) {
      T s = ss[tid];
      for (int k = 0; k < lr; ++k) s += sx[no + k * nr + tid];
      out[rb + tid] = (rv - s) * si[tid];
    }
  }
}

// x[i] = v (kernel timing and layout tuning only).
template <class T>
__global__ void k_fill_value(T* __restrict__ x, int64_t n, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// rho = r^T z.  init: p = z, rho.  Otherwise beta = rho_new / rho.
template <int K, class T, int SYS = 0>
__global__ void k_cg_rho(Args a, int init) {
  using C = CgSys<SYS>;
  const T* __restrict__ r = (const T*)C::r(a);
  const T* __restrict__ z = (const T*)C::z(a);
  T* __restrict__ p = (T*)C::p(a);
  const int t = threadIdx.x % K;
  const bool live = SF(a, C::ACTIVE, t, K) != 0.0;
  double vals[1] = {0.0};
  T acc = 0;
  const int stride = (gridDim.x * blockDim.x) / K;
  if (live) {
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / K; i < C::n(a); i += stride) {
      const size_t idx = (size_t)i * K + t;
      const T zv = z[idx];
      acc += r[idx] * zv;
      if (init) p[idx] = zv;
    }
  }
  vals[0] = (double)acc;
  block_partials<K, 1>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K];
    finalize_partials<K, 1>(a.partial, gridDim.x, tot);
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      if (SF(a, C::ACTIVE, s, K) != 0.0) {
        if (init) {
          SF(a, C::RHO, s, K) = tot[s];
        } else {
          SF(a, C::ALPHA, s, K) = tot[s] / SF(a, C::RHO, s, K);  // beta, consumed by k_cg_pupdate
          SF(a, C::RHO, s, K) = tot[s];
        }
      }
    }
    if (threadIdx.x == 0) *a.counter = 0;
  }
}

// p = z + beta p (beta kept in the ALPHA field between k_cg_rho and this kernel).
template <int K, class T, int SYS = 0>
__global__ void k_cg_pupdate(Args a) {
  using C = CgSys<SYS>;
  const T* __restrict__ z = (const T*)C::z(a);
  T* __restrict__ p = (T*)C::p(a);
  const int t = threadIdx.x % K;
  if (SF(a, C::ACTIVE, t, K) == 0.0) return;
  const T beta = (T)SF(a, C::ALPHA, t, K);
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / K; i < C::n(a); i += stride) {
    const size_t idx = (size_t)i * K + t;
    p[idx] = z[idx] + beta * p[idx];
  }
}

// ------------------------------------------------------ Jacobi blocks ----
// z = r / diag for the diagonally preconditioned CG blocks (Sec. 6.2: the
// preconditioner of the inner PCG is the diagonal of A_h or of Q).
template <int K, class T, int SYS>
__global__ void k_jacobi(Args a) {
  using C = CgSys<SYS>;
  const T* __restrict__ r = (const T*)C::r(a);
  T* __restrict__ z = (T*)C::z(a);
  const int t = threadIdx.x % K;
  if (SF(a, C::ACTIVE, t, K) == 0.0) return;
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / K; i < C::n(a); i += stride) {
    const double d = SYS ? a.Qdiag[i] : a.A_val[a.A_diag[i]];
    const size_t idx = (size_t)i * K + t;
    z[idx] = r[idx] / (T)d;
  }
}

// ------------------------------------------------- pressure-block IC(0) ----
// z = (L L^T)^{-1} r for the IC(0) factor L = L1 x L1 [x L1] of Q (natural
// numbering), applied one direction at a time: (L L^T)^{-1} is the Kronecker
// product of Q1^{-1} = L1^{-T} L1^{-1}, so along direction `axis` every line
// of the pressure grid (m = N + p - 1 points, stride m^(dim-1-axis)) gets a
// banded forward and backward substitution with L1 (half-bandwidth p - 1):
//   y_s = (x_s - sum_{o=1}^{p-1} L1[s][s-o] y_{s-o}) / L1[s][s],
//   z_s = (y_s - sum_{o=1}^{p-1} L1[s+o][s] z_{s+o}) / L1[s][s].
// One thread per (line, RHS); the lines are independent.  src and dst are
// distinct buffers (the host alternates them between directions); the
// values of a line are fetched kQPF steps ahead of their use.
constexpr int kQPMAX = 6;  // largest velocity degree p (band width of L1)
constexpr int kQPF = 8;    // prefetch distance along a line
template <int K, class T>
__global__ void k_q_lines(Args a, int axis, const T* __restrict__ src, T* __restrict__ dst) {
  const int m = a.qm, p = a.qp;
  const T* __restrict__ l1 = pick<T>(a.l1, a.l1_32);
  int64_t stride = 1;
  for (int d = a.dim - 1; d > axis; --d) stride *= m;
  const int64_t nlines = (int64_t)a.n_p / m;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(tid % K);
  const int64_t line = tid / K;
  if (line >= nlines || SF(a, S_Q_ACTIVE, t, K) == 0.0) return;
  const int64_t base = (line / stride) * stride * m + line % stride;
  auto at = [&](int s) { return (size_t)(base + (int64_t)s * stride) * K + t; };
  T win[kQPMAX];  // win[o-1] = the value o steps back along the sweep
  T pf[kQPF];     // values of the next kQPF points
#pragma unroll
  for (int o = 0; o < kQPMAX; ++o) win[o] = T(0);
#pragma unroll
  for (int u = 0; u < kQPF; ++u) pf[u] = u < m ? src[at(u)] : T(0);
  for (int s = 0; s < m; ++s) {
    T v = pf[0];
#pragma unroll
    for (int u = 0; u < kQPF - 1; ++u) pf[u] = pf[u + 1];
    pf[kQPF - 1] = s + kQPF < m ? src[at(s + kQPF)] : T(0);
#pragma unroll
    for (int o = 1; o < kQPMAX; ++o)
      if (o < p && s - o >= 0) v -= l1[s * p + o] * win[o - 1];
    v = v / l1[s * p];
#pragma unroll
    for (int o = kQPMAX - 1; o > 0; --o) win[o] = win[o - 1];
    win[0] = v;
    dst[at(s)] = v;
  }
#pragma unroll
  for (int o = 0; o < kQPMAX; ++o) win[o] = T(0);
#pragma unroll
  for (int u = 0; u < kQPF; ++u) pf[u] = m - 1 - u >= 0 ? dst[at(m - 1 - u)] : T(0);
  for (int s = m - 1; s >= 0; --s) {
    T v = pf[0];
#pragma unroll
    for (int u = 0; u < kQPF - 1; ++u) pf[u] = pf[u + 1];
    pf[kQPF - 1] = s - kQPF >= 0 ? dst[at(s - kQPF)] : T(0);
#pragma unroll
    for (int o = 1; o < kQPMAX; ++o)
      if (o < p && s + o < m) v -= l1[(s + o) * p + o] * win[o - 1];
    v = v / l1[s * p];
#pragma unroll
    for (int o = kQPMAX - 1; o > 0; --o) win[o] = win[o - 1];
    win[0] = v;
    dst[at(s)] = v;
  }
}

// --------------------------------------------------------------- exit ----
// r = b - K x: ||r||^2, w^T x_p and w^T 1 for the zero-mean filter.
template <int K>
__global__ void k_residual(Args a) {
  using M = Map<K>;
  const double* __restrict__ x = a.x;
  const int n = a.n_u + a.n_p;
  const int lane = threadIdx.x & 31;
  const int g = lane % M::G;
  const int t = (K == 1) ? 0 : g;
  double vals[3] = {0.0, 0.0, 0.0};
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / M::G;
  const int ng = (gridDim.x * blockDim.x) / M::G;
  for (int r = gid; r < n; r += ng) {
    double y = 0.0;
    if (r < a.n_u) {
      if (K == 1) {
        for (int e = a.A_ptr[r] + g; e < a.A_ptr[r + 1]; e += M::G) y += a.A_val[e] * x[a.A_col[e]];
        for (int e = a.Bt_ptr[r] + g; e < a.Bt_ptr[r + 1]; e += M::G) y += a.Bt_val[e] * x[a.n_u + a.Bt_col[e]];
      } else {
        for (int e = a.A_ptr[r]; e < a.A_ptr[r + 1]; ++e) y += a.A_val[e] * x[(size_t)a.A_col[e] * K + t];
        for (int e = a.Bt_ptr[r]; e < a.Bt_ptr[r + 1]; ++e)
          y += a.Bt_val[e] * x[(size_t)(a.n_u + a.Bt_col[e]) * K + t];
      }
    } else {
      const int kr = r - a.n_u;
      if (K == 1) {
        for (int e = a.B_ptr[kr] + g; e < a.B_ptr[kr + 1]; e += M::G) y += a.B_val[e] * x[a.B_col[e]];
      } else {
        for (int e = a.B_ptr[kr]; e < a.B_ptr[kr + 1]; ++e) y += a.B_val[e] * x[(size_t)a.B_col[e] * K + t];
      }
    }
    if (K == 1) y = group_sum<M::G>(y);
    if (K > 1 || g == 0) {
      const size_t idx = (size_t)r * K + t;
      const double res = a.b[idx] - y;
      vals[0] += res * res;
      if (r >= a.n_u) {
        vals[1] += a.wmean[r - a.n_u] * x[idx];
        vals[2] += a.wmean[r - a.n_u];
      }
    }
  }
  block_partials<K, 3>(vals, a.partial);
  if (last_block(a.counter)) {
    __shared__ double tot[K * 3];
    finalize_partials<K, 3>(a.partial, gridDim.x, tot);
    if (threadIdx.x < K) {
      const int s = threadIdx.x;
      const double bn = SF(a, S_BNORM, s, K);
      SF(a, S_TRUE_RES, s, K) = bn > 0.0 ? sqrt(tot[s * 3]) / bn : 0.0;
      SF(a, S_PMEAN, s, K) = tot[s * 3 + 2] != 0.0 ? tot[s * 3 + 1] / tot[s * 3 + 2] : 0.0;
    }
    if (threadIdx.x == 0) *a.counter = 0;
  }
}

// out [k][n] (natural numbering) from x; pressure shifted to zero mean.
template <int K>
__global__ void k_scatter(Args a, double* __restrict__ out) {
  const int n = a.n_u + a.n_p;
  const int t = threadIdx.x % K;
  if (t >= a.k) return;
  const double pm = SF(a, S_PMEAN, t, K);
  const int stride = (gridDim.x * blockDim.x) / K;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) / K; r < n; r += stride) {
    const size_t idx = (size_t)r * K + t;
    if (r < a.n_u) out[(size_t)t * n + a.order[r]] = a.x[idx];
    else out[(size_t)t * n + r] = a.x[idx] - pm;
  }
}

// Adjoint right-hand side: the pressure part of dL/d(filtered p) is mapped by
// P^T, P = I - 1 w^T / (w^T 1):  P^T g = g - w (1^T g) / (w^T 1).
__global__ void k_adjoint_coef(int n_u, int n_p, int k, const double* __restrict__ g,
                               const double* __restrict__ w, double* __restrict__ coef) {
  __shared__ double s1[kBlock], s2[kBlock];
  const int t = blockIdx.x;
  if (t >= k) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n_p; i += blockDim.x) {
    a += g[(size_t)t * (n_u + n_p) + n_u + i];
    b += w[i];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) coef[t] = s1[0] / s2[0];
}

__global__ void k_adjoint_rhs(int n_u, int n_p, int k, const double* __restrict__ g,
                              const double* __restrict__ w, const double* __restrict__ coef,
                              double* __restrict__ out) {
  const size_t n = (size_t)n_u + n_p, total = n * k;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / n, r = i % n;
    out[i] = r < (size_t)n_u ? g[i] : g[i] - w[r - n_u] * coef[t];
  }
}

// Operators in natural numbering (one vector, FP64):
// which 0: y = K x; 1: y = A x_u; 2: y = B x_u; 3: y = B^T x_p; 4: y = Q x_p.
__global__ void k_apply_natural(Args a, int which, const double* __restrict__ xin, double* __restrict__ yout) {
  const int lane = threadIdx.x & 31, g = lane & 7;
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, ng = (gridDim.x * blockDim.x) >> 3;
  const int nu = a.n_u;
  const int rows = (which == 0) ? nu + a.n_p : ((which == 2 || which == 4) ? a.n_p : nu);
  const double* xu = xin;
  const double* xp = (which == 0) ? xin + nu : xin;
  for (int r = gid; r < rows; r += ng) {
    double y = 0.0;
    int out_index;
    if (which == 4) {
      for (int e = a.Q_ptr[r] + g; e < a.Q_ptr[r + 1]; e += 8) y += a.Q_val[e] * xp[a.Q_col[e]];
      out_index = r;
    } else if ((which == 0 && r < nu) || which == 1 || which == 3) {
      if (which != 3)
        for (int e = a.A_ptr[r] + g; e < a.A_ptr[r + 1]; e += 8) y += a.A_val[e] * xu[a.order[a.A_col[e]]];
      if (which != 1)
        for (int e = a.Bt_ptr[r] + g; e < a.Bt_ptr[r + 1]; e += 8) y += a.Bt_val[e] * xp[a.Bt_col[e]];
      out_index = a.order[r];
    } else {
      const int kr = (which == 0) ? r - nu : r;
      for (int e = a.B_ptr[kr] + g; e < a.B_ptr[kr + 1]; e += 8) y += a.B_val[e] * xu[a.order[a.B_col[e]]];
      out_index = (which == 0) ? r : kr;
    }
    y = group_sum<8>(y);
    if (g == 0) yout[out_index] = y;
  }
}

// dL/dnu = -lam_u^T A_h u / nu for each RHS (natural-numbered inputs [k][n]).
__global__ void k_dnu(Args a, int k, const double* __restrict__ lam, const double* __restrict__ xv,
                      double* __restrict__ partial, unsigned* counter, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, g = lane & 7;
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, ng = (gridDim.x * blockDim.x) >> 3;
  const size_t n = (size_t)a.n_u + a.n_p;
  for (int t = 0; t < k; ++t) {
    double vals[1] = {0.0};
    const double* u = xv + (size_t)t * n;
    const double* l = lam + (size_t)t * n;
    for (int r = gid; r < a.n_u; r += ng) {
      double y = 0.0;
      for (int e = a.A_ptr[r] + g; e < a.A_ptr[r + 1]; e += 8) y += a.A_val[e] * u[a.order[a.A_col[e]]];
      y = group_sum<8>(y);
      if (g == 0) vals[0] += l[a.order[r]] * y;
    }
    block_partials<1, 1>(vals, partial + (size_t)t * gridDim.x);
  }
  if (last_block(counter)) {
    __shared__ double tot[1];
    for (int t = 0; t < k; ++t) {
      finalize_partials<1, 1>(partial + (size_t)t * gridDim.x, gridDim.x, tot);
      if (threadIdx.x == 0) out[t] = -tot[0] / a.nu;
      __syncthreads();
    }
    if (threadIdx.x == 0) *counter = 0;
  }
}

}  // namespace

}  // namespace gbs
