/* gbstokes.h -- C ABI of the GB300 (sm_103a) Stokes solver library.
 *
 * Method (Cortes & Coutinho, arXiv:1309.5048): divergence-conforming
 * (Raviart-Thomas type) B-spline discretisation of Stokes flow on the unit
 * square or cube with Nitsche no-slip terms (Sec. 3.2, Sec. 4), solved by
 * preconditioned MINRES (Sec. 5) with the block-diagonal preconditioner
 * diag(M_A, M_Q) of Sec. 5.1.  By default M_A^{-1} is a relaxed inner
 * conjugate-gradient solve on A_h preconditioned by incomplete Cholesky IC(0)
 * (Sec. 6.4) and M_Q = Diag(Q_nu), Q_nu = Q / (2 nu) (Sec. 5.1); the other
 * blocks of Sec. 5.1 (Diag(A), diagonally preconditioned CG on A_h or Q, and
 * the IC(0)-preconditioned CG on Q of Sec. 6.4) are options of gb_solve.  The
 * loads of the manufactured solution (Sec. 6.2), the lid-driven cavity
 * (Sec. 6.4) and a Fourier forcing, an adjoint solve and Ritz-value
 * diagnostics of the MINRES Lanczos process are provided.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Status:   every function returns GB_OK (0) or a GB_ERR_* code and never
 *           throws; gb_last_error() gives a one-line message for the calling
 *           thread.
 * Memory:   arguments named *_dev are device pointers owned by the caller
 *           (e.g. torch tensors); the library borrows them for the duration
 *           of the call only.  *_host arguments are host memory.  The context
 *           owns everything else (patterns, values, factors, workspaces).
 * Streams:  all device work is ordered on the stream given to
 *           gb_setup_pattern; calls that return host results synchronise it.
 * Numbering: velocity DOFs are numbered component-major, then
 *           lexicographically over the 1D function indices with the last
 *           direction fastest; component c has degree p in direction c and
 *           p-1 in the others, without its first and last function in
 *           direction c (no-penetration space V_{0,h}, Sec. 3.2).  Pressure
 *           DOFs (degree p-1, full space Q_h) are lexicographic the same way.
 *           A solution or right-hand side vector is [u (n_u); p (n_p)].
 * Batches:  k right-hand sides are stored RHS-major, [k][n] contiguous
 *           (a row-major torch tensor of shape (k, n)); 1 <= k <= 32.
 * Index width: matrices are stored with 32-bit column indices and row
 *           pointers; problems with more than 2^31 - 1 nonzeros in one
 *           matrix are rejected with GB_ERR_INVALID_ARG.
 * Threading: a context may be used by one host thread at a time.
 */
#ifndef GBSTOKES_H
#define GBSTOKES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_OK 0
#define GB_ERR_INVALID_ARG 1    /* bad size, pointer, option or call order */
#define GB_ERR_CUDA 2           /* a CUDA runtime call failed */
#define GB_ERR_OOM 3            /* device or host allocation failed */
#define GB_ERR_IC0_BREAKDOWN 4  /* IC(0) met a non-positive pivot */
#define GB_ERR_NOT_CONVERGED 5  /* iteration cap reached; outputs written */
#define GB_ERR_NONFINITE 6      /* NaN/Inf met in the right-hand side or iterates */
#define GB_ERR_DEVICE_TIMEOUT 7 /* a bounded device wait gave up: the TMA-staged sweep
                                   (layout 10) waits on the completion of its own
                                   bulk copies with a 2 s limit; no kernel waits
                                   on another kernel or block */

/* Orderings of A_h applied before IC(0).  The paper reorders A by reverse
 * Cuthill-McKee (Sec. 6.4); natural and multicolour orderings are offered
 * because the depth of the factor's DAG bounds the parallelism of the
 * triangular solves. */
#define GB_ORDER_NATURAL 0
#define GB_ORDER_RCM 1
#define GB_ORDER_MULTICOLOUR 2

/* Precision of the inner preconditioner.  FP64 everywhere, or the inner
 * IC(0)-CG in FP32 (FP32 copies of A_h and of the FP64 IC(0) factor, FP32
 * vectors, FP64 across-thread reductions) with the outer MINRES recurrence,
 * residual norms and the factorisation in FP64. */
#define GB_PREC_FP64 0
#define GB_PREC_MIXED 1

/* Pressure block M_Q of the preconditioner (Sec. 5.1, Sec. 6.4).
 * GB_PRESSURE_DIAG: M_Q = Diag(Q_nu).  GB_PRESSURE_PCG: M_Q^{-1} r_p is a CG
 * solve with Q_nu = Q / (2 nu) preconditioned by IC(0) of Q in the natural
 * order ("IC(0)-PCG(A,Q)"), with the same relative tolerance and cap as the
 * velocity block.  In that order the IC(0) factor of Q is its exact Cholesky
 * factor (Q is a Kronecker product of banded 1D mass matrices), so the
 * pressure CG normally stops after one iteration. */
#define GB_PRESSURE_DIAG 0
#define GB_PRESSURE_PCG 1
/* GB_PRESSURE_JACOBI_PCG: the CG solve with Q_nu preconditioned by its
 * diagonal ("PCG(A,Q)" of Sec. 6.2). */
#define GB_PRESSURE_JACOBI_PCG 2

/* Velocity block M_A of the preconditioner (Sec. 5.1).
 * GB_VELOCITY_IC0_PCG: CG on A_h preconditioned by IC(0) ("PCG(A)", Sec. 6.4);
 * GB_VELOCITY_DIAG: M_A = Diag(A_h) ("Diag(A,Q)");
 * GB_VELOCITY_JACOBI_PCG: CG on A_h preconditioned by its diagonal
 * ("PCG(A)", Sec. 6.2).  The CG blocks stop at ||r|| <= inner_tol ||b||. */
#define GB_VELOCITY_IC0_PCG 0
#define GB_VELOCITY_DIAG 1
#define GB_VELOCITY_JACOBI_PCG 2

/* MINRES stopping rule.
 * GB_STOP_RESIDUAL: ||b - K x_j||_2 / ||b||_2 <= tol after step j, the
 * paper's relative residual (it reproduces the MINRES counts of the paper's
 * square-domain tables); the residual is carried by the recurrence
 * r_j = r_{j-1} - c_{j+1} eta_j K w_{j+1} with K w from the Lanczos products.
 * GB_STOP_ESTIMATE: |eta_j| / gamma_1 <= tol, the M^{-1}-norm residual
 * ratio of the Lanczos/Givens recurrence (eq. minimax_precond). */
#define GB_STOP_RESIDUAL 0
#define GB_STOP_ESTIMATE 1

typedef struct gb_ctx gb_ctx;

typedef struct {
  int dim;      /* 2 or 3 */
  int N;        /* elements per direction, >= 1 */
  int p;        /* velocity degree (pressure degree k' = p - 1), 2 <= p <= 6 */
  int ordering; /* GB_ORDER_* */
} gb_problem;

typedef struct {
  double tol;       /* outer stop tolerance (see stop_rule) */
  double inner_tol; /* inner CG stop: ||r||_2 <= inner_tol ||b||_2 from x_0 = 0 */
  int precision;    /* GB_PREC_* */
  int max_outer;    /* MINRES iteration cap (>= 1) */
  int max_inner;    /* inner CG iteration cap per application (>= 1) */
  int use_graph;    /* 1: run the solve as one captured CUDA graph with device-
                       side loop control; 0: host-driven loop */
  const int32_t* forced_inner_host; /* optional (k == 1 only): replay mode.  The
                       i-th preconditioner application runs exactly
                       forced_inner_host[i] inner iterations, ignoring
                       inner_tol.  NULL for normal operation. */
  int64_t nforced;  /* length of forced_inner_host */
  int pressure_block; /* GB_PRESSURE_* */
  const int32_t* forced_q_host; /* optional replay of the pressure CG counts
                       (GB_PRESSURE_PCG, k == 1): the i-th application runs
                       exactly forced_q_host[i] iterations.  NULL otherwise. */
  int64_t nforced_q; /* length of forced_q_host */
  int stop_rule;      /* GB_STOP_* (0: the 2-norm relative residual) */
  int velocity_block; /* GB_VELOCITY_* (0: IC(0)-preconditioned CG) */
} gb_solve_opts;

typedef struct {
  int outer_its;       /* MINRES iterations */
  int precond_apps;    /* preconditioner applications (outer_its + 1) */
  int64_t inner_its_total; /* inner CG iterations over all applications */
  int inner_its_max;   /* largest inner count of one application */
  double relres_est;   /* |eta| / gamma_1 at exit (recurrence estimate) */
  double relres_true;  /* ||b - K x||_2 / ||b||_2 recomputed at exit */
  int64_t q_inner_its_total; /* pressure CG iterations (GB_PRESSURE_PCG) */
  int q_inner_its_max;       /* largest pressure CG count of one application */
  int status;          /* GB_OK, GB_ERR_NOT_CONVERGED, GB_ERR_NONFINITE,
                          GB_ERR_INVALID_ARG (inconsistent pressure rhs) or
                          GB_ERR_DEVICE_TIMEOUT (every column; the other
                          fields are then not filled) */
} gb_info;

/* ---------------------------------------------------------------- setup --
 * Builds the spaces (Sec. 3.2), the sparsity patterns of A_h, B, B^T (support
 * overlap of the tensor-product B-splines), the ordering, the IC(0) pattern
 * (lower triangle of the permuted A_h) with its level sets, and uploads them.
 * `stream` is a cudaStream_t (NULL: legacy default stream).  On success *out
 * receives a new context; release it with gb_destroy.  Host work: O(nnz). */
int gb_setup_pattern(const gb_problem* prob, void* stream, gb_ctx** out);

/* out[0..9] = n_u, n_p, nnz(A_h), nnz(B), nnz(L) (IC(0) factor incl. diagonal),
 * number of forward levels, number of backward levels, nnz(Q) (structural),
 * bytes of device memory held by the context for the operators, the factors
 * and their kernel layouts at the time of the call (the solve workspace is
 * not counted), number of colours used by the ordering (0 unless
 * multicolour). */
int gb_sizes(const gb_ctx* ctx, int64_t* out_host);

/* Assembles A_h = a - eta_h, B and Diag(Q) (Sec. 4: [A_h]_ij = a_h(Phi_j,Phi_i),
 * [B]_kj = -(div Phi_j, phi_k), [Q]_kl = (phi_l, phi_k)) and w_k = (phi_k, 1)
 * on the device.  nu > 0 is the viscosity; cpen is the Nitsche constant C_pen
 * (<= 0 selects 5 (k' + 1), Sec. 6.2); h_F = 1/N.  Invalidates the factor. */
int gb_assemble(gb_ctx* ctx, double nu, double cpen);

/* Load vector f_i = (f, Phi_i) for the forcing
 *   f_d(x) = sum_{m<nmodes} amp[m][d] prod_k sin(pi kappa[m][k] x_k)
 * (kappa_host: int32 [nmodes][dim], amp_host: double [nmodes][dim]),
 * integrated with p+3 Gauss points per direction and element.  f_dev: n_u
 * doubles, natural numbering. */
int gb_load_fourier(gb_ctx* ctx, int nmodes, const int32_t* kappa_host,
                    const double* amp_host, double* f_dev);

/* Load vector of the manufactured solution of Sec. 6.2 (2D only, the sign of
 * u_2 taken so that div u = 0), f = -div(2 nu grad^s u) + grad p
 * (eq. manufactured_force), with the nu of the last gb_assemble. */
int gb_load_manufactured(gb_ctx* ctx, double* f_dev);

/* Load of the lid-driven cavity (Sec. 6.4): no body force, and the Nitsche
 * right-hand side l_h of eq. nitsche_rhs with lid velocity g = e_1 on the
 * face x_dim = 1 (y = 1 in 2D), g = 0 elsewhere, with the nu and C_pen of the
 * last gb_assemble.  f_dev: n_u doubles, natural numbering (the pressure part
 * of the right-hand side is zero). */
int gb_load_cavity(gb_ctx* ctx, double* f_dev);

/* IC(0) of the permuted A_h (Sec. 6.4): L L^T = A on the pattern of L, no
 * fill, FP64, level-scheduled on the device; also builds the FP32 copies used
 * by GB_PREC_MIXED.  On GB_ERR_IC0_BREAKDOWN *breakdown_row_host (may be NULL)
 * receives the first offending row in the ordering's numbering. */
int gb_factor_ic0(gb_ctx* ctx, int64_t* breakdown_row_host);

/* Preconditioned MINRES (Sec. 5) on K x = b, K = [A_h B^T; B 0], for k
 * right-hand sides at once, from x_0 = 0.  rhs_dev: [k][n_u + n_p] doubles;
 * the pressure part of each rhs must satisfy 1^T g_p = 0 (K is singular with
 * kernel [0; 1]); a rhs with |1^T g_p| > 1e-10 sqrt(n_p) ||g_p||_2 is not
 * solved (its x is zero, its info status GB_ERR_INVALID_ARG).  The pressure
 * of x is filtered to zero mean, p <- p - (w^T p / w^T 1) 1 (Sec. 6.4).
 * x_dev: [k][n_u + n_p].  info_host: k entries, status GB_OK,
 * GB_ERR_NOT_CONVERGED (max_outer reached; x still written),
 * GB_ERR_NONFINITE (NaN/Inf met) or GB_ERR_INVALID_ARG.  The call returns the
 * most severe per-rhs status (nonfinite > invalid > not converged). */
int gb_solve(gb_ctx* ctx, const double* rhs_dev, double* x_dev, int k,
             const gb_solve_opts* opts, gb_info* info_host);

/* Same as gb_solve with host buffers: rhs_host and x_host are [k][n] host
 * arrays (pinned memory recommended); copies are stream-ordered and the call
 * returns after the results are in x_host. */
int gb_solve_host(gb_ctx* ctx, const double* rhs_host, double* x_host, int k,
                  const gb_solve_opts* opts, gb_info* info_host);

/* Adjoint solve for a loss L(u, p) of a solution of gb_solve: K is symmetric
 * (Sec. 5), so lambda solves K lambda = [dL/du; P^T dL/dp] with the same
 * preconditioned MINRES, where P is the zero-mean pressure filter.
 * grad_dev, lam_dev: [k][n_u + n_p].  dL/df = lambda_u.  Same options/info. */
int gb_solve_adjoint(gb_ctx* ctx, const double* grad_dev, double* lam_dev, int k,
                     const gb_solve_opts* opts, gb_info* info_host);

/* dL/dnu = -lambda_u^T A_0 u for each of k pairs, with A_0 = A_h / nu (A_h is
 * linear in nu, Sec. 3.1 and eq. nitsche_lhs) and f independent of nu.
 * lam_dev, x_dev: [k][n_u + n_p]; out_host: k doubles. */
int gb_dnu(gb_ctx* ctx, const double* lam_dev, const double* x_dev, int k, double* out_host);

/* The same dL/dnu as gb_dnu, computed without allocating any device memory.
 * The paper has no counterpart.  It is meant for callers that cannot call
 * cudaMalloc when they need the viscosity gradient: programs whose device
 * memory is handed out by their own pool or framework, which forbids raw
 * allocations next to it (they would fragment the pool or exceed its
 * budget), and callers that have already spent a fixed memory budget.
 * gb_dnu may allocate the context's solve workspace on first use; this call
 * never does.  Its reduction scratch is a static device array inside the
 * library, sized for k <= 32 and the largest launch (about 304 KiB); every
 * GPU that loads the library holds it until the process exits.  k > 32 is
 * rejected with GB_ERR_INVALID_ARG.  The first call on a device looks up
 * that array's device address (make it before any stream capture).  All
 * calls share the array, so calls that overlap on the GPU race; each call
 * clears the parts that must start at zero.  The call copies the k results
 * to out_host and waits for them on the context's stream before it
 * returns.  The context must be assembled.  Arguments, layout and result are
 * those of gb_dnu. */
int gb_dnu_noalloc(gb_ctx* ctx, const double* lam_dev, const double* x_dev, int k, double* out_host);

/* Spectral diagnostics.  MINRES is the Lanczos process on M^{-1} K in the
 * M-inner product (Sec. 5); after j steps the tridiagonal T_j (diagonal
 * delta_1..delta_j, off-diagonal gamma_2..gamma_j) represents M^{-1} K on the
 * Krylov space, and its eigenvalues (Ritz values) approximate eigenvalues of
 * M^{-1} K, the extremal ones first -- on meshes too large for a dense
 * eigensolver (the paper's Tables neg_and_pos_eig_k_2/k_3 are dense).
 * gb_lanczos: T_j of right-hand side `rhs` (0 <= rhs < k) of the last solve;
 * *count = j; delta_host receives min(j, cap) values delta_1.., gamma_host
 * min(j+1, cap+1) values gamma_1, gamma_2, .. (gamma_1 = ||b||_{M^{-1}}).
 * Either pointer may be NULL.  Without a completed solve: GB_ERR_INVALID_ARG.
 * gb_ritz_extremes: out_host[0..3] = lambda^-_min, lambda^-_max, lambda^+_min,
 * lambda^+_max of the Ritz values (bisection on Sturm sequences, host);
 * exclude_one != 0 skips Ritz values within 1e-6 of 1 (the paper discards the
 * eigenvalue 1, of multiplicity n_u - n_p when M_A = A_h); NaN where a side
 * has no Ritz value. */
int gb_lanczos(gb_ctx* ctx, int rhs, double* delta_host, double* gamma_host, int cap, int* count);
int gb_ritz_extremes(gb_ctx* ctx, int rhs, int exclude_one, double* out_host);

/* y = K x (which = 0), y_u = A_h x_u (which = 1), y_p = B x_u (which = 2),
 * y_u = B^T x_p (which = 3), y_p = Q x_p (which = 4, the pressure mass
 * matrix), all in natural numbering, FP64, one vector.
 * x_dev / y_dev sizes follow the operator. */
int gb_apply(gb_ctx* ctx, int which, const double* x_dev, double* y_dev);

/* Kernel layout of single-right-hand-side solves (k == 1) for one precision
 * (GB_PREC_*).  spmv: 0 CSR with 8 lanes per row, 1 SELL-32 with one thread
 * per row, 2 / 3 SELL-32 with 2 / 4 warps per 32-row slice.  trsv (the IC(0) sweeps): 0 CSR, 1 SELL-32, 2 / 3 / 4 staged (each
 * block stages its rows of a level in shared memory and gathers the solution
 * entries they need in one round trip; about 4 / 12 / 32 entries per lane),
 * 5 / 6 packed (the staged scheme on a k-major copy of each block, so that a
 * warp gathers the same stencil entry of neighbouring rows; about 12 / 32
 * entries per lane), 7 / 8 split packed (the packed scheme with each row's
 * entries split by the level of their column: a level sums the entries of
 * levels two or more steps back before it waits for the level just before it,
 * and releases the next level only after that wait; about 12 / 32 entries per
 * lane), 9 SELL-32 with 1 / 2 / 4 / 8 warps per 32-row slice chosen per level
 * from its longest row (every lane loads up to 12 of its slots before the
 * wait for the previous level and then gathers them at once), 10 the same
 * slice groups streamed into shared memory by bulk copies (cp.async.bulk with
 * an mbarrier), two stages per block, the first two groups fetched before the
 * wait (available when every factor row has at most 88 off-diagonal entries:
 * 2D with velocity degree 3), 11 the SELL form of 9 with four slots loaded
 * before the wait and the rest read in a loop (W for about 16 slots per lane;
 * few registers, many warps per SM), 12 the same with about 8 slots per lane,
 * 13 the form of 11 on a grid of the resident blocks, each taking several
 * slice groups of a level in turn, 14 the form of 11 with about 32 slots per
 * lane, 15 the form of 11 with two slots loaded before the wait, 16 / 17 the
 * form of 11 with about 24 / 48 slots per lane, 18 the form of 14 whose
 * levels of one warp per slice (rows of at most 32 entries) load 12 slots
 * before the wait.
 * -1 automatic.  Automatic (the default) chooses at the first single-RHS
 * solve of that precision: it times the SpMV layouts alone, then each sweep
 * layout inside the graph of a one-step solve of this problem with 12 inner
 * iterations per preconditioner application, and keeps the fastest (a later
 * candidate must be 3 % faster to replace an earlier one).  The layouts
 * differ only in the summation order inside a row.  Values outside
 * these ranges return GB_ERR_INVALID_ARG, and so do trsv 10 when a factor row
 * has more than 88 off-diagonal entries and trsv 2 - 8 when a row of
 * the factor has more than 2048 off-diagonal entries (3D with velocity degree
 * 5 or 6 on all but the coarsest meshes): those layouts are then not built,
 * and the automatic choice skips them.  gb_get_kernel_variants reports the
 * current choice (-1: not made). */
int gb_set_kernel_variants(gb_ctx* ctx, int precision, int spmv, int trsv);
int gb_get_kernel_variants(const gb_ctx* ctx, int precision, int* spmv, int* trsv);

/* IC(0) sweep kernel of batched solves (k > 1; width 8 for k <= 8, 32 for
 * k <= 32) for one precision: 0 one row per lane group with the column
 * indices read as it goes, 1 staged (each row's indices and values copied to
 * shared memory before the wait for the previous level, then the solution
 * entries loaded 16 at a time), -1 automatic (timed at the first batched
 * solve of that precision and width; the faster by 3 % is kept).  Both sum
 * in the same order.  gb_get_batch_sweep reports the choice (-1: not made). */
int gb_set_batch_sweep(gb_ctx* ctx, int precision, int width, int variant);
int gb_get_batch_sweep(const gb_ctx* ctx, int precision, int width, int* variant);

/* Benchmark instrumentation.  Times `reps` (>= 1) launches of one kernel
 * family of the most recent gb_solve, with the same batch width, precision
 * and launch configuration, on the context's stream with CUDA events, after
 * one untimed launch; *ms_host receives the mean milliseconds per launch.
 *  which 0: inner CG product q = A p with its p^T q reduction (one kernel)
 *        1: one IC(0) preconditioner application, forward then backward
 *           triangular solve over all levels (2 x levels launches)
 *        2: Stokes operator product K z with its reduction (one kernel)
 *        3: forward triangular solve over all levels (levels launches)
 * Before each timed sweep (which 1, 3) an untimed inner CG product runs, so
 * that the factor is read with the L2 contents of a solve (where A_h streams
 * through L2 between preconditioner applications), not from a warm L2.
 * The buffers of the last solve are reused and overwritten (its returned
 * solution is not touched).  GB_ERR_INVALID_ARG before any solve. */
int gb_time_kernel(gb_ctx* ctx, int which, int reps, double* ms_host);

/* Copies internal arrays to the host for inspection and parity tests.
 *  what 0: A_h CSR in natural numbering: rowptr int64 [n_u+1], col int32,
 *          val double (any of the three pointers may be NULL)
 *  what 1: B CSR (natural), same layout ([n_p+1] rowptr)
 *  what 2: IC(0) factor L in the ordering's numbering (lower, diagonal
 *          last in each row), same layout
 *  what 3: ordering: p0 = int32 perm[new] = old (n_u); p1 = int32 forward
 *          level per row in the ordering's numbering; p2 = int32 backward
 *          level
 *  what 4: Diag(Q) (p2 double [n_p]) and w (p1 double [n_p])
 *  what 5: Q CSR in natural numbering: rowptr int32 [n_p+1], col int32,
 *          val double [nnz(Q)]
 *  what 6: the 1D mass matrix Q1 of the degree p-1 B-splines and its
 *          Cholesky factor L1 (after gb_factor_ic0), as bands of
 *          (N + p - 1) x p doubles: p0[a*p + o] = Q1[a][a-o],
 *          p1[a*p + o] = L1[a][a-o] (0 where a < o).  IC(0) of Q in the
 *          natural order equals L1 x L1 (x L1 in 3D). */
int gb_export(gb_ctx* ctx, int what, void* p0, void* p1, void* p2);

/* Releases all device and host memory of the context (NULL is allowed). */
void gb_destroy(gb_ctx* ctx);

const char* gb_status_string(int status);
const char* gb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBSTOKES_H */
