// oracle.hpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded FP64 CPU restatement of the method of
// Cortes & Coutinho, "Performance Evaluation of Block Diagonal Preconditioners
// for Divergence-Conforming B-Spline Discretization of Stokes Equations"
// (arXiv:1309.5048).  It exists to check the CUDA library against, and to be
// timed as the CPU baseline.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg may load it; the product path never does.  It
// shares no code, header, table or constant with the CUDA library.
//
// Contents (each function cites the passage it follows):
//   spline.cpp    Sec. 2.1  open knot vectors, Cox-de Boor recursion,
//                            Gauss-Legendre rules
//   assembly.cpp  Sec. 3.2, Sec. 4  spaces V_{0,h}, Q_h, numbering, element-
//                            loop quadrature of A_h = a - eta_h, B, Q, loads,
//                            error norms of the Sec. 6.2 manufactured solution
//   ordering.cpp  Sec. 6.4 (RCM before IC(0)), level sets of the IC(0) DAG
//   solvers.cpp   Sec. 5   IC(0), inner PCG, preconditioned MINRES, pressure
//                            filter, adjoint quantities
//   capi.cpp      extern "C" wrappers used through ctypes by the tests
#pragma once
#include <cstdint>
#include <vector>

namespace oracle {

// Compressed sparse rows, FP64 values, sorted column indices per row.
struct Csr {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
  // position of column j in row i, or -1
  int64_t find(int64_t i, int32_t j) const;
};

// ---------------------------------------------------------------- spline.cpp
// Uniform open knot vector on [0,1] with N elements, degree q, maximal
// continuity: {0 (q+1 times), 1/N, ..., (N-1)/N, 1 (q+1 times)}; N+q functions.
struct Knots {
  int N = 0, q = 0;
  std::vector<double> xi;
  int nfun() const { return N + q; }
};
Knots open_uniform(int N, int q);
// Values and first derivatives, at x in element e (x in [e/N,(e+1)/N]), of the
// q+1 functions that are nonzero there: function indices e .. e+q.
void eval_basis(const Knots& K, int e, double x, double* val, double* der);
// Value and derivative of one function i at x (evaluated on element e).
void eval_one(const Knots& K, int i, int e, double x, double* val, double* der);
// n-point Gauss-Legendre rule on [-1,1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// -------------------------------------------------------------- assembly.cpp
struct Problem {
  int dim = 2, N = 8, p = 3;
  double nu = 1.0, cpen = 15.0;
  // velocity component c has degree p in direction c and p-1 elsewhere; its
  // first and last functions in direction c are removed (no penetration).
  int64_t nvc[3] = {0, 0, 0};   // DOFs per velocity component
  int64_t voff[3] = {0, 0, 0};  // first global index of component c
  int64_t n_u = 0, n_p = 0;
  Knots Kp, Kq;  // degree p and degree p-1 knot vectors
  Csr A, B, Q;   // natural numbering; B is n_p x n_u
  std::vector<double> wmean;  // w_k = integral of pressure function k

  int deg(int c, int k) const { return k == c ? p : p - 1; }
  int vlen(int c, int k) const { return k == c ? N + p - 2 : N + p - 1; }
  int plen() const { return N + p - 1; }
  // global velocity index of component c with 1D function indices a[]
  int64_t vindex(int c, const int* a) const;
  void vdecode(int64_t i, int* c, int* a) const;
  int64_t pindex(const int* a) const;
  void pdecode(int64_t k, int* a) const;
};

// Build spaces, patterns and the matrices A_h, B, Q (Sec. 4, the discrete
// Stokes system).  If rows_u / rows_p are non-null only the flagged rows are
// assembled (others stay empty): used to sample rows of very large problems.
void setup_problem(Problem& P, int dim, int N, int p, double nu, double cpen,
                   const std::vector<char>* rows_u = nullptr,
                   const std::vector<char>* rows_p = nullptr);
// Load vector f_i = (f, Phi_i) for the Fourier forcing
// f_d(x) = sum_m amp[m][d] prod_k sin(pi kappa[m][k] x_k).
void load_fourier(const Problem& P, int nmodes, const int* kappa, const double* amp,
                  std::vector<double>& f);
// Load vector for the Sec. 6.2 manufactured solution (2D only).
void load_manufactured(const Problem& P, std::vector<double>& f);
// Lid-driven cavity (Sec. 6.4): f = 0 and the Nitsche load l_h of
// eq. nitsche_rhs with lid velocity e_1 on the face x_dim = 1.
void load_cavity(const Problem& P, std::vector<double>& f);
// Errors |u-u_h|_{H1}, ||u-u_h||_{L2}, ||p-p_h||_{L2} for Sec. 6.2 (2D only).
void manufactured_errors(const Problem& P, const double* u, const double* p, double out[3]);
// Exact manufactured fields at (x,y): u1,u2,p,f1,f2 (for pinning).
void manufactured_point(double nu, double x, double y, double out[5]);

// -------------------------------------------------------------- ordering.cpp
// perm[new] = old.  kind 0 natural, 1 reverse Cuthill-McKee, 2 multicolour.
void make_ordering(const Problem& P, int kind, std::vector<int32_t>& perm);
// Colour of velocity DOF i (natural numbering) in the multicolour ordering.
int64_t velocity_colour(const Problem& P, int64_t i);
// The same three orderings of the pressure space, applied to Q before its
// IC(0) (Sec. 6.4 reorders A and Q separately by reverse Cuthill-McKee).
void make_pressure_ordering(const Problem& P, int kind, std::vector<int32_t>& perm);
// Lower-triangular pattern of perm A perm^T (diagonal included, sorted).
void lower_pattern(const Csr& A, const std::vector<int32_t>& perm, Csr& L);
// level(i) = 0 without off-diagonal entries, else 1 + max level(k) over
// L_ik != 0 (k < i).  rlevel is the same for L^T (the reverse DAG).
void level_sets(const Csr& L, std::vector<int32_t>& level, std::vector<int32_t>& rlevel);

// --------------------------------------------------------------- solvers.cpp
// IC(0) of perm A perm^T on pattern L (values overwritten).  Returns -1 on
// success, else the (permuted) row where the pivot was not positive.
int64_t ic0(const Csr& A, const std::vector<int32_t>& perm, Csr& L);

// Pressure block of the preconditioner (Sec. 5.1): Diag(Q_nu), or Q_nu
// approximated by a CG solve with the same relative tolerance and cap as the
// velocity block, preconditioned by IC(0) of Q ("IC(0)-PCG(A,Q)", Sec. 6.4)
// or by the diagonal of Q ("PCG(A,Q)", Sec. 6.2).
enum PressureBlock { PRESSURE_DIAG = 0, PRESSURE_PCG = 1, PRESSURE_JACOBI_PCG = 2 };
// Velocity block (Sec. 5.1): a CG solve with A_h preconditioned by IC(0)
// ("PCG(A)" of Sec. 6.4), Diag(A_h) ("Diag(A,Q)"), or a CG solve
// preconditioned by the diagonal of A_h ("PCG(A)" of Sec. 6.2).
enum VelocityBlock { VELOCITY_IC0_PCG = 0, VELOCITY_DIAG = 1, VELOCITY_JACOBI_PCG = 2 };

struct Precond {
  const Problem* P;
  const Csr* L;                  // IC(0) factor of A_h, permuted numbering
  const std::vector<int32_t>* perm;
  double inner_tol;
  int max_inner;
  const int32_t* forced = nullptr;  // replay: inner counts per application
  int64_t nforced = 0;
  int pressure = PRESSURE_DIAG;
  int velocity = VELOCITY_IC0_PCG;
  const Csr* LQ = nullptr;       // IC(0) factor of Q (PRESSURE_PCG)
  const std::vector<int32_t>* permQ = nullptr;
  const int32_t* forced_q = nullptr;  // replay: pressure CG counts per application
  int64_t nforced_q = 0;
  // outputs
  std::vector<int32_t> counts;   // inner iterations of each application
  std::vector<int32_t> qcounts;  // pressure CG iterations of each application
};
// MINRES stopping rule: the 2-norm relative residual ||b - K x_j|| / ||b||
// (the paper's "relative residual", Sec. 6.2; it reproduces the iteration
// counts of Table niter_square_k_2), or the recurrence's M^{-1}-norm
// estimate |eta_j| / gamma_1 (eq. minimax_precond).
enum StopRule { STOP_RESIDUAL = 0, STOP_ESTIMATE = 1 };
struct MinresInfo {
  int outer = 0;
  double relres_est = 0, relres_true = 0;
  int status = 0;  // 0 converged, 1 hit max_outer, 2 breakdown
  std::vector<double> hist;   // |eta|/gamma_1 after each step
  std::vector<double> hist2;  // ||b - K x_j|| / ||b|| after each step (STOP_RESIDUAL)
  // Lanczos tridiagonal T_j of M^{-1} K in the M-inner product: diagonal
  // delta_1..delta_j and off-diagonal gamma_2..gamma_{j+1} (gamma[0] = gamma_1)
  std::vector<double> delta, gamma;
};
void spmv(const Csr& M, const double* x, double* y);
void stokes_apply(const Problem& P, const double* x, double* y);
int pcg_ic0(const Problem& P, Precond& M, const double* b, double* x, int forced_its);
// The same CG on the pressure mass matrix Q with its IC(0) factor.
int pcg_ic0_q(const Problem& P, Precond& M, const double* b, double* x, int forced_its);
// CG with the diagonal (Jacobi) preconditioner of Mat, same stopping rule.
int pcg_jacobi(const Csr& Mat, double tol, int max_it, const double* b, double* x, int forced_its);
void precond_apply(const Problem& P, Precond& M, const double* r, double* z);
void minres(const Problem& P, Precond& M, const double* b, double* x, double tol,
            int max_outer, MinresInfo& info, int stop_rule = STOP_RESIDUAL);
void pressure_filter(const Problem& P, double* pres);

}  // namespace oracle
