"""The IC(0)-PCG pressure block of the oracle (Sec. 6.4, "IC(0)-PCG(A,Q)")
pinned against the mathematics and the paper's tables.

Q is the Kronecker product of 1D mass matrices of the degree-(p-1) B-splines
(Q = Q1 x Q1 [x Q1] in the lexicographic numbering), each banded with
half-bandwidth p-1, so its exact Cholesky factor L1 x L1 [x L1] lies inside
the lower pattern of Q: IC(0) loses nothing and equals the dense Cholesky
factor (also after the paper's reverse Cuthill-McKee reordering, not after a
multicolour one).  That is why the paper sees PCG(Q) converge in one
iteration at every mesh size and tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from conftest import read_golden


def _mass_1d(oracle_mod, N, q):
    """1D Gram matrix of the N + q degree-q B-splines on [0, 1] (uniform open
    knots), by Gauss quadrature with q + 1 points per element."""
    gx, gw = oracle_mod.gauss(q + 1)
    M = np.zeros((N + q, N + q))
    for e in range(N):
        for x, w in zip(gx, gw):
            v, _ = oracle_mod.basis(N, q, e, (e + 0.5 * (x + 1.0)) / N)
            M[e:e + q + 1, e:e + q + 1] += 0.5 * w / N * np.outer(v, v)
    return M


@pytest.mark.parametrize("qordering", ["natural", "rcm"])
@pytest.mark.parametrize("dim,N,p", [(2, 8, 3), (2, 6, 4), (3, 3, 3), (2, 5, 2)])
def test_ic0_of_q_is_the_cholesky_factor(oracle_mod, qordering, dim, N, p):
    P = oracle_mod.Problem(dim, N, p, qordering=qordering)
    assert P.factor_q() < 0
    perm, _, _ = P.ordering_arrays_q()
    Q = P.scipy("Q").toarray()
    Lc = np.linalg.cholesky(Q[np.ix_(perm, perm)])
    L = P.scipy("LQ").toarray()
    assert np.abs(L - Lc).max() <= 1e-13 * np.abs(Lc).max()


def test_ic0_of_q_is_inexact_under_multicolour(oracle_mod):
    P = oracle_mod.Problem(2, 8, 3, qordering="multicolour")
    assert P.factor_q() < 0
    perm, _, _ = P.ordering_arrays_q()
    Q = P.scipy("Q").toarray()[np.ix_(perm, perm)]
    L = P.scipy("LQ").toarray()
    assert np.abs(L @ L.T - Q).max() > 1e-3 * np.abs(Q).max()
    # ... but exact on the pattern (the defining property of IC(0))
    pat = (np.tril(Q) != 0) | (np.triu(Q) != 0)
    assert np.abs(np.where(pat, L @ L.T - Q, 0.0)).max() <= 1e-14 * np.abs(Q).max()


@pytest.mark.parametrize("dim,N,p", [(2, 7, 3), (3, 3, 3), (2, 4, 4)])
def test_ic0_of_q_natural_is_kronecker_of_1d_factors(oracle_mod, dim, N, p):
    """Natural order: IC(0)(Q) = L1 x L1 [x L1] with L1 = chol(1D mass matrix)."""
    P = oracle_mod.Problem(dim, N, p)
    assert P.factor_q() < 0
    L1 = np.linalg.cholesky(_mass_1d(oracle_mod, N, p - 1))
    K = L1
    for _ in range(dim - 1):
        K = np.kron(K, L1)
    L = P.scipy("LQ").toarray()
    assert np.abs(L - K).max() <= 1e-13 * np.abs(K).max()


def test_ic_q_sizes_match_paper(oracle_mod):
    """nnz(IC(Q)) of the paper's tables: the oracle at 1/h <= 32, the closed
    form (nnz(Q) + n_p) / 2 of a full-diagonal lower pattern at every size."""
    for kp, inv_h, nnz_ic, *_ in read_golden("paper_ic_q.txt"):
        kp, N, nnz_ic = int(kp), int(inv_h), int(nnz_ic)
        p = kp + 1
        m = N + p - 1
        band = m * (2 * p - 1) - (p - 1) * p  # pairs |a - b| <= p - 1 in 1D
        assert (band ** 2 + m ** 2) // 2 == nnz_ic
        if N <= 32:
            P = oracle_mod.Problem(2, N, p)
            assert P.nnzLQ == nnz_ic


@pytest.mark.parametrize("kp,N", [(2, 8), (2, 16), (3, 8)])
def test_pcg_q_converges_in_one_iteration(oracle_mod, kp, N):
    """Tables tab:ic_pgc_tols_k2/k3: one PCG(Q) iteration per application at
    PCG tolerances 1e-3 and 1e-6 (Fourier forcing instead of the cavity)."""
    from paper_1309_5048_gb300.inputs import fourier_modes
    want = {int(r[1]): r for r in read_golden("paper_ic_q.txt") if int(r[0]) == kp}[N]
    P = oracle_mod.Problem(2, N, kp + 1)
    assert P.factor() < 0 and P.factor_q() < 0
    kappa, amp = fourier_modes(2, seed=1)
    b = np.concatenate([P.load_fourier(kappa, amp), np.zeros(P.n_p)])
    for tol, col in ((1e-3, 3), (1e-6, 4)):
        x, info = P.minres(b, tol=1e-8, inner_tol=tol, pressure="pcg")
        assert info["status"] == 0
        q = info["qcounts"]
        assert len(q) == info["outer"] + 1
        assert q[0] == 0  # the initial residual has no pressure part
        assert np.all(q[1:] == int(want[col]))


def test_pcg_q_solves_q_and_minres_matches_direct_solve(oracle_mod):
    P = oracle_mod.Problem(2, 9, 3, ordering="rcm")
    assert P.factor() < 0 and P.factor_q() < 0
    rng = np.random.default_rng(2)
    r = rng.standard_normal(P.n_p)
    y, its = P.pcg_q(r, 1e-12)
    Q = P.scipy("Q")
    assert its == 1
    assert np.linalg.norm(Q @ y - r) <= 1e-13 * np.linalg.norm(r)
    # the pressure block of the preconditioner is 2 nu Q^{-1} r_p
    z, _ = P.precond(np.concatenate([np.zeros(P.n_u), r]), 1e-12, pressure="pcg")
    np.testing.assert_allclose(z[P.n_u:], 2.0 * P.nu * spl.spsolve(Q.tocsc(), r), rtol=1e-11)
    # MINRES with IC(0)-PCG(A,Q) reaches the direct solution
    f = P.load_manufactured()
    A, B = P.scipy("A"), P.scipy("B")
    w = P.wmean()
    K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(w.reshape(-1, 1))],
                 [None, sp.csr_matrix(w.reshape(1, -1)), None]]).tocsc()
    xd = spl.spsolve(K, np.concatenate([f, np.zeros(P.n_p + 1)]))[:P.n_u + P.n_p]
    b = np.concatenate([f, np.zeros(P.n_p)])
    x, info = P.minres(b, tol=1e-13, inner_tol=1e-3, pressure="pcg")
    assert info["status"] == 0
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    # far fewer MINRES steps than with Diag(Q) (Sec. 6.4)
    _, i_diag = P.minres(b, tol=1e-8, inner_tol=1e-3)
    _, i_pcg = P.minres(b, tol=1e-8, inner_tol=1e-3, pressure="pcg")
    assert i_pcg["outer"] < 0.5 * i_diag["outer"]
    # replay of both inner count lists reproduces the solve exactly
    x1, i1 = P.minres(b, tol=1e-8, inner_tol=1e-3, pressure="pcg")
    x2, _ = P.minres(b, tol=1e-8, inner_tol=1e-3, pressure="pcg", forced=i1["counts"], forced_q=i1["qcounts"])
    assert np.array_equal(x1, x2)
