"""Ritz values of the MINRES Lanczos tridiagonal (spectral diagnostics):
the eigenvalues of T_j recorded by the oracle's MINRES
approximate the extremal eigenvalues of M^{-1} K.  Pinned against a dense
generalised eigensolve at h = 1/8 and against the paper's Table
neg_and_pos_eig_k_2 (Sec. 6.4, h = 1/32, the eigenvalues 0 and 1 disregarded)."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

from conftest import read_golden

BLOCKS = {"diag": dict(velocity="diag", pressure="diag"),
          "ideal_diag": dict(velocity="ic0_pcg", pressure="diag", inner_tol=1e-14)}


def ritz_extremes(info, exclude_one):
    d, g = info["delta"], info["gamma"]
    r = sl.eigvalsh_tridiagonal(d, g[1:len(d)])
    if exclude_one:
        r = r[np.abs(r - 1.0) > 1e-6]
    neg, pos = r[r < 0], r[r > 0]
    return np.array([neg.min(), neg.max(), pos.min(), pos.max()])


def solve(oracle_mod, N, p, block):
    P = oracle_mod.Problem(2, N, p)
    if block == "ideal_diag":
        assert P.factor() < 0
    b = np.concatenate([P.load_manufactured(), np.zeros(P.n_p)])
    _, info = P.minres(b, tol=1e-13, max_outer=20000, max_inner=5000, **BLOCKS[block])
    assert info["status"] == 0
    assert len(info["delta"]) == info["outer"] and len(info["gamma"]) == info["outer"] + 1
    return P, info


@pytest.mark.parametrize("block", ["diag", "ideal_diag"])
def test_ritz_extremes_match_dense_spectrum(oracle_mod, block):
    P, info = solve(oracle_mod, 8, 3, block)
    A, B, Q = P.scipy("A"), P.scipy("B"), P.scipy("Q")
    K = sp.bmat([[A, B.T], [B, None]]).toarray()
    Mu = np.diag(A.diagonal()) if block == "diag" else A.toarray()
    M = sl.block_diag(Mu, np.diag(Q.diagonal() / (2.0 * P.nu)))
    ev = sl.eigh(K, M, eigvals_only=True)
    ev = ev[np.abs(ev) > 1e-9]  # the pressure null space
    if block == "ideal_diag":
        ev = ev[np.abs(ev - 1.0) > 1e-6]
    dense = np.array([ev[ev < 0].min(), ev[ev < 0].max(), ev[ev > 0].min(), ev.max()])
    ritz = ritz_extremes(info, block == "ideal_diag")
    # the outer extremes converge first (1e-9 here); the two next to 0 last:
    # by the time MINRES reaches 1e-13 they agree to 2e-6 (Diag) / 4e-4 (Ideal)
    np.testing.assert_allclose(ritz[[0, 3]], dense[[0, 3]], rtol=1e-8)
    np.testing.assert_allclose(ritz[[1, 2]], dense[[1, 2]], rtol=1e-3)


@pytest.mark.parametrize("block", ["diag", "ideal_diag"])
def test_ritz_extremes_match_paper_table(oracle_mod, block):
    want = {r[1]: [float(v) for v in r[2:]] for r in read_golden("paper_spectra.txt")
            if r[0] == "2" and not r[0].startswith("#")}[block]
    _, info = solve(oracle_mod, 32, 3, block)
    ritz = ritz_extremes(info, block == "ideal_diag")
    np.testing.assert_allclose(ritz, want, rtol=5e-3)
