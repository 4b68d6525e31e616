"""The lid-driven cavity of Sec. 6.4 in the oracle.

* The load: the Nitsche right-hand side of eq. nitsche_rhs with lid velocity
  e_1 on x_dim = 1, computed by the oracle with face quadrature, against its
  closed form built here from scipy B-splines: only the first velocity
  component contributes, l = 2 nu prod_{m != k} int B_{a_m} *
  (-(1/2) B'_{a_k}(1) + (C_pen / h) B_{a_k}(1)).
* The MINRES counts of Tables niter_cavity_k_2 and ic_pgc_tols_k2 within 15 %
  (2-norm stop at 1e-12).  The paper's velocity space has two more DOFs
  than the one built here (its size tables exceed the closed-form counts by
  2), most likely at corners, and the cavity's singularity sits at the lid's
  corners, so exact counts are not expected here (the square-domain tables
  are pinned exactly).  The mean inner PCG(A) counts are held to 15 % for
  the IC(0) blocks and 25 % for the diagonally preconditioned ones.
  Excluded: PCG(A,Q) at h = 1/8, whose printed mean inner count (14.3) is
  half of what a diagonally preconditioned CG needs here (29.6).
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from conftest import read_golden


def _knots(N, q):
    return np.concatenate([np.zeros(q), np.linspace(0.0, 1.0, N + 1), np.ones(q)])


def _spline(N, q, a):
    c = np.zeros(N + q)
    c[a] = 1.0
    return BSpline(_knots(N, q), c, q)


@pytest.mark.parametrize("dim,N,p", [(2, 6, 3), (2, 4, 4), (3, 3, 3), (2, 5, 2)])
def test_cavity_load_closed_form(oracle_mod, dim, N, p):
    P = oracle_mod.Problem(dim, N, p, nu=0.7)
    f = P.load_cavity()
    m = N + p - 1  # degree p-1 functions per direction
    k = dim - 1
    want = np.zeros(P.n_u)
    # first velocity component: degree p in x (first and last removed), p-1 elsewhere
    shape = [N + p - 2] + [m] * (dim - 1)
    for idx in np.ndindex(*shape):
        a = list(idx)
        a[0] += 1
        b = _spline(N, p - 1, a[k])
        end = -0.5 * b.derivative()(1.0) + P.cpen * N * b(1.0)
        w = 1.0
        for d in range(dim):
            if d != k:
                q = p if d == 0 else p - 1
                w *= _spline(N, q, a[d]).integrate(0.0, 1.0)
        flat = 0
        for d in range(dim):
            flat = flat * shape[d] + idx[d]
        want[flat] = 2.0 * P.nu * w * end
    np.testing.assert_allclose(f, want, rtol=1e-12, atol=1e-13 * np.abs(want).max())
    assert np.count_nonzero(f) == np.count_nonzero(want) > 0


COLS = ["Ideal(A,Q)", "PCG(A,Q)", "Ideal(A),Diag(Q)", "PCG(A),Diag(Q)", "Diag(A,Q)"]
CASES = [(h, c) for h in (8, 16, 32) for c in COLS if (h, c) != (8, "PCG(A,Q)")]


@pytest.mark.parametrize("inv_h,col", CASES)
def test_cavity_counts_near_paper(oracle_mod, inv_h, col):
    rows = {r[0]: r[1:] for r in read_golden("paper_niter_cavity.txt") if r[0] != "ic0"}
    want = rows[str(inv_h)][COLS.index(col)]
    P = oracle_mod.Problem(2, inv_h, 3, ordering="rcm")
    assert P.factor() < 0 and P.factor_q() < 0
    b = np.concatenate([P.load_cavity(), np.zeros(P.n_p)])
    opts = {"Ideal(A,Q)": dict(velocity="ic0_pcg", pressure="pcg", inner_tol=1e-14),
            "PCG(A,Q)": dict(velocity="jacobi_pcg", pressure="jacobi_pcg", inner_tol=1e-6),
            "Ideal(A),Diag(Q)": dict(velocity="ic0_pcg", pressure="diag", inner_tol=1e-14),
            "PCG(A),Diag(Q)": dict(velocity="jacobi_pcg", pressure="diag", inner_tol=1e-6),
            "Diag(A,Q)": dict(velocity="diag", pressure="diag")}[col]
    _, info = P.minres(b, tol=1e-12, max_outer=20000, max_inner=5000, **opts)
    assert info["status"] == 0
    outer = int(want.split("/")[0])
    assert abs(info["outer"] - outer) <= 0.15 * outer, (info["outer"], want)
    if col == "PCG(A,Q)":
        mean_a = float(want.split("/")[1])
        assert abs(info["counts"][1:].mean() - mean_a) <= 0.25 * mean_a


@pytest.mark.parametrize("inv_h", [8, 16, 32])
def test_cavity_ic0_pcg_counts_near_paper(oracle_mod, inv_h):
    """Table ic_pgc_tols_k2: RCM orderings of A and Q, IC(0)-PCG blocks."""
    rows = {int(r[1]): r[2:] for r in read_golden("paper_niter_cavity.txt") if r[0] == "ic0"}
    P = oracle_mod.Problem(2, inv_h, 3, ordering="rcm", qordering="rcm")
    assert P.factor() < 0 and P.factor_q() < 0
    b = np.concatenate([P.load_cavity(), np.zeros(P.n_p)])
    for tol, want in zip((1e-3, 1e-6), rows[inv_h]):
        outer, mean_a, mean_q = (float(v) for v in want.split("/"))
        _, info = P.minres(b, tol=1e-12, inner_tol=tol, pressure="pcg")
        assert info["status"] == 0
        assert abs(info["outer"] - outer) <= 0.15 * outer, (tol, info["outer"], want)
        assert abs(info["counts"].mean() - mean_a) <= 0.15 * mean_a, (tol, info["counts"].mean(), want)
        assert np.all(info["qcounts"][1:] == mean_q)
