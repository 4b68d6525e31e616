"""Pins of the oracle's B-spline basis and quadrature (Sec. 2.1).

Each check compares the oracle with something other than itself: numpy's
Gauss-Legendre routine, scipy's independent B-spline implementation, exact
rational integration with sympy, and finite differences.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline


def open_knots(N, q):
    return np.concatenate([np.zeros(q), np.arange(N + 1) / N, np.ones(q)])


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_legendre_matches_numpy_and_is_exact(oracle_mod, n):
    x, w = oracle_mod.gauss(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-14)
    np.testing.assert_allclose(w, wr, atol=1e-14)
    for k in range(2 * n):  # exact for degree <= 2n-1
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("N", [1, 3, 7])
def test_basis_matches_scipy_bspline(oracle_mod, q, N):
    t = open_knots(N, q)
    rng = np.random.default_rng(q * 10 + N)
    for e in range(N):
        for x in np.concatenate([[e / N, (e + 1) / N], e / N + rng.random(4) / N]):
            v, d = oracle_mod.basis(N, q, e, x)
            for t_i in range(q + 1):
                i = e + t_i
                c = np.zeros(N + q)
                c[i] = 1.0
                s = BSpline(t, c, q, extrapolate=False)
                # evaluate inside the element (right end from the left)
                xe = min(x, (e + 1) / N - 1e-15) if x >= (e + 1) / N else x
                ref = s(xe)
                dref = s.derivative()(xe)
                assert abs(v[t_i] - ref) < 1e-12
                assert abs(d[t_i] - dref) < 1e-9 * max(1.0, abs(dref))


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_partition_of_unity_and_derivative_by_finite_differences(oracle_mod, q):
    N = 5
    for e in range(N):
        for x in np.linspace(e / N + 1e-3, (e + 1) / N - 1e-3, 5):
            v, d = oracle_mod.basis(N, q, e, x)
            assert abs(v.sum() - 1.0) < 1e-14
            assert abs(d.sum()) < 1e-11
            h = 1e-6
            vp, _ = oracle_mod.basis(N, q, e, x + h)
            vm, _ = oracle_mod.basis(N, q, e, x - h)
            np.testing.assert_allclose(d, (vp - vm) / (2 * h), atol=1e-6 * q * N * N)


def test_pressure_mass_is_exact_rational_kronecker(oracle_mod):
    """Q of the 2D pressure space (degree p-1) equals Q1 (x) Q1 where Q1 is the
    1D B-spline Gram matrix integrated exactly with sympy (Sec. 3.2, Q_h is a
    tensor-product space on the identity map)."""
    import sympy as sp
    N, p = 3, 3
    q = p - 1
    X = sp.Symbol("x")
    knots = [sp.Integer(0)] * q + [sp.Rational(k, N) for k in range(N + 1)] + [sp.Integer(1)] * q
    basis = sp.bspline_basis_set(q, knots, X)
    n = len(basis)
    Q1 = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            Q1[i, j] = float(sp.integrate(basis[i] * basis[j], (X, 0, 1)))
    P = oracle_mod.Problem(2, N, p)
    Q = P.scipy("Q").toarray()
    np.testing.assert_allclose(Q, np.kron(Q1, Q1), atol=1e-15)
    # integral of each pressure function: closed form (xi_{k+q+1} - xi_k)/(q+1) per direction
    t = [float(v) for v in knots]
    w1 = np.array([(t[k + q + 1] - t[k]) / (q + 1) for k in range(n)])
    np.testing.assert_allclose(P.wmean(), np.kron(w1, w1), atol=1e-15)
