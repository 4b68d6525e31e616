"""GPU spectral diagnostics: the Lanczos tridiagonal recorded
by the device MINRES equals the oracle's under replay, and the library's
host-side bisection (gb_ritz_extremes) gives the eigenvalues of that
tridiagonal; at h = 1/32 they reproduce the paper's Table neg_and_pos_eig_k_2."""
import numpy as np
import pytest
import scipy.linalg as sl

from conftest import read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_5048_gb300 as m
    m.load_library()
    return m


def test_lanczos_record_and_ritz_extremes(oracle_mod, gb):
    ref = oracle_mod.Problem(2, 10, 3, ordering="multicolour")
    s = gb.Stokes(2, 10, 3, ordering="multicolour")
    s.assemble(1.0)
    assert ref.factor() < 0
    s.factor_ic0()
    b = np.concatenate([ref.load_manufactured(), np.zeros(ref.n_p)])
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_manufactured()
    xr, ir = ref.minres(b, tol=1e-10, inner_tol=1e-2)
    x, info = s.solve(rhs, tol=1e-10, inner_tol=1e-2, forced=ir["counts"])
    d, g = s.lanczos()
    assert len(d) == info["outer_its"] == len(ir["delta"])
    np.testing.assert_allclose(d, ir["delta"], rtol=1e-10, atol=1e-12 * np.abs(ir["delta"]).max())
    np.testing.assert_allclose(g, ir["gamma"], rtol=1e-10)
    r = sl.eigvalsh_tridiagonal(d, g[1:len(d)])
    want = np.array([r[r < 0].min(), r[r < 0].max(), r[r > 0].min(), r.max()])
    np.testing.assert_allclose(s.ritz_extremes(), want, rtol=1e-12)
    with pytest.raises(gb.GbError):
        s.lanczos(rhs=1)  # only one right-hand side was solved


@pytest.mark.parametrize("block", ["diag", "ideal_diag"])
def test_ritz_extremes_match_paper_table(gb, block):
    want = {r[1]: [float(v) for v in r[2:]] for r in read_golden("paper_spectra.txt") if r[0] == "2"}[block]
    s = gb.Stokes(2, 32, 3)
    s.assemble(1.0)
    s.factor_ic0()
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_manufactured()
    opts = dict(velocity="diag") if block == "diag" else dict(inner_tol=1e-14)
    _, info = s.solve(rhs, tol=1e-13, max_outer=20000, max_inner=5000, **opts)
    assert info["status"] == 0
    np.testing.assert_allclose(s.ritz_extremes(exclude_one=block == "ideal_diag"), want, rtol=5e-3)
