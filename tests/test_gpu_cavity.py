"""GPU parity for the lid-driven cavity (Sec. 6.4): the Nitsche load of
eq. nitsche_rhs against the oracle's face quadrature, and replayed solves
with the paper's best strategy, IC(0)-PCG(A,Q) with A reordered by RCM."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_5048_gb300 as m
    m.load_library()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dim,N,p,nu", [(2, 6, 3, 1.0), (3, 3, 3, 0.5), (2, 4, 4, 2.0), (2, 1, 2, 1.0)])
def test_cavity_load(oracle_mod, gb, dim, N, p, nu):
    ref = oracle_mod.Problem(dim, N, p, nu=nu)
    s = gb.Stokes(dim, N, p)
    s.assemble(nu)
    f = s.load_cavity().cpu().numpy()
    fr = ref.load_cavity()
    np.testing.assert_allclose(f, fr, rtol=1e-12, atol=1e-13 * np.abs(fr).max())


@pytest.mark.parametrize("ordering", ["rcm", "multicolour"])
@pytest.mark.parametrize("inner_tol", [1e-3, 1e-6])
def test_cavity_replay_parity(oracle_mod, gb, ordering, inner_tol):
    ref = oracle_mod.Problem(2, 12, 3, ordering=ordering)
    s = gb.Stokes(2, 12, 3, ordering=ordering)
    s.assemble(1.0)
    assert ref.factor() < 0 and ref.factor_q() < 0
    s.factor_ic0()
    b = np.concatenate([ref.load_cavity(), np.zeros(ref.n_p)])
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_cavity()
    xr, ir = ref.minres(b, tol=1e-12, inner_tol=inner_tol, pressure="pcg")
    assert ir["status"] == 0
    x, info = s.solve(rhs, tol=1e-12, inner_tol=inner_tol, pressure="pcg", forced=ir["counts"],
                      forced_q=ir["qcounts"])
    assert info["outer_its"] == ir["outer"]
    assert rel(x.cpu().numpy(), xr) <= 1e-10
    assert info["relres_true"] <= 1.01e-12
