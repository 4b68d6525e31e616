"""GPU parity of the IC(0)-PCG pressure block (Sec. 6.4, "IC(0)-PCG(A,Q)")
against the oracle: the pressure mass matrix Q, its exact IC(0) factor
(L1 x L1 [x L1] in the natural order, Kronecker line solves on the device),
replayed FP64 solves (velocity and pressure inner counts forced) within
1e-10, free-mode mixed precision, batched right-hand sides and the
one-iteration behaviour of the pressure CG."""
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


def pair(oracle_mod, gb, dim, N, p, ordering="natural"):
    ref = oracle_mod.Problem(dim, N, p, ordering=ordering)
    s = gb.Stokes(dim, N, p, ordering=ordering)
    s.assemble(1.0)
    assert ref.factor() < 0 and ref.factor_q() < 0
    s.factor_ic0()
    return ref, s


def fourier_rhs(ref, s, seed):
    from paper_1309_5048_gb300.inputs import fourier_modes
    kappa, amp = fourier_modes(ref.dim, seed=seed)
    b = np.concatenate([ref.load_fourier(kappa, amp), np.zeros(ref.n_p)])
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_fourier(kappa, amp)
    return b, rhs


@pytest.mark.parametrize("dim,N,p", [(2, 7, 3), (3, 3, 3), (2, 5, 4), (2, 1, 2)])
def test_q_matrix_and_factor(oracle_mod, gb, dim, N, p):
    ref, s = pair(oracle_mod, gb, dim, N, p)
    ptr, col, val = s.q_csr()
    rp, rc, rv = ref.csr("Q")
    assert np.array_equal(ptr, rp) and np.array_equal(col, rc)
    np.testing.assert_allclose(val, rv, rtol=1e-13, atol=1e-15 * np.abs(rv).max())
    # IC(0) of Q: the oracle's general factorisation vs the Kronecker product of
    # the device's 1D factor
    m = N + p - 1
    _, l1b = s.q_factor_bands()
    L1 = np.zeros((m, m))
    for a in range(m):
        for o in range(p):
            if a - o >= 0:
                L1[a, a - o] = l1b[a, o]
    K = L1
    for _ in range(dim - 1):
        K = np.kron(K, L1)
    LQ = ref.scipy("LQ").toarray()
    assert np.abs(K - LQ).max() <= 1e-13 * np.abs(LQ).max()
    rng = np.random.default_rng(3)
    x = rng.standard_normal(s.n_p)
    np.testing.assert_allclose(s.apply("Q", x).cpu().numpy(), ref.scipy("Q") @ x, rtol=1e-12,
                               atol=1e-14 * np.abs(rv).max() * np.abs(x).max())


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("ordering", ["natural", "multicolour"])
@pytest.mark.parametrize("dim,N,p", [(2, 12, 3), (3, 4, 3), (2, 9, 4)])
def test_pcg_pressure_replay_parity(oracle_mod, gb, use_graph, ordering, dim, N, p):
    """FP64, both inner count lists of the oracle replayed: rel diff <= 1e-10."""
    ref, s = pair(oracle_mod, gb, dim, N, p, ordering)
    b, rhs = fourier_rhs(ref, s, 7)
    xr, ir = ref.minres(b, tol=1e-8, inner_tol=1e-2, pressure="pcg")
    assert ir["status"] == 0
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, pressure="pcg", forced=ir["counts"],
                      forced_q=ir["qcounts"], use_graph=use_graph)
    assert info["outer_its"] == ir["outer"]
    assert info["inner_its_total"] == int(ir["counts"].sum())
    assert info["q_inner_its_total"] == int(ir["qcounts"].sum())
    assert rel(x.cpu().numpy(), xr) <= 1e-10


def test_pcg_pressure_free_mode_and_one_iteration(oracle_mod, gb):
    """Without replay: the pressure CG takes one iteration per application
    (the factor is exact), the outer count drops well below the Diag(Q)
    one, and FP64 / mixed solves agree with the oracle."""
    ref, s = pair(oracle_mod, gb, 2, 16, 3, "multicolour")
    b, rhs = fourier_rhs(ref, s, 5)
    xr, ir = ref.minres(b, tol=1e-10, inner_tol=1e-2, pressure="pcg")
    for precision, bound in (("fp64", 1e-9), ("mixed", 1e-7)):
        x, info = s.solve(rhs, tol=1e-10, inner_tol=1e-2, pressure="pcg", precision=precision)
        assert info["status"] == 0
        assert info["q_inner_its_max"] == 1
        assert info["q_inner_its_total"] == info["outer_its"]  # the first application has no pressure part
        assert rel(x.cpu().numpy(), xr) <= bound
    _, i_diag = s.solve(rhs, tol=1e-10, inner_tol=1e-2)
    assert info["outer_its"] < 0.5 * i_diag["outer_its"]


def test_pcg_pressure_batched(oracle_mod, gb):
    from paper_1309_5048_gb300.inputs import fourier_modes
    ref, s = pair(oracle_mod, gb, 2, 10, 3, "multicolour")
    k = 5
    rhs = torch.zeros(k, s.n, dtype=torch.float64, device="cuda")
    bs = []
    for t in range(k):
        kappa, amp = fourier_modes(2, seed=200 + t)
        rhs[t, : s.n_u] = s.load_fourier(kappa, amp)
        bs.append(np.concatenate([ref.load_fourier(kappa, amp), np.zeros(ref.n_p)]))
    for precision, bound in (("fp64", 1e-9), ("mixed", 1e-7)):
        X, infos = s.solve(rhs, tol=1e-11, inner_tol=1e-2, pressure="pcg", precision=precision)
        X = X.cpu().numpy()
        for t in range(k):
            xr, _ = ref.minres(bs[t], tol=1e-11, inner_tol=1e-2, pressure="pcg")
            assert infos[t]["status"] == 0 and infos[t]["q_inner_its_max"] == 1
            assert rel(X[t], xr) <= bound, (precision, t, rel(X[t], xr))


def test_pcg_pressure_argument_checks(oracle_mod, gb):
    ref, s = pair(oracle_mod, gb, 2, 4, 3)
    _, rhs = fourier_rhs(ref, s, 1)
    with pytest.raises(gb.GbError):
        s.solve(rhs, forced_q=[1, 1, 1])  # pressure replay needs the PCG block
    with pytest.raises(gb.GbError):
        s.solve(torch.stack([rhs, rhs]), pressure="pcg", forced_q=[1, 1])  # replay needs k == 1
