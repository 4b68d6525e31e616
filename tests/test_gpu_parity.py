"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars (stated per test):
* patterns, orderings, level sets: bit-identical;
* assembled values, loads, IC(0) factor, operator products: relative 1e-12
  (FP64, different summation order);
* plain FP64 solve in replay mode (the oracle's inner-CG counts forced on the
  GPU, so both run the same sequence of operations): relative solution
  difference <= 1e-10;
* free mode: both solutions within their own tolerance of a tight oracle solve;
* mixed precision (FP32 inner preconditioner): relative difference <= 1e-7 to
  the FP64 oracle at an outer tolerance of 1e-10.
"""
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


def make_pair(oracle_mod, gb, dim, N, p, ordering="natural", nu=1.0, cpen=None):
    ref = oracle_mod.Problem(dim, N, p, nu=nu, cpen=cpen, ordering=ordering)
    s = gb.Stokes(dim, N, p, ordering=ordering)
    s.assemble(nu, cpen)
    return ref, s


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [(2, 7, 3), (2, 5, 4), (2, 1, 3), (3, 3, 3), (3, 2, 2)]


@pytest.mark.parametrize("ordering", ["natural", "rcm", "multicolour"])
@pytest.mark.parametrize("dim,N,p", CASES)
def test_patterns_orderings_levels_and_values(oracle_mod, gb, ordering, dim, N, p):
    ref, s = make_pair(oracle_mod, gb, dim, N, p, ordering)
    assert (s.n_u, s.n_p, s.nnzA, s.nnzB, s.nnzL) == (ref.n_u, ref.n_p, ref.nnzA, ref.nnzB, ref.nnzL)
    assert (s.nlevels, s.nrlevels) == (ref.nlevels, ref.nrlevels)
    perm, lev, rlev = s.ordering_arrays()
    rperm, rlev_o, rrlev_o = ref.ordering_arrays()
    assert np.array_equal(perm, rperm)
    assert np.array_equal(lev, rlev_o)
    assert np.array_equal(rlev, rrlev_o)
    for which in ("A", "B"):
        ptr, col, val = s.csr(which)
        rptr, rcol, rval = ref.csr(which)
        assert np.array_equal(ptr, rptr) and np.array_equal(col, rcol)
        assert np.abs(val - rval).max() <= 1e-12 * np.abs(rval).max()
    w, qd = s.pressure_arrays()
    Q = ref.scipy("Q")
    np.testing.assert_allclose(qd, Q.diagonal(), rtol=1e-13)
    np.testing.assert_allclose(w, ref.wmean(), rtol=1e-13)


@pytest.mark.parametrize("dim,N,p", [(2, 9, 3), (2, 6, 4), (3, 3, 3)])
def test_load_vectors(oracle_mod, gb, dim, N, p):
    from paper_1309_5048_gb300.inputs import fourier_modes
    ref, s = make_pair(oracle_mod, gb, dim, N, p, nu=0.9)
    kappa, amp = fourier_modes(dim, seed=3)
    f = s.load_fourier(kappa, amp).cpu().numpy()
    fr = ref.load_fourier(kappa, amp)
    assert np.abs(f - fr).max() <= 1e-12 * np.abs(fr).max()
    if dim == 2:
        f = s.load_manufactured().cpu().numpy()
        fr = ref.load_manufactured()
        assert np.abs(f - fr).max() <= 1e-12 * np.abs(fr).max()


@pytest.mark.parametrize("ordering", ["natural", "rcm", "multicolour"])
@pytest.mark.parametrize("dim,N,p", [(2, 8, 3), (2, 6, 4), (3, 3, 3), (3, 1, 2)])
def test_ic0_factor(oracle_mod, gb, ordering, dim, N, p):
    ref, s = make_pair(oracle_mod, gb, dim, N, p, ordering)
    assert ref.factor() < 0
    s.factor_ic0()
    ptr, col, val = s.csr("L")
    rptr, rcol, rval = ref.csr("L")
    assert np.array_equal(ptr, rptr) and np.array_equal(col, rcol)
    assert np.abs(val - rval).max() <= 1e-12 * np.abs(rval).max()


@pytest.mark.parametrize("dim,N,p", [(2, 8, 3), (3, 3, 3)])
def test_operator_products(oracle_mod, gb, dim, N, p):
    ref, s = make_pair(oracle_mod, gb, dim, N, p, "multicolour")
    rng = np.random.default_rng(1)
    x = rng.standard_normal(ref.n_u + ref.n_p)
    y = s.apply("K", x).cpu().numpy()
    yr = ref.stokes_apply(x)
    assert np.abs(y - yr).max() <= 1e-12 * np.abs(yr).max()
    A, B = ref.scipy("A"), ref.scipy("B")
    xu, xp = x[: ref.n_u], x[ref.n_u:]
    np.testing.assert_allclose(s.apply("A", xu).cpu().numpy(), A @ xu, atol=1e-12 * np.abs(A @ xu).max())
    np.testing.assert_allclose(s.apply("B", xu).cpu().numpy(), B @ xu, atol=1e-12 * np.abs(B @ xu).max())
    np.testing.assert_allclose(s.apply("Bt", xp).cpu().numpy(), B.T @ xp, atol=1e-12 * np.abs(B.T @ xp).max())


def _rhs(ref, s, kind, seed=0):
    from paper_1309_5048_gb300.inputs import fourier_modes
    if kind == "manufactured":
        fr = ref.load_manufactured()
        f = s.load_manufactured()
    else:
        kappa, amp = fourier_modes(ref.dim, seed=seed)
        fr = ref.load_fourier(kappa, amp)
        f = s.load_fourier(kappa, amp)
    b = np.concatenate([fr, np.zeros(ref.n_p)])
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = f
    return b, rhs


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("ordering", ["natural", "multicolour", "rcm"])
@pytest.mark.parametrize("dim,N,p,kind", [(2, 16, 3, "manufactured"), (2, 11, 4, "fourier"),
                                          (3, 4, 3, "fourier"), (2, 1, 2, "fourier")])
def test_solve_replay_parity(oracle_mod, gb, use_graph, ordering, dim, N, p, kind):
    """FP64 solve, inner counts of the oracle replayed: rel diff <= 1e-10."""
    ref, s = make_pair(oracle_mod, gb, dim, N, p, ordering)
    assert ref.factor() < 0
    s.factor_ic0()
    b, rhs = _rhs(ref, s, kind)
    xr, ir = ref.minres(b, tol=1e-8, inner_tol=1e-2)
    assert ir["status"] == 0
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, forced=ir["counts"], use_graph=use_graph)
    x = x.cpu().numpy()
    assert info["outer_its"] == ir["outer"]
    assert info["inner_its_total"] == int(ir["counts"].sum())
    assert rel(x, xr) <= 1e-10
    assert abs(info["relres_est"] - ir["relres_est"]) <= 1e-6 * ir["relres_est"] + 1e-14
    assert abs(info["relres_true"] - ir["relres_true"]) <= 1e-4 * ir["relres_true"] + 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ordering", ["natural", "multicolour"])
def test_solve_free_mode(oracle_mod, gb, precision, ordering):
    """Without replay both solves meet the tolerance and agree with a tight
    oracle solve to the accuracy the tolerance allows."""
    ref, s = make_pair(oracle_mod, gb, 2, 16, 3, ordering)
    assert ref.factor() < 0
    s.factor_ic0()
    b, rhs = _rhs(ref, s, "fourier", seed=5)
    x_tight, _ = ref.minres(b, tol=1e-13, inner_tol=1e-2)
    xr, ir = ref.minres(b, tol=1e-8, inner_tol=1e-2)
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, precision=precision)
    x = x.cpu().numpy()
    assert info["status"] == 0 and info["relres_true"] <= 1.01e-8
    e_ref = rel(xr, x_tight)
    e_gpu = rel(x, x_tight)
    assert e_gpu <= max(10 * e_ref, 1e-7), (e_gpu, e_ref)
    # tighter outer tolerance: both within 1e-7 of each other
    x10, info10 = s.solve(rhs, tol=1e-10, inner_tol=1e-2, precision=precision)
    xr10, _ = ref.minres(b, tol=1e-10, inner_tol=1e-2)
    assert rel(x10.cpu().numpy(), xr10) <= 1e-7


@pytest.mark.parametrize("variant", ["warp", "staged"])
def test_batched_sweep_kernels_agree(oracle_mod, gb, variant):
    """Both batched IC(0) sweep kernels (widths 8 and 32, FP64 and mixed)
    give each column the oracle's solution (free mode).  FP64 at 1e-12 within
    1e-9; mixed at 1e-10 within 10x the error of the oracle's own 1e-10 solve
    against a 1e-13 one (3D: K's condition number turns 1e-10 residuals into
    ~1e-7 solution differences), and at least 1e-6."""
    from paper_1309_5048_gb300.inputs import fourier_modes
    ref, s = make_pair(oracle_mod, gb, 3, 4, 3, "multicolour")
    assert ref.factor() < 0
    s.factor_ic0()
    for prec in ("fp64", "mixed"):
        for w in (8, 32):
            s.set_batch_sweep(prec, w, variant)
    for k in (5, 20):
        rhs = torch.zeros(k, s.n, dtype=torch.float64, device="cuda")
        bs = []
        for t in range(k):
            kappa, amp = fourier_modes(3, seed=300 + t)
            rhs[t, : s.n_u] = s.load_fourier(kappa, amp)
            bs.append(np.concatenate([ref.load_fourier(kappa, amp), np.zeros(ref.n_p)]))
        for prec, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
            X, infos = s.solve(rhs, tol=tol, inner_tol=1e-2, precision=prec)
            X = X.cpu().numpy()
            for t in (0, k - 1):
                xr, _ = ref.minres(bs[t], tol=tol, inner_tol=1e-2)
                assert infos[t]["status"] == 0
                if prec == "fp64":
                    assert rel(X[t], xr) <= 1e-9, (variant, k, prec, t, rel(X[t], xr))
                else:
                    xt, _ = ref.minres(bs[t], tol=1e-13, inner_tol=1e-2)
                    bound = max(10 * rel(xr, xt), 1e-6)
                    assert rel(X[t], xt) <= bound, (variant, k, prec, t, rel(X[t], xt), bound)
    assert s.batch_sweep("fp64", 8) == variant and s.batch_sweep("mixed", 32) == variant


def test_batched_columns_match_single_solves(oracle_mod, gb):
    """k right-hand sides in one launch (K = 8 and K = 32 layouts): each
    column equals its own single solve to the tolerance's accuracy and all
    meet the stopping rule."""
    from paper_1309_5048_gb300.inputs import fourier_modes
    ref, s = make_pair(oracle_mod, gb, 2, 12, 3, "multicolour")
    assert ref.factor() < 0
    s.factor_ic0()
    for k in (3, 17):
        rhs = torch.zeros(k, s.n, dtype=torch.float64, device="cuda")
        bs = []
        for t in range(k):
            kappa, amp = fourier_modes(2, seed=100 + t)
            rhs[t, : s.n_u] = s.load_fourier(kappa, amp)
            bs.append(np.concatenate([ref.load_fourier(kappa, amp), np.zeros(ref.n_p)]))
        X, infos = s.solve(rhs, tol=1e-12, inner_tol=1e-2)
        X = X.cpu().numpy()
        for t in range(k):
            xr, _ = ref.minres(bs[t], tol=1e-12, inner_tol=1e-2)
            assert infos[t]["status"] == 0
            assert rel(X[t], xr) <= 1e-9, (k, t, rel(X[t], xr))
        # mixed precision, batched
        Xm, infos = s.solve(rhs, tol=1e-10, inner_tol=1e-2, precision="mixed")
        Xm = Xm.cpu().numpy()
        for t in range(k):
            xr, _ = ref.minres(bs[t], tol=1e-10, inner_tol=1e-2)
            assert rel(Xm[t], xr) <= 1e-7


def test_host_buffer_solve_matches_device_solve(oracle_mod, gb):
    ref, s = make_pair(oracle_mod, gb, 2, 10, 3)
    s.factor_ic0()
    _, rhs = _rhs(ref, s, "fourier", seed=9)
    x_dev, _ = s.solve(rhs, tol=1e-9)
    x_host, _ = s.solve_host(rhs.cpu().pin_memory(), tol=1e-9)
    assert rel(x_host.numpy().ravel(), x_dev.cpu().numpy()) <= 1e-14


def test_adjoint_and_dnu_match_oracle(oracle_mod, gb):
    """dL/df = lambda_u and dL/dnu = -lambda_u^T A_0 u for L = 1/2||u-u_t||^2."""
    from paper_1309_5048_gb300.inputs import target_velocity
    nu = 0.8
    ref, s = make_pair(oracle_mod, gb, 2, 8, 3, "natural", nu=nu)
    assert ref.factor() < 0
    s.factor_ic0()
    b, rhs = _rhs(ref, s, "fourier", seed=2)
    xr, _ = ref.minres(b, tol=1e-13, inner_tol=1e-3)
    x, _ = s.solve(rhs, tol=1e-13, inner_tol=1e-3)
    u = xr[: ref.n_u]
    ut = target_velocity(ref.n_u, float(np.sqrt(np.mean(u ** 2))))
    g = np.concatenate([u - ut, np.zeros(ref.n_p)])
    lr, _ = ref.minres(g, tol=1e-13, inner_tol=1e-3)
    lam, _ = s.solve_adjoint(torch.tensor(g, device="cuda"), tol=1e-13, inner_tol=1e-3)
    assert rel(lam.cpu().numpy()[: ref.n_u], lr[: ref.n_u]) <= 1e-9
    d = s.dnu(lam, x)[0]
    dr = ref.dnu(lr[: ref.n_u], u)
    assert abs(d - dr) <= 1e-9 * abs(dr)


def test_autograd_function_against_finite_differences(oracle_mod, gb):
    from paper_1309_5048_gb300.autograd import stokes_solve
    from paper_1309_5048_gb300.inputs import fourier_modes, target_velocity
    nu0 = 0.9
    s = gb.Stokes(2, 8, 3)
    s.assemble(nu0)
    s.factor_ic0()
    kappa, amp = fourier_modes(2, seed=4)
    f = s.load_fourier(kappa, amp).clone().requires_grad_(True)
    nu = torch.tensor(nu0, dtype=torch.float64, device="cuda", requires_grad=True)
    opts = dict(tol=1e-13, inner_tol=1e-3)
    x = stokes_solve(f, nu, s, **opts)
    ut = torch.tensor(target_velocity(s.n_u, float(x.detach()[: s.n_u].pow(2).mean().sqrt())), device="cuda")
    loss = 0.5 * (x[: s.n_u] - ut).pow(2).sum()
    loss.backward()

    def L(nu_v, f_v):
        with torch.no_grad():
            xx = stokes_solve(f_v, torch.tensor(nu_v, dtype=torch.float64), s, **opts)
            return float(0.5 * (xx[: s.n_u] - ut).pow(2).sum())

    h = 1e-6
    fd = (L(nu0 + h, f.detach()) - L(nu0 - h, f.detach())) / (2 * h)
    assert abs(fd - float(nu.grad)) <= 1e-6 * abs(fd)
    d = torch.randn(s.n_u, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    d /= d.norm()
    eps = 1e-3
    fd_f = (L(nu0, f.detach() + eps * d) - L(nu0, f.detach() - eps * d)) / (2 * eps)
    assert abs(fd_f - float((f.grad * d).sum())) <= 1e-6 * abs(fd_f)


def test_edge_cases(oracle_mod, gb):
    ref, s = make_pair(oracle_mod, gb, 2, 6, 3)
    s.factor_ic0()
    # zero right-hand side: zero solution, no iteration
    x, info = s.solve(torch.zeros(s.n, dtype=torch.float64, device="cuda"))
    assert info["status"] == 0 and info["outer_its"] == 0 and not x.abs().max().item()
    # a NaN in the right-hand side is reported
    bad = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    bad[3] = float("nan")
    with pytest.raises(gb.GbError) as ei:
        s.solve(bad)
    assert ei.value.status == 6  # GB_ERR_NONFINITE
    # iteration cap reached: NOT_CONVERGED with the iterate written
    _, rhs = _rhs(ref, s, "fourier", seed=1)
    x, info = s.solve(rhs, tol=1e-14, max_outer=3)
    assert info["status"] == 5 and info["outer_its"] == 3 and torch.isfinite(x).all()
    # C_pen too small for coercivity (Sec. 4): A_h indefinite, IC(0) breaks
    # down, at the oracle's row (C_pen = 1 fails at a later row than the first)
    refb = oracle_mod.Problem(2, 6, 3, cpen=1.0)
    row_ref = refb.factor()
    assert row_ref > 0
    sb = gb.Stokes(2, 6, 3)
    sb.assemble(1.0, 1.0)
    with pytest.raises(gb.GbError) as ei:
        sb.factor_ic0()
    assert ei.value.row == row_ref
    # invalid arguments are rejected with a status, not a crash
    with pytest.raises(gb.GbError):
        s.solve(torch.zeros(33, s.n, dtype=torch.float64, device="cuda"))
    with pytest.raises(gb.GbError):
        gb.Stokes(4, 3, 3)


LAYOUT_PAIRS = [("csr", "csr"), ("sell", "sell"), ("csr", "sell"), ("sell", "csr"), ("csr", "staged4"),
                ("sell", "staged12"), ("csr", "staged32"), ("csr", "packed12"), ("sell", "packed32"),
                ("sell2w", "packed32"), ("sell4w", "csr"), ("csr", "split12"), ("sell2w", "split32"),
                ("sell", "sellw"), ("sell2w", "sellw"), ("sell", "sellwl"), ("csr", "sellwl8"),
                ("sell2w", "sellwlr"), ("sell", "sellwl32"), ("csr", "sellwl2"),
                ("sell", "sellwl24"), ("sell", "sellwl48"), ("sell", "sellwlh")]


@pytest.mark.parametrize("spmv,trsv", LAYOUT_PAIRS)
@pytest.mark.parametrize("dim,N,p", [(2, 13, 3), (3, 3, 3), (2, 40, 4)])
def test_single_rhs_layouts_replay_parity(oracle_mod, gb, spmv, trsv, dim, N, p):
    """Every single-RHS layout of the inner SpMV (CSR 8 lanes per row,
    SELL-32 thread per row) and of the IC(0) sweeps (also the staged and
    packed forms, whose levels are split over many blocks at 2D 40^2, and the
    SELL form with several warps per slice, whose rows in 3D and at degree 4
    are longer than its prefetch) reproduces the oracle (<= 1e-10)."""
    ref, s = make_pair(oracle_mod, gb, dim, N, p, "multicolour")
    assert ref.factor() < 0
    s.factor_ic0()
    s.set_kernel_variants("fp64", spmv, trsv)
    s.set_kernel_variants("mixed", spmv, trsv)
    assert s.kernel_variants("fp64") == (spmv, trsv)
    b, rhs = _rhs(ref, s, "fourier", seed=11)
    xr, ir = ref.minres(b, tol=1e-8, inner_tol=1e-2)
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, forced=ir["counts"])
    assert rel(x.cpu().numpy(), xr) <= 1e-10
    x10, _ = s.solve(rhs, tol=1e-10, inner_tol=1e-2, precision="mixed")
    xr10, _ = ref.minres(b, tol=1e-10, inner_tol=1e-2)
    assert rel(x10.cpu().numpy(), xr10) <= 1e-7


@pytest.mark.parametrize("N", [13, 60])
def test_tma_sweep_replay_parity(oracle_mod, gb, N):
    """The TMA-staged SELL sweep (factor slices streamed into shared memory by
    bulk copies, two stages per block): at 2D 60^2 a level has about 340
    slices, so blocks take several slice groups in turn through both stages
    and the copies of later groups overlap the gathers of earlier ones."""
    ref, s = make_pair(oracle_mod, gb, 2, N, 3, "multicolour")
    assert ref.factor() < 0
    s.factor_ic0()
    for prec in ("fp64", "mixed"):
        s.set_kernel_variants(prec, "sell", "tma")
    assert s.kernel_variants("fp64") == ("sell", "tma")
    b, rhs = _rhs(ref, s, "fourier", seed=12)
    xr, ir = ref.minres(b, tol=1e-8, inner_tol=1e-2)
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, forced=ir["counts"])
    assert info["status"] == 0
    assert rel(x.cpu().numpy(), xr) <= 1e-10
    x10, i10 = s.solve(rhs, tol=1e-10, inner_tol=1e-2, precision="mixed")
    xr10, _ = ref.minres(b, tol=1e-10, inner_tol=1e-2)
    assert i10["status"] == 0
    assert rel(x10.cpu().numpy(), xr10) <= 1e-7


@pytest.mark.parametrize("dim,N,p", [(2, 8, 4), (3, 3, 3)])
def test_tma_sweep_is_refused_for_long_rows(gb, dim, N, p):
    """Velocity degree 4 in 2D and every 3D problem have factor rows longer
    than 88 entries, more than a slice group's stage holds: the layout is
    refused with an invalid-argument status."""
    s = gb.Stokes(dim, N, p, ordering="multicolour")
    with pytest.raises(gb.GbError) as ei:
        s.set_kernel_variants("fp64", "sell", "tma")
    assert ei.value.status == 1


def test_layout_autotune_makes_a_choice(oracle_mod, gb):
    _, s = make_pair(oracle_mod, gb, 2, 20, 3, "multicolour")
    s.factor_ic0()
    assert s.kernel_variants("fp64") == ("unset", "unset")
    _, rhs = _rhs(oracle_mod.Problem(2, 20, 3), s, "fourier", seed=3)
    s.solve(rhs, tol=1e-6)
    spmv, trsv = s.kernel_variants("fp64")
    assert spmv in ("csr", "sell", "sell2w", "sell4w") and trsv in ("csr", "sell", "staged4", "staged12", "staged32", "packed12",
                                                 "packed32", "split12", "split32", "sellw", "tma", "sellwl",
                                                 "sellwl8", "sellwlr", "sellwl32",
                                                 "sellwl2", "sellwl24", "sellwl48", "sellwlh")


@pytest.mark.slow
def test_full_size_2d_256_replay_parity(oracle_mod, gb):
    """The benchmark workload (2D, 256 x 256 elements, k' = 2, Fourier
    forcing seed 0) at full size: replayed FP64 solve vs the oracle."""
    ref, s = make_pair(oracle_mod, gb, 2, 256, 3, "multicolour")
    assert ref.factor() < 0
    s.factor_ic0()
    b, rhs = _rhs(ref, s, "fourier", seed=0)
    xr, ir = ref.minres(b, tol=1e-8, inner_tol=1e-2)
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, forced=ir["counts"])
    assert info["outer_its"] == ir["outer"]
    assert rel(x.cpu().numpy(), xr) <= 1e-10


@pytest.mark.slow
def test_full_size_2d_256_mixed_free_mode_against_a_tight_oracle_solve(oracle_mod, gb):
    """The benchmark forcing at 2D 256^2 (k' = 2) in the mixed form (FP32
    inner IC(0)-CG, FP64 MINRES), in free mode -- its own inner counts, no
    replay -- solved to 1e-10 and compared element by element with the discrete
    solution: the relative solution difference and the largest entry
    difference (relative to the largest entry) are within 1e-7.  The FP64
    form in free mode is held to the same comparison.  The reference is the
    oracle's FP64 solve at tol 1e-12 with inner tolerance 1e-4 (with the
    relaxed inner tolerance 1e-2 the preconditioner varies from step to step
    and MINRES can level off near 1e-12; every solve here is capped)."""
    ref, s = make_pair(oracle_mod, gb, 2, 256, 3, "multicolour")
    assert ref.factor() < 0
    s.factor_ic0()
    b, rhs = _rhs(ref, s, "fourier", seed=0)
    xr, ir = ref.minres(b, tol=1e-12, inner_tol=1e-4, max_outer=600)
    assert ir["status"] == 0 and ir["relres_true"] <= 1e-12
    scale = np.abs(xr).max()
    for prec in ("mixed", "fp64"):
        x, info = s.solve(rhs, tol=1e-10, inner_tol=1e-2, precision=prec, max_outer=1500)
        assert info["status"] == 0 and info["relres_true"] <= 1e-10
        xv = x.cpu().numpy()
        assert rel(xv, xr) <= 1e-7, (prec, rel(xv, xr))
        assert np.abs(xv - xr).max() <= 1e-7 * scale, (prec, np.abs(xv - xr).max() / scale)


def test_pressure_rhs_consistency_check(oracle_mod, gb):
    """K is singular with kernel [0; 1] (B^T 1 = 0), so a right-hand side is
    consistent only if 1^T g_p = 0.  A zero-sum pressure part is solved and
    matches the oracle; a column with a nonzero sum is not solved and reports
    an invalid argument, while the other columns of the batch are solved."""
    ref, s = make_pair(oracle_mod, gb, 2, 6, 3)
    assert ref.factor() < 0
    s.factor_ic0()
    b, rhs = _rhs(ref, s, "fourier", seed=4)
    rng = np.random.default_rng(9)
    gp = rng.standard_normal(ref.n_p)
    gp -= gp.mean()
    b[ref.n_u:] = gp
    rhs[s.n_u:] = torch.tensor(gp, device="cuda")
    xr, _ = ref.minres(b, tol=1e-12, inner_tol=1e-4)
    x, info = s.solve(rhs, tol=1e-12, inner_tol=1e-4)
    assert info["status"] == 0
    assert rel(x.cpu().numpy(), xr) <= 1e-8
    bad = rhs.clone()
    bad[s.n_u] += 1.0
    with pytest.raises(gb.GbError) as ei:
        s.solve(bad)
    assert ei.value.status == 1
    pair = torch.stack([rhs, bad])
    out = torch.full_like(pair, 7.0)
    with pytest.raises(gb.GbError) as ei:
        s.solve(pair, out=out, tol=1e-12, inner_tol=1e-4)
    assert ei.value.status == 1
    assert rel(out[0].cpu().numpy(), xr) <= 1e-8
    assert not out[1].any()
