"""GPU parity at the full workload sizes (slow).

The oracle cannot assemble or solve these problems whole in test time, so
the checks use outputs it can compute one by one and properties that hold at
any size:
* operator products on sampled rows: the oracle assembles only the sampled
  rows of A_h and B (element loop restricted to their supports) and forms
  (A x)_i, (B x)_k; B^T is checked through (B^T y).v = y.(B v);
* solutions: the residual b - K x on sampled rows recomputed from the
  oracle's rows, the true residual, the discrete divergence B u and the
  zero-mean pressure w^T p;
* the adjoint gradient dL/dnu against its closed form -(u - u_t)^T u / nu,
  exact because A_h is linear in nu and B is not (the oracle gradient is
  checked at small sizes in test_gpu_parity.py).
Workloads: 2D 256^2 at k'=3, 3D 32^3, 2D 1024^2, 3D 48^3 (k'=2 unless noted),
multicolour ordering as in bench.py.
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

WORKLOADS = {
    "2d256p4": (2, 256, 4),
    "3d32": (3, 32, 3),
    "2d1024": (2, 1024, 3),
    "3d48": (3, 48, 3),
}


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_5048_gb300 as m
    m.load_library()
    return m


_cache = {}


def problem(gb, name):
    if name not in _cache:
        dim, N, p = WORKLOADS[name]
        s = gb.Stokes(dim, N, p, ordering="multicolour")
        s.assemble(1.0)
        s.factor_ic0()
        _cache.clear()  # keep one large problem resident at a time
        _cache[name] = s
    return _cache[name]


def sampled_oracle(oracle_mod, s, nrows_u=48, nrows_p=24, seed=0):
    rng = np.random.default_rng(seed)
    ru = np.sort(rng.choice(s.n_u, nrows_u, replace=False))
    rp = np.sort(rng.choice(s.n_p, nrows_p, replace=False))
    mu = np.zeros(s.n_u, np.int8)
    mp = np.zeros(s.n_p, np.int8)
    mu[ru] = 1
    mp[rp] = 1
    ref = oracle_mod.Problem(s.dim, s.N, s.p, nu=1.0, rows_u=mu, rows_p=mp)
    return ref, ru, rp


def row_products(ref, x_u, ru, rp):
    A = ref.scipy("A")
    B = ref.scipy("B")
    return (A @ x_u)[ru], (B @ x_u)[rp]


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_sampled_operator_rows(oracle_mod, gb, name):
    s = problem(gb, name)
    ref, ru, rp = sampled_oracle(oracle_mod, s)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(s.n)
    xu, xp = x[: s.n_u], x[s.n_u:]
    Ax = s.apply("A", xu).cpu().numpy()
    Bx = s.apply("B", xu).cpu().numpy()
    Ax_ref, Bx_ref = row_products(ref, xu, ru, rp)
    np.testing.assert_allclose(Ax[ru], Ax_ref, rtol=1e-11, atol=1e-12 * np.abs(Ax_ref).max())
    np.testing.assert_allclose(Bx[rp], Bx_ref, rtol=1e-11, atol=1e-12 * np.abs(Bx_ref).max())
    # B^T is the transpose of B: (B^T y).v = y.(B v)
    v = rng.standard_normal(s.n_u)
    lhs = float(s.apply("Bt", xp).cpu().numpy() @ v)
    rhs = float(xp @ s.apply("B", v).cpu().numpy())
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))
    # the full operator is the block matrix
    y = s.apply("K", x).cpu().numpy()
    np.testing.assert_allclose(y[: s.n_u], Ax + s.apply("Bt", xp).cpu().numpy(), rtol=1e-12, atol=1e-12 * np.abs(y).max())
    np.testing.assert_allclose(y[s.n_u:], Bx, rtol=1e-12, atol=1e-12 * np.abs(Bx).max())


def _rhs(s, k, seed0):
    from paper_1309_5048_gb300.inputs import fourier_modes
    r = torch.zeros(k, s.n, dtype=torch.float64, device="cuda")
    for t in range(k):
        kap, amp = fourier_modes(s.dim, seed=seed0 + t)
        r[t, : s.n_u] = s.load_fourier(kap, amp)
    return r


@pytest.mark.parametrize("name,precision", [("2d256p4", "fp64"), ("3d32", "fp64"), ("3d32", "mixed"),
                                            ("2d1024", "mixed")])
def test_full_size_solution_properties(oracle_mod, gb, name, precision):
    s = problem(gb, name)
    rhs = _rhs(s, 1, 0)[0]
    x, info = s.solve(rhs, tol=1e-8, inner_tol=1e-2, precision=precision)
    assert info["status"] == 0
    b = rhs.cpu().numpy()
    xv = x.cpu().numpy()
    r = b - s.apply("K", x).cpu().numpy()
    relres = np.linalg.norm(r) / np.linalg.norm(b)
    assert abs(relres - info["relres_true"]) <= 1e-3 * relres + 1e-15
    # the 2-norm stopping rule (carried by a recurrence on the device)
    assert relres <= 1.01e-8
    # the residual on sampled rows, from the oracle's own rows of A_h and B
    ref, ru, rp = sampled_oracle(oracle_mod, s, seed=2)
    xu, xp = xv[: s.n_u], xv[s.n_u:]
    Ax_ref, Bx_ref = row_products(ref, xu, ru, rp)
    Btp = s.apply("Bt", xp).cpu().numpy()
    r_u = b[ru] - (Ax_ref + Btp[ru])
    np.testing.assert_allclose(r_u, r[ru], atol=1e-10 * np.abs(b).max())
    # incompressibility (Sec. 3.2: divergence-free discrete velocity) and zero-mean pressure
    assert np.linalg.norm(s.apply("B", xu).cpu().numpy()) <= 1e-6 * np.linalg.norm(b)
    w, _ = s.pressure_arrays()
    assert abs(w @ xp) <= 1e-12 * np.abs(xp).max() * np.abs(w).sum()


def test_full_size_3d48_batched_and_adjoint(gb):
    """3D 48^3: a batch of 32 forcings in one graph launch (FP32 inner
    preconditioner, Diag(Q_nu) pressure block), every column meeting the
    contract tolerance 1e-8 on its 2-norm relative residual ||b - K x|| / ||b||
    (the stopping rule, carried by a recurrence on the device and recomputed
    here from the true residual); then the adjoint for L = 1/2 ||u - u_t||^2
    against its closed form.

    A_h is 2 nu times a nu-free matrix and B does not depend on nu, so
    u(nu) = u(1) / nu and dL/dnu = -(u - u_t)^T u / nu exactly (the oracle
    test of the adjoint pins the same identity at small size)."""
    from paper_1309_5048_gb300.inputs import target_velocity
    s = problem(gb, "3d48")
    R = _rhs(s, 32, 0)
    X, infos = s.solve(R, tol=1e-8, inner_tol=1e-2, precision="mixed")
    assert all(i["status"] == 0 and i["relres_true"] <= 1.01e-8 for i in infos)
    for t in (0, 13, 31):
        r = R[t] - s.apply("K", X[t])
        rel = float(r.norm() / R[t].norm())
        assert rel <= 1.01e-8
        assert abs(rel - infos[t]["relres_true"]) <= 1e-3 * rel
    # adjoint of one column, FP64 solves: dL/dnu = -lambda_u^T A_0 u
    x0, i0 = s.solve(R[1], tol=1e-9, inner_tol=1e-2)
    assert i0["status"] == 0
    u = x0[: s.n_u]
    ut = torch.tensor(target_velocity(s.n_u, float(u.pow(2).mean().sqrt())), device="cuda")
    g = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    g[: s.n_u] = u - ut
    lam, il = s.solve_adjoint(g, tol=1e-9, inner_tol=1e-2)
    assert il["status"] == 0
    d = s.dnu(lam, x0)[0]
    closed = -float((u - ut) @ u)
    assert abs(d - closed) <= 1e-6 * abs(closed), (d, closed)


def test_3d_degree_5_without_block_layouts(gb):
    """3D, velocity degree 5, 10^3 elements: interior factor rows have more
    than 2048 off-diagonal entries (2690 couplings per interior row of A_h at
    degree 5), so the staged, packed and split sweep layouts (and the TMA
    layout, limited to 88 entries per row) are not built and are refused; the
    autotuner picks among the others and the solve (IC(0)-PCG(Q) pressure
    block, which keeps the MINRES steps few at this degree) reaches its
    tolerance, its reported true residual matching one recomputed here."""
    from paper_1309_5048_gb300.inputs import fourier_modes
    s = gb.Stokes(3, 10, 5, ordering="multicolour")
    s.assemble(1.0)
    s.factor_ic0()
    for layout in ("staged12", "packed32", "split32", "tma"):
        with pytest.raises(gb.GbError) as ei:
            s.set_kernel_variants("fp64", "sell", layout)
        assert ei.value.status == 1
    kap, amp = fourier_modes(3, seed=3)
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_fourier(kap, amp)
    x, info = s.solve(rhs, tol=1e-6, inner_tol=1e-2, max_outer=1500, pressure="pcg")
    assert s.kernel_variants("fp64")[1] in ("csr", "sell", "sellw", "sellwl", "sellwl8", "sellwlr", "sellwl32",
                                            "sellwl2", "sellwl24", "sellwl48", "sellwlh")
    assert info["status"] == 0 and info["relres_true"] <= 1.01e-6
    r = rhs - s.apply("K", x)
    rel = float(r.norm() / rhs.norm())
    assert abs(rel - info["relres_true"]) <= 1e-3 * rel
