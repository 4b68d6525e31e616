"""GPU parity of the other preconditioner blocks of Sec. 5.1 and of the two
MINRES stopping rules, against the oracle; and the MINRES iteration counts of
the paper's square-domain tables (Sec. 6.2, Tables niter_square_k_2) reproduced
by the GPU solver with the 2-norm stopping rule."""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def pair(oracle_mod, gb, dim, N, p, ordering="natural"):
    ref = oracle_mod.Problem(dim, N, p, ordering=ordering)
    s = gb.Stokes(dim, N, p, ordering=ordering)
    s.assemble(1.0)
    assert ref.factor() < 0 and ref.factor_q() < 0
    s.factor_ic0()
    return ref, s


def manufactured(ref, s):
    b = np.concatenate([ref.load_manufactured(), np.zeros(ref.n_p)])
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_manufactured()
    return b, rhs


@pytest.mark.parametrize("stop", ["residual", "estimate"])
@pytest.mark.parametrize("velocity,pressure", [("jacobi_pcg", "diag"), ("jacobi_pcg", "jacobi_pcg"),
                                               ("ic0_pcg", "jacobi_pcg"), ("ic0_pcg", "diag")])
def test_cg_blocks_replay_parity(oracle_mod, gb, stop, velocity, pressure):
    """FP64, the oracle's inner counts replayed: rel diff <= 1e-10, same
    MINRES step count, for each CG block and both stopping rules."""
    ref, s = pair(oracle_mod, gb, 2, 10, 3, "multicolour")
    b, rhs = manufactured(ref, s)
    xr, ir = ref.minres(b, tol=1e-9, inner_tol=1e-3, velocity=velocity, pressure=pressure, stop=stop)
    assert ir["status"] == 0
    fq = ir["qcounts"] if pressure != "diag" else None
    for use_graph in (True, False):
        x, info = s.solve(rhs, tol=1e-9, inner_tol=1e-3, velocity=velocity, pressure=pressure, stop=stop,
                          forced=ir["counts"], forced_q=fq, use_graph=use_graph)
        assert info["outer_its"] == ir["outer"]
        assert rel(x.cpu().numpy(), xr) <= 1e-10
    if stop == "residual":
        assert info["relres_true"] <= 1.01e-9


def test_diag_block_parity(oracle_mod, gb):
    """Diag(A,Q) (no inner solve, a fixed preconditioner): both solves meet
    the 2-norm tolerance and agree; the step counts agree to within 2 %."""
    ref, s = pair(oracle_mod, gb, 2, 8, 3)
    b, rhs = manufactured(ref, s)
    xr, ir = ref.minres(b, tol=1e-10, velocity="diag", pressure="diag", max_outer=5000)
    x, info = s.solve(rhs, tol=1e-10, velocity="diag", pressure="diag", max_outer=5000)
    assert info["status"] == 0 and info["relres_true"] <= 1.01e-10
    assert abs(info["outer_its"] - ir["outer"]) <= max(1, 0.02 * ir["outer"])
    assert info["inner_its_total"] == 0
    assert rel(x.cpu().numpy(), xr) <= 1e-7


PINNED = [(16, "PCG(A),Diag(Q)"), (32, "PCG(A),Diag(Q)"), (16, "Diag(A,Q)"), (32, "Diag(A,Q)"),
          (16, "Ideal(A,Q)"), (32, "Ideal(A,Q)"), (32, "Ideal(A),Diag(Q)")]
COLS = ["Ideal(A,Q)", "PCG(A,Q)", "Ideal(A),Diag(Q)", "PCG(A),Diag(Q)", "Diag(A,Q)"]


@pytest.mark.parametrize("inv_h,col", PINNED)
def test_gpu_iteration_counts_match_paper_table(oracle_mod, gb, inv_h, col):
    """Table niter_square_k_2 (k' = 2): MINRES steps to ||b - Kx|| / ||b|| <=
    1e-12 on the manufactured problem, within 2 % of the printed count
    (Ideal blocks: IC(0)-PCG at 1e-14 for A, the exact IC(0)-PCG of Q)."""
    want = {(int(r[0]), int(r[1])): r[2:] for r in read_golden("paper_niter_square.txt")}[(2, inv_h)]
    want = int(want[COLS.index(col)])
    s = gb.Stokes(2, inv_h, 3)
    s.assemble(1.0)
    s.factor_ic0()
    rhs = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    rhs[: s.n_u] = s.load_manufactured()
    opts = {"Ideal(A,Q)": dict(velocity="ic0_pcg", pressure="pcg", inner_tol=1e-14),
            "Ideal(A),Diag(Q)": dict(velocity="ic0_pcg", pressure="diag", inner_tol=1e-14),
            "PCG(A),Diag(Q)": dict(velocity="jacobi_pcg", pressure="diag", inner_tol=1e-6),
            "Diag(A,Q)": dict(velocity="diag", pressure="diag")}[col]
    _, info = s.solve(rhs, tol=1e-12, max_outer=20000, max_inner=5000, **opts)
    assert info["status"] == 0
    assert abs(info["outer_its"] - want) <= max(1, 0.02 * want), (info["outer_its"], want)


def test_block_argument_checks(oracle_mod, gb):
    ref, s = pair(oracle_mod, gb, 2, 4, 3)
    _, rhs = manufactured(ref, s)
    with pytest.raises(gb.GbError):
        s.solve(rhs, velocity="diag", forced=[1, 1, 1])  # no velocity CG to replay
    # the diagonal velocity block needs no IC(0) factor
    s2 = gb.Stokes(2, 4, 3)
    s2.assemble(1.0)
    x, info = s2.solve(rhs, velocity="diag", tol=1e-8, max_outer=5000)
    assert info["status"] == 0
    with pytest.raises(gb.GbError):
        s2.solve(rhs)  # the IC(0) block does
