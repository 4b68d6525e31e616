"""The benchmark's algorithmic-byte model without a GPU.

The per-launch and per-iteration byte counts of bench.py are checked against
figures computed independently from the closed-form sizes of two workloads
(2D 256^2 and 3D 32^3, velocity degree 3, k' = 2): nnz(A_h), nnz(B), nnz(L)
and the unknown counts n_u = 2 (N+p-1)(N+p-2), n_p = (N+p-1)^2 in 2D and
n_u = 3 (N+p-1)^2 (N+p-2), n_p = (N+p-1)^3 in 3D.  Each stored nonzero is read
once as value + 32-bit index; each vector operand is read or written once.
"""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

MB = 1e6


def sizes(dim, N, p, nnzA, nnzB, nnzL):
    m = N + p - 1
    n_u = 2 * m * (m - 1) if dim == 2 else 3 * m * m * (m - 1)
    n_p = m ** dim
    return SimpleNamespace(dim=dim, n_u=n_u, n_p=n_p, n=n_u + n_p, nnzA=nnzA, nnzB=nnzB, nnzL=nnzL)


S2 = sizes(2, 256, 3, 9_307_608, 3_944_448, 4_720_110)
S3 = sizes(3, 32, 3, 53_944_848, 15_492_096, 27_029_646)


def inner_iteration(s, precision):
    return (bench.algorithmic_bytes(s, "cg_spmv", precision, 1) + bench.algorithmic_bytes(s, "ic0_apply", precision, 1)
            + bench.cg_vector_bytes(s, precision))


def test_unknown_counts():
    assert (S2.n_u, S2.n_p) == (132_612, 66_564)
    assert (S3.n_u, S3.n_p) == (114_444, 39_304)


@pytest.mark.parametrize("s,fp64_mb,fp32_mb", [(S2, 242.5, 159.5), (S3, 1311.2, 872.3)])
def test_inner_iteration_bytes(s, fp64_mb, fp32_mb):
    assert round(inner_iteration(s, "fp64") / MB, 1) == fp64_mb
    assert round(inner_iteration(s, "mixed") / MB, 1) == fp32_mb


@pytest.mark.parametrize("s,stokes_mb,minres_mb", [(S2, 210.9, 23.9), (S3, 1022.7, 18.2)])
def test_operator_and_minres_vector_bytes(s, stokes_mb, minres_mb):
    assert round(bench.algorithmic_bytes(s, "stokes_apply", "fp64", 1) / MB, 1) == stokes_mb
    assert round(bench.minres_vector_bytes(s) / MB, 1) == minres_mb


def test_solve_bytes_adds_the_measured_counts():
    info = {"outer_its": 137, "inner_its_total": 5152, "precond_apps": 138}
    total = bench.solve_bytes(S2, info, "fp64")
    # every inner iteration once, one extra IC(0) application per
    # preconditioner application, outer + 1 Stokes products, outer MINRES steps
    expect = (5152 * inner_iteration(S2, "fp64") + 138 * bench.algorithmic_bytes(S2, "ic0_apply", "fp64", 1)
              + 138 * bench.algorithmic_bytes(S2, "stokes_apply", "fp64", 1) + 137 * bench.minres_vector_bytes(S2))
    assert total == expect
    # with no inner work the solve moves only the outer loop's bytes
    zero = bench.solve_bytes(S2, {"outer_its": 0, "inner_its_total": 0, "precond_apps": 0}, "fp64")
    assert zero == bench.algorithmic_bytes(S2, "stokes_apply", "fp64", 1)
