"""gb_dnu_noalloc: dL/dnu without any device allocation.

Some callers of this library cannot call cudaMalloc while they need the
viscosity gradient: code that runs during a CUDA graph capture, programs whose
device memory is owned by a pool or framework that forbids new allocations,
or callers that have spent a fixed memory budget.  gb_dnu_noalloc serves them
from a static device array inside the library.  This test calls it through the
C ABI and checks it against gb_dnu (the allocating entry point) on two calls
in a row, with the relative tolerance the other FP64 reduction tests use.  It
sits in its own file, collected last, and works both alone in a fresh process
and after the other tests.
"""
import ctypes as C

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


def test_dnu_noalloc_matches_dnu_on_two_calls(gb):
    from paper_1309_5048_gb300.inputs import fourier_modes
    L = gb.load_library()
    s = gb.Stokes(2, 12, 3, ordering="multicolour")
    s.assemble(0.7)
    s.factor_ic0()
    k = 3
    rhs = torch.zeros(k, s.n, dtype=torch.float64, device="cuda")
    for t in range(k):
        kap, amp = fourier_modes(2, seed=40 + t)
        rhs[t, : s.n_u] = s.load_fourier(kap, amp)
    x, _ = s.solve(rhs, tol=1e-10)
    lam, _ = s.solve_adjoint(x * 0.5 + 1.0, tol=1e-10)
    x = x.contiguous()
    lam = lam.contiguous()
    ref = np.zeros(k)
    assert L.gb_dnu(s._h, C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()), k,
                    ref.ctypes.data_as(C.c_void_p)) == 0
    assert np.all(np.isfinite(ref)) and np.abs(ref).max() > 0
    for _ in range(2):  # the shared static scratch keeps the last call's contents
        out = np.full(k, np.nan)
        rc = L.gb_dnu_noalloc(s._h, C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()), k,
                              out.ctypes.data_as(C.c_void_p))
        assert rc == 0, L.gb_last_error().decode()
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=0)
    # a single right-hand side after a batch of three
    one = np.full(1, np.nan)
    assert L.gb_dnu_noalloc(s._h, C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()), 1,
                            one.ctypes.data_as(C.c_void_p)) == 0
    np.testing.assert_allclose(one, ref[:1], rtol=1e-12, atol=0)


def test_dnu_noalloc_rejects_sizes_beyond_its_scratch(gb):
    L = gb.load_library()
    s = gb.Stokes(2, 4, 3)
    s.assemble(1.0)
    big = torch.zeros(33, s.n, dtype=torch.float64, device="cuda")
    out = np.zeros(33)
    rc = L.gb_dnu_noalloc(s._h, C.c_void_p(big.data_ptr()), C.c_void_p(big.data_ptr()), 33,
                          out.ctypes.data_as(C.c_void_p))
    assert rc == 1  # GB_ERR_INVALID_ARG
    assert b"k must be in [1, 32]" in L.gb_last_error()
