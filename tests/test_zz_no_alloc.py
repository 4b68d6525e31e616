"""gb_dnu_noalloc: dL/dnu without any device allocation.

Some callers of this library cannot call cudaMalloc when they need the
viscosity gradient: programs whose device memory is handed out by their own
pool or framework, which forbids raw allocations beside it, and callers that
have already spent a fixed memory budget.  gb_dnu_noalloc serves them from a
static device array inside the library.  These tests call it through the C
ABI: on a fresh context (set up and assembled only, so no solve workspace
exists) they check that the call leaves the device's free memory and the
context's held bytes unchanged, and they check its value against gb_dnu (the
allocating entry point) on two calls in a row, with the relative tolerance
the other FP64 reduction tests use.  The file is collected last and works
both alone in a fresh process and after the other tests.
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


def _held_bytes(L, s):
    out = np.zeros(10, np.int64)
    assert L.gb_sizes(s._h, out.ctypes.data_as(C.c_void_p)) == 0
    return int(out[8])


def test_dnu_noalloc_allocates_nothing_on_a_fresh_context(gb):
    """First call on a context that never solved: no workspace appears, the
    device's free memory does not shrink, and the value equals gb_dnu's."""
    L = gb.load_library()
    # a call on another context first, so that loading the library's device
    # code (which holds the static array) happens outside the measured window
    warm = gb.Stokes(2, 4, 3)
    warm.assemble(1.0)
    z = torch.zeros(1, warm.n, dtype=torch.float64, device="cuda")
    one = np.zeros(1)
    assert L.gb_dnu_noalloc(warm._h, C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()), 1,
                            one.ctypes.data_as(C.c_void_p)) == 0
    s = gb.Stokes(2, 10, 3, ordering="multicolour")
    s.assemble(1.3)
    k = 2
    g = torch.Generator(device="cpu").manual_seed(7)
    lam = torch.randn(k, s.n, dtype=torch.float64, generator=g).cuda().contiguous()
    x = torch.randn(k, s.n, dtype=torch.float64, generator=g).cuda().contiguous()
    torch.cuda.synchronize()
    held0 = _held_bytes(L, s)
    free0, _ = torch.cuda.mem_get_info()
    outs = []
    for _ in range(2):
        out = np.full(k, np.nan)
        rc = L.gb_dnu_noalloc(s._h, C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()), k,
                              out.ctypes.data_as(C.c_void_p))
        assert rc == 0, L.gb_last_error().decode()
        outs.append(out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert _held_bytes(L, s) == held0
    assert free1 >= free0, "device free memory shrank by %d bytes" % (free0 - free1)
    ref = np.zeros(k)
    assert L.gb_dnu(s._h, C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()), k,
                    ref.ctypes.data_as(C.c_void_p)) == 0
    assert np.all(np.isfinite(ref)) and np.abs(ref).max() > 0
    for out in outs:
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=0)
