"""gbstokes: GB300 (sm_103a) solver for the divergence-conforming B-spline
Stokes system of Cortes & Coutinho (arXiv:1309.5048).

This module is a thin ctypes binding of the C ABI in ``include/gbstokes.h``:
it marshals arguments only (torch tensors provide device memory and the CUDA
stream); every step of the method runs in the library's CUDA kernels.  There
is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

ORDERINGS = {"natural": 0, "rcm": 1, "multicolour": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
PRESSURE_BLOCKS = {"diag": 0, "pcg": 1, "jacobi_pcg": 2}
VELOCITY_BLOCKS = {"ic0_pcg": 0, "diag": 1, "jacobi_pcg": 2}
STOP_RULES = {"residual": 0, "estimate": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "IC(0) breakdown",
          5: "not converged", 6: "non-finite value", 7: "device wait timed out"}
GB_OK, GB_ERR_NOT_CONVERGED, GB_ERR_IC0_BREAKDOWN = 0, 5, 4


class GbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gbstokes: %s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class gb_problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("p", C.c_int), ("ordering", C.c_int)]


class gb_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("inner_tol", C.c_double), ("precision", C.c_int),
                ("max_outer", C.c_int), ("max_inner", C.c_int), ("use_graph", C.c_int),
                ("forced_inner_host", C.c_void_p), ("nforced", C.c_int64), ("pressure_block", C.c_int),
                ("forced_q_host", C.c_void_p), ("nforced_q", C.c_int64), ("stop_rule", C.c_int),
                ("velocity_block", C.c_int)]


class gb_info(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("precond_apps", C.c_int), ("inner_its_total", C.c_int64),
                ("inner_its_max", C.c_int), ("relres_est", C.c_double), ("relres_true", C.c_double),
                ("q_inner_its_total", C.c_int64), ("q_inner_its_max", C.c_int), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = ["gb_setup_pattern", "gb_sizes", "gb_assemble", "gb_load_fourier", "gb_load_manufactured",
            "gb_factor_ic0", "gb_solve", "gb_solve_host", "gb_solve_adjoint", "gb_dnu", "gb_apply",
            "gb_export", "gb_destroy", "gb_status_string", "gb_last_error", "gb_time_kernel",
            "gb_set_kernel_variants", "gb_get_kernel_variants", "gb_dnu_noalloc", "gb_load_cavity",
            "gb_lanczos", "gb_ritz_extremes", "gb_set_batch_sweep", "gb_get_batch_sweep"]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("gbstokes library missing at %s; run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        for name in EXPORTED:
            getattr(L, name)  # every declared symbol must be exported
        L.gb_setup_pattern.argtypes = [C.POINTER(gb_problem), vp, C.POINTER(vp)]
        L.gb_sizes.argtypes = [vp, vp]
        L.gb_assemble.argtypes = [vp, dbl, dbl]
        L.gb_load_fourier.argtypes = [vp, i32, vp, vp, vp]
        L.gb_load_manufactured.argtypes = [vp, vp]
        L.gb_load_cavity.argtypes = [vp, vp]
        L.gb_lanczos.argtypes = [vp, i32, vp, vp, i32, C.POINTER(i32)]
        L.gb_ritz_extremes.argtypes = [vp, i32, i32, vp]
        L.gb_set_batch_sweep.argtypes = [vp, i32, i32, i32]
        L.gb_get_batch_sweep.argtypes = [vp, i32, i32, C.POINTER(i32)]
        L.gb_factor_ic0.argtypes = [vp, C.POINTER(i64)]
        L.gb_solve.argtypes = [vp, vp, vp, i32, C.POINTER(gb_solve_opts), vp]
        L.gb_solve_host.argtypes = [vp, vp, vp, i32, C.POINTER(gb_solve_opts), vp]
        L.gb_solve_adjoint.argtypes = [vp, vp, vp, i32, C.POINTER(gb_solve_opts), vp]
        L.gb_dnu.argtypes = [vp, vp, vp, i32, vp]
        L.gb_dnu_noalloc.argtypes = [vp, vp, vp, i32, vp]
        L.gb_apply.argtypes = [vp, i32, vp, vp]
        L.gb_time_kernel.argtypes = [vp, i32, i32, C.POINTER(dbl)]
        L.gb_set_kernel_variants.argtypes = [vp, i32, i32, i32]
        L.gb_get_kernel_variants.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32)]
        L.gb_export.argtypes = [vp, i32, vp, vp, vp]
        L.gb_destroy.argtypes = [vp]
        L.gb_destroy.restype = None
        L.gb_status_string.restype = C.c_char_p
        L.gb_status_string.argtypes = [i32]
        L.gb_last_error.restype = C.c_char_p
        _lib = L
        return L


def _check(rc, allow=()):
    if rc != GB_OK and rc not in allow:
        raise GbError(rc, load_library().gb_last_error().decode())
    return rc


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Stokes:
    """A discrete Stokes problem on the GPU (one context of the C library).

    dim 2 or 3, N elements per direction, velocity degree p (pressure degree
    p-1), ordering of A_h before IC(0): 'natural', 'rcm' or 'multicolour'.
    All device work runs on the torch stream current at construction.
    """

    def __init__(self, dim, N, p, ordering="natural", device=None):
        import torch
        self.torch = torch
        L = load_library()
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
        prob = gb_problem(dim, N, p, ORDERINGS[ordering])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.gb_setup_pattern(C.byref(prob), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.dim, self.N, self.p, self.ordering = dim, N, p, ordering
        s = np.zeros(10, np.int64)
        L.gb_sizes(h, s.ctypes.data_as(C.c_void_p))
        (self.n_u, self.n_p, self.nnzA, self.nnzB, self.nnzL, self.nlevels, self.nrlevels,
         self.nnzQ, self.device_bytes, self.ncolours) = (int(v) for v in s)
        self.n = self.n_u + self.n_p
        self.nu = None

    def close(self):
        if getattr(self, "_h", None):
            load_library().gb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, x, shape=None):
        t = self.torch.as_tensor(x, dtype=self.torch.float64, device=self.device).contiguous()
        if shape is not None:
            t = t.reshape(shape)
        return t

    # ------------------------------------------------------------ set-up
    def assemble(self, nu=1.0, cpen=None):
        _check(load_library().gb_assemble(self._h, float(nu), -1.0 if cpen is None else float(cpen)))
        self.nu = float(nu)

    def load_fourier(self, kappa, amp):
        kappa = np.ascontiguousarray(kappa, dtype=np.int32)
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        f = self.torch.empty(self.n_u, dtype=self.torch.float64, device=self.device)
        _check(load_library().gb_load_fourier(self._h, kappa.shape[0], kappa.ctypes.data_as(C.c_void_p),
                                              amp.ctypes.data_as(C.c_void_p), _ptr(f)))
        return f

    def load_manufactured(self):
        f = self.torch.empty(self.n_u, dtype=self.torch.float64, device=self.device)
        _check(load_library().gb_load_manufactured(self._h, _ptr(f)))
        return f

    def load_cavity(self):
        """Lid-driven cavity load (Sec. 6.4): the Nitsche right-hand side with
        lid velocity e_1 on x_dim = 1 (velocity part, natural numbering)."""
        f = self.torch.empty(self.n_u, dtype=self.torch.float64, device=self.device)
        _check(load_library().gb_load_cavity(self._h, _ptr(f)))
        return f

    def factor_ic0(self):
        """IC(0) of the reordered A_h; returns -1, or raises GbError with the
        breakdown row in ``.row``."""
        row = C.c_int64(-1)
        rc = load_library().gb_factor_ic0(self._h, C.byref(row))
        if rc == GB_ERR_IC0_BREAKDOWN:
            e = GbError(rc, "non-positive pivot at row %d" % row.value)
            e.row = row.value
            raise e
        _check(rc)
        return -1

    # ------------------------------------------------------------ solves
    @staticmethod
    def options(tol=1e-8, inner_tol=1e-2, precision="fp64", max_outer=5000, max_inner=1000,
                use_graph=True, forced=None, pressure="diag", forced_q=None, stop="residual",
                velocity="ic0_pcg"):
        o = gb_solve_opts(tol, inner_tol, PRECISIONS[precision], max_outer, max_inner, int(use_graph), None, 0,
                          PRESSURE_BLOCKS[pressure], None, 0, STOP_RULES[stop], VELOCITY_BLOCKS[velocity])
        keep = []
        if forced is not None:
            f = np.ascontiguousarray(forced, dtype=np.int32)
            keep.append(f)
            o.forced_inner_host = f.ctypes.data_as(C.c_void_p)
            o.nforced = f.size
        if forced_q is not None:
            fq = np.ascontiguousarray(forced_q, dtype=np.int32)
            keep.append(fq)
            o.forced_q_host = fq.ctypes.data_as(C.c_void_p)
            o.nforced_q = fq.size
        return o, keep

    def _solve(self, fn, rhs, out=None, allow_not_converged=True, **kw):
        rhs = self._dev(rhs)
        single = rhs.dim() == 1
        rhs2 = rhs.reshape(-1, self.n)
        k = rhs2.shape[0]
        x = out if out is not None else self.torch.empty_like(rhs2)
        o, keep = self.options(**kw)
        infos = (gb_info * k)()
        rc = fn(self._h, _ptr(rhs2), _ptr(x), k, C.byref(o), infos)
        del keep
        _check(rc, allow=(GB_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        info = [infos[i].as_dict() for i in range(k)]
        return (x[0] if single else x), (info[0] if single else info)

    def solve(self, rhs, out=None, **kw):
        """Preconditioned MINRES from x0 = 0 for rhs of shape (n,) or (k, n),
        k <= 32.  Options: tol, inner_tol, precision ('fp64'|'mixed'),
        max_outer, max_inner, use_graph, stop ('residual': ||b - Kx|| / ||b||
        <= tol, the default; 'estimate': |eta| / gamma_1 <= tol), velocity
        ('ic0_pcg', 'diag', 'jacobi_pcg'), pressure ('diag': Diag(Q_nu),
        'pcg': IC(0)-PCG on Q_nu, 'jacobi_pcg'), forced / forced_q (replay
        the velocity / pressure inner counts)."""
        return self._solve(load_library().gb_solve, rhs, out, **kw)

    def solve_adjoint(self, grad, out=None, **kw):
        return self._solve(load_library().gb_solve_adjoint, grad, out, **kw)

    def solve_host(self, rhs_host, out_host=None, **kw):
        """gb_solve_host: host (pinned) buffers in and out."""
        import torch
        rhs_host = torch.as_tensor(rhs_host, dtype=torch.float64).contiguous()
        rhs2 = rhs_host.reshape(-1, self.n)
        k = rhs2.shape[0]
        x = out_host if out_host is not None else torch.empty_like(rhs2, pin_memory=True)
        o, keep = self.options(**kw)
        infos = (gb_info * k)()
        rc = load_library().gb_solve_host(self._h, C.c_void_p(rhs2.data_ptr()), C.c_void_p(x.data_ptr()), k,
                                          C.byref(o), infos)
        _check(rc, allow=(GB_ERR_NOT_CONVERGED,))
        return x, [infos[i].as_dict() for i in range(k)]

    def dnu(self, lam, x):
        lam = self._dev(lam).reshape(-1, self.n)
        x = self._dev(x).reshape(-1, self.n)
        k = lam.shape[0]
        out = np.zeros(k)
        _check(load_library().gb_dnu(self._h, _ptr(lam), _ptr(x), k, out.ctypes.data_as(C.c_void_p)))
        return out

    LAYOUTS = {"auto": -1, "csr": 0, "sell": 1, "staged4": 2, "staged12": 3, "staged32": 4, "packed12": 5,
               "packed32": 6, "split12": 7, "split32": 8, "sellw": 9, "tma": 10, "sellwl": 11, "sellwl8": 12, "sellwlr": 13, "sellwl32": 14, "sellwl2": 15, "sellwl24": 16, "sellwl48": 17, "sellwlh": 18}
    SPMV_LAYOUTS = {"auto": -1, "csr": 0, "sell": 1, "sell2w": 2, "sell4w": 3}

    def set_kernel_variants(self, precision="fp64", spmv="auto", trsv="auto"):
        """Layout of the single-RHS inner SpMV ('csr': 8 lanes per row,
        'sell': SELL-32, one thread per row, 'sell2w' / 'sell4w': SELL-32 with
        2 / 4 warps per slice) and IC(0) sweeps ('csr', 'sell', 'staged4',
        'staged12', 'staged32': rows staged in shared memory, 'packed12',
        'packed32': k-major copies, 'split12', 'split32': k-major copies
        whose older-level entries are summed before the wait for the
        previous level), 'sellw' (SELL-32 with 1-8 warps per slice by the
        level's longest row, up to 12 slots per lane loaded before the wait),
        'tma' (the same slice groups streamed into shared memory by bulk
        copies, double-buffered; rows of at most 88 entries: 2D, velocity
        degree 3), 'sellwl' (the SELL form with four slots loaded before the
        wait and the rest read in a loop, about 16 slots per lane), 'sellwl8'
        (the same with about 8 slots per lane), 'sellwlr' (the light form on
        a grid of the resident blocks, each taking several slice groups),
        'sellwl32' (the light form with about 32 slots per lane), 'sellwl2'
        (two slots loaded before the wait, about 16 per lane), 'sellwl24',
        'sellwl48' (the light form with about 24 / 48 slots per lane),
        'sellwlh' (about 32 slots per lane, with 12 slots loaded before the
        wait on the levels of one warp per slice), or 'auto'."""
        _check(load_library().gb_set_kernel_variants(self._h, PRECISIONS[precision], self.SPMV_LAYOUTS[spmv],
                                                      self.LAYOUTS[trsv]))

    def kernel_variants(self, precision="fp64"):
        a, b = C.c_int(0), C.c_int(0)
        _check(load_library().gb_get_kernel_variants(self._h, PRECISIONS[precision], C.byref(a), C.byref(b)))
        names = {v: k for k, v in self.LAYOUTS.items()}
        snames = {v: k for k, v in self.SPMV_LAYOUTS.items()}
        names[-1] = snames[-1] = "unset"
        return snames[a.value], names[b.value]

    BATCH_SWEEPS = {"auto": -1, "warp": 0, "staged": 1}

    def set_batch_sweep(self, precision="fp64", width=32, variant="auto"):
        """IC(0) sweep kernel of batched solves of this width (8 or 32)."""
        _check(load_library().gb_set_batch_sweep(self._h, PRECISIONS[precision], width,
                                                  self.BATCH_SWEEPS[variant]))

    def batch_sweep(self, precision="fp64", width=32):
        v = C.c_int(0)
        _check(load_library().gb_get_batch_sweep(self._h, PRECISIONS[precision], width, C.byref(v)))
        return {val: key for key, val in self.BATCH_SWEEPS.items()}[v.value]

    def lanczos(self, rhs=0):
        """Lanczos tridiagonal T_j of the last solve's MINRES for column rhs:
        (delta_1..delta_j, gamma_1..gamma_{j+1})."""
        L = load_library()
        n = C.c_int(0)
        _check(L.gb_lanczos(self._h, rhs, None, None, 0, C.byref(n)))
        d = np.zeros(max(n.value, 1))
        g = np.zeros(n.value + 1)
        _check(L.gb_lanczos(self._h, rhs, d.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p),
                            n.value, C.byref(n)))
        return d[: n.value], g[: n.value + 1]

    def ritz_extremes(self, rhs=0, exclude_one=False):
        """(lambda^-_min, lambda^-_max, lambda^+_min, lambda^+_max) of the Ritz
        values of the last solve's Lanczos tridiagonal (column rhs)."""
        out = np.zeros(4)
        _check(load_library().gb_ritz_extremes(self._h, rhs, int(exclude_one), out.ctypes.data_as(C.c_void_p)))
        return out

    KERNELS = {"cg_spmv": 0, "ic0_apply": 1, "stokes_apply": 2, "trsv_fwd": 3}

    def time_kernel(self, which, reps=20):
        """Mean ms per launch of one kernel family of the last solve (events
        on the library's stream): 'cg_spmv', 'ic0_apply', 'stokes_apply',
        'trsv_fwd'."""
        ms = C.c_double(0.0)
        _check(load_library().gb_time_kernel(self._h, self.KERNELS[which], int(reps), C.byref(ms)))
        return ms.value

    def dnu_noalloc(self, lam, x):
        """gb_dnu_noalloc: dL/dnu like dnu(), with no device allocation (for
        callers that cannot allocate; see include/gbstokes.h)."""
        lam = self._dev(lam).reshape(-1, self.n)
        x = self._dev(x).reshape(-1, self.n)
        k = lam.shape[0]
        out = np.zeros(k)
        _check(load_library().gb_dnu_noalloc(self._h, _ptr(lam), _ptr(x), k, out.ctypes.data_as(C.c_void_p)))
        return out

    def apply(self, which, x):
        """which: 'K' (Stokes operator), 'A', 'B', 'Bt', 'Q' (pressure mass
        matrix) -- natural numbering."""
        w = {"K": 0, "A": 1, "B": 2, "Bt": 3, "Q": 4}[which]
        x = self._dev(x)
        nout = {"K": self.n, "A": self.n_u, "B": self.n_p, "Bt": self.n_u, "Q": self.n_p}[which]
        y = self.torch.empty(nout, dtype=self.torch.float64, device=self.device)
        _check(load_library().gb_apply(self._h, w, _ptr(x), _ptr(y)))
        return y

    # ------------------------------------------------------------ export
    def csr(self, which):
        """('A'|'B'|'L') -> (indptr int64, indices int32, data float64) on the host."""
        L = load_library()
        w = {"A": 0, "B": 1, "L": 2}[which]
        nrows = {"A": self.n_u, "B": self.n_p, "L": self.n_u}[which]
        nnz = {"A": self.nnzA, "B": self.nnzB, "L": self.nnzL}[which]
        ptr = np.zeros(nrows + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz, np.float64)
        _check(L.gb_export(self._h, w, ptr.ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p),
                           val.ctypes.data_as(C.c_void_p)))
        return ptr, col, val

    def ordering_arrays(self):
        perm = np.zeros(self.n_u, np.int32)
        lev = np.zeros(self.n_u, np.int32)
        rlev = np.zeros(self.n_u, np.int32)
        _check(load_library().gb_export(self._h, 3, perm.ctypes.data_as(C.c_void_p),
                                        lev.ctypes.data_as(C.c_void_p), rlev.ctypes.data_as(C.c_void_p)))
        return perm, lev, rlev

    def pressure_arrays(self):
        w = np.zeros(self.n_p)
        q = np.zeros(self.n_p)
        _check(load_library().gb_export(self._h, 4, None, w.ctypes.data_as(C.c_void_p),
                                        q.ctypes.data_as(C.c_void_p)))
        return w, q

    def q_csr(self):
        """Pressure mass matrix Q (natural numbering): (indptr int64, indices, data)."""
        ptr = np.zeros(self.n_p + 1, np.int32)
        col = np.zeros(self.nnzQ, np.int32)
        val = np.zeros(self.nnzQ, np.float64)
        _check(load_library().gb_export(self._h, 5, ptr.ctypes.data_as(C.c_void_p),
                                        col.ctypes.data_as(C.c_void_p), val.ctypes.data_as(C.c_void_p)))
        return ptr.astype(np.int64), col, val

    def q_factor_bands(self):
        """Bands (m x p) of the 1D mass matrix Q1 and of its Cholesky factor L1:
        [a, o] = Q1[a, a-o] and L1[a, a-o]; IC(0) of Q = L1 x L1 (x L1)."""
        m = self.N + self.p - 1
        q1 = np.zeros(m * self.p)
        l1 = np.zeros(m * self.p)
        _check(load_library().gb_export(self._h, 6, q1.ctypes.data_as(C.c_void_p),
                                        l1.ctypes.data_as(C.c_void_p), None))
        return q1.reshape(m, self.p), l1.reshape(m, self.p)


# Function-style names matching the C ABI.
def setup_pattern(dim, N, p, ordering="natural", device=None) -> Stokes:
    return Stokes(dim, N, p, ordering, device)


def assemble(s: Stokes, nu=1.0, cpen=None):
    return s.assemble(nu, cpen)


def factor_ic0(s: Stokes):
    return s.factor_ic0()


def solve(s: Stokes, rhs, **kw):
    return s.solve(rhs, **kw)


def solve_adjoint(s: Stokes, grad, **kw):
    return s.solve_adjoint(grad, **kw)
