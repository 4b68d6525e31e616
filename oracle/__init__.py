"""Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

A slow, single-threaded, obviously-correct restatement (C++ in this folder)
of the method of Cortes & Coutinho, arXiv:1309.5048: divergence-conforming
B-spline discretisation of Stokes flow (Sec. 3-4) solved by preconditioned
MINRES with the block-diagonal preconditioner diag(IC(0)-PCG(A), Diag(Q_nu))
(Sec. 5, Sec. 6.4).  It shares no code with the CUDA library.  Only the
tests, ``__graft_entry__.smoke`` and ``bench.py``'s CPU-baseline leg load it.

This module compiles the C++ sources with g++ into ``oracle/_build`` and wraps
the ``extern "C"`` entry points with ctypes and numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["spline.cpp", "assembly.cpp", "ordering.cpp", "solvers.cpp", "capi.cpp"]
_lock = threading.Lock()
_lib = None

ORDERINGS = {"natural": 0, "rcm": 1, "multicolour": 2}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, no FMA contraction so the
    results are the same on x86-64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, "oracle.hpp")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.or_last_error.restype = C.c_char_p
            L.or_create.restype = vp
            L.or_create.argtypes = [i32, i32, i32, dbl, dbl, i32, i32, vp, vp]
            L.or_destroy.argtypes = [vp]
            for name in ("or_sizes", "or_csr", "or_wmean", "or_perm", "or_load_fourier",
                         "or_load_manufactured", "or_manufactured_errors", "or_minres", "or_load_cavity",
                         "or_pcg", "or_precond", "or_stokes_apply", "or_filter", "or_perm_q",
                         "or_pcg_q", "or_colours"):
                getattr(L, name).restype = i32
            L.or_sizes.argtypes = [vp, vp]
            L.or_csr.argtypes = [vp, i32, vp, vp, vp]
            L.or_wmean.argtypes = [vp, vp]
            L.or_perm.argtypes = [vp, vp, vp, vp]
            L.or_perm_q.argtypes = [vp, vp, vp, vp]
            L.or_colours.argtypes = [vp, vp]
            L.or_factor.restype = i64
            L.or_factor.argtypes = [vp]
            L.or_factor_q.restype = i64
            L.or_factor_q.argtypes = [vp]
            L.or_load_fourier.argtypes = [vp, i32, vp, vp, vp]
            L.or_load_manufactured.argtypes = [vp, vp]
            L.or_load_cavity.argtypes = [vp, vp]
            L.or_manufactured_errors.argtypes = [vp, vp, vp, vp]
            L.or_manufactured_point.argtypes = [dbl, dbl, dbl, vp]
            L.or_minres.argtypes = [vp, vp, vp, dbl, dbl, i32, i32, vp, i64, i32, vp, i64, i32, i32, vp]
            L.or_counts.restype = i64
            L.or_counts.argtypes = [vp, vp, i64]
            L.or_qcounts.restype = i64
            L.or_qcounts.argtypes = [vp, vp, i64]
            L.or_hist.restype = i64
            L.or_hist.argtypes = [vp, i32, vp, i64]
            L.or_pcg.argtypes = [vp, vp, vp, dbl, i32]
            L.or_pcg_q.argtypes = [vp, vp, vp, dbl, i32]
            L.or_precond.argtypes = [vp, vp, vp, dbl, i32, i32]
            L.or_stokes_apply.argtypes = [vp, vp, vp]
            L.or_filter.argtypes = [vp, vp]
            L.or_dnu.restype = dbl
            L.or_dnu.argtypes = [vp, vp, vp]
            L.or_basis.argtypes = [i32, i32, i32, dbl, vp, vp]
            L.or_gauss.argtypes = [i32, vp, vp]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


PRESSURE_BLOCKS = {"diag": 0, "pcg": 1, "jacobi_pcg": 2}
VELOCITY_BLOCKS = {"ic0_pcg": 0, "diag": 1, "jacobi_pcg": 2}
STOP_RULES = {"residual": 0, "estimate": 1}


def default_cpen(p: int) -> float:
    """C_pen = 5(k'+1) with k' = p-1 (Sec. 6.2)."""
    return 5.0 * p


class Problem:
    """One discrete Stokes problem assembled by the oracle.

    dim 2 or 3, N elements per direction, velocity degree p (pressure degree
    k' = p-1), viscosity nu, Nitsche constant cpen (None -> 5(k'+1)), ordering
    of A before IC(0), qordering of Q before its IC(0) (natural: the factor
    is then exact, see factor_q).  ``rows_u`` / ``rows_p`` (boolean masks)
    restrict the assembly to sampled rows of a large problem (no ordering or
    factor then).
    """

    def __init__(self, dim, N, p, nu=1.0, cpen=None, ordering="natural", rows_u=None, rows_p=None,
                 qordering="natural"):
        L = lib()
        self.dim, self.N, self.p, self.nu = dim, N, p, float(nu)
        self.cpen = default_cpen(p) if cpen is None else float(cpen)
        self.ordering = ordering
        su = None if rows_u is None else np.ascontiguousarray(rows_u, dtype=np.int8)
        sp = None if rows_p is None else np.ascontiguousarray(rows_p, dtype=np.int8)
        if (su is None) != (sp is None):
            n_u, n_p = sizes_closed_form(dim, N, p)[:2]
            if su is None:
                su = np.zeros(n_u, np.int8)
            if sp is None:
                sp = np.zeros(n_p, np.int8)
        h = L.or_create(dim, N, p, self.nu, self.cpen, ORDERINGS[ordering], ORDERINGS[qordering],
                        _p(su), _p(sp))
        if not h:
            raise RuntimeError(L.or_last_error().decode())
        self._h = h
        s = np.zeros(11, np.int64)
        L.or_sizes(h, _p(s))
        (self.n_u, self.n_p, self.nnzA, self.nnzB, self.nnzQ, self.nnzL,
         self.nlevels, self.nrlevels, self.nnzLQ, self.nqlevels, self.nqrlevels) = (int(v) for v in s)
        self.factored = False
        self.qfactored = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    # --- matrices ---------------------------------------------------------
    def csr(self, which):
        """('A'|'B'|'Q'|'L'|'LQ') -> (indptr int64, indices int32, data float64).
        L and LQ are the IC(0) factors of A and Q in their orderings."""
        w = {"A": 0, "B": 1, "Q": 2, "L": 3, "LQ": 4}[which]
        nrows = {"A": self.n_u, "B": self.n_p, "Q": self.n_p, "L": self.n_u, "LQ": self.n_p}[which]
        nnz = {"A": self.nnzA, "B": self.nnzB, "Q": self.nnzQ, "L": self.nnzL, "LQ": self.nnzLQ}[which]
        ptr = np.zeros(nrows + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz, np.float64)
        lib().or_csr(self._h, w, _p(ptr), _p(col), _p(val))
        return ptr, col, val

    def scipy(self, which):
        import scipy.sparse as sp
        ptr, col, val = self.csr(which)
        ncols = {"A": self.n_u, "B": self.n_u, "Q": self.n_p, "L": self.n_u, "LQ": self.n_p}[which]
        return sp.csr_matrix((val, col, ptr), shape=(len(ptr) - 1, ncols))

    def wmean(self):
        w = np.zeros(self.n_p)
        lib().or_wmean(self._h, _p(w))
        return w

    def ordering_arrays(self):
        """(perm[new] = old, level, rlevel) in permuted numbering."""
        perm = np.zeros(self.n_u, np.int32)
        lev = np.zeros(self.n_u, np.int32)
        rlev = np.zeros(self.n_u, np.int32)
        lib().or_perm(self._h, _p(perm), _p(lev), _p(rlev))
        return perm, lev, rlev

    def colours(self):
        """Colour of every velocity DOF (natural numbering) under the
        multicolour rule: (component, index mod (degree + 1) per direction)."""
        out = np.zeros(self.n_u, np.int64)
        lib().or_colours(self._h, _p(out))
        return out

    def ordering_arrays_q(self):
        """Ordering of the pressure space before IC(0) of Q: (perm, level, rlevel)."""
        perm = np.zeros(self.n_p, np.int32)
        lev = np.zeros(self.n_p, np.int32)
        rlev = np.zeros(self.n_p, np.int32)
        lib().or_perm_q(self._h, _p(perm), _p(lev), _p(rlev))
        return perm, lev, rlev

    def factor(self):
        r = lib().or_factor(self._h)
        if r == -99:
            raise RuntimeError(lib().or_last_error().decode())
        self.factored = r < 0
        return int(r)

    def factor_q(self):
        """IC(0) of the reordered pressure mass matrix Q (Sec. 6.4)."""
        r = lib().or_factor_q(self._h)
        if r == -99:
            raise RuntimeError(lib().or_last_error().decode())
        self.qfactored = r < 0
        return int(r)

    # --- loads --------------------------------------------------------------
    def load_fourier(self, kappa, amp):
        kappa = np.ascontiguousarray(kappa, dtype=np.int32)
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        assert kappa.shape == amp.shape and kappa.shape[1] == self.dim
        f = np.zeros(self.n_u)
        if lib().or_load_fourier(self._h, kappa.shape[0], _p(kappa), _p(amp), _p(f)) != 0:
            raise RuntimeError(lib().or_last_error().decode())
        return f

    def load_manufactured(self):
        f = np.zeros(self.n_u)
        if lib().or_load_manufactured(self._h, _p(f)) != 0:
            raise RuntimeError(lib().or_last_error().decode())
        return f

    def load_cavity(self):
        """Lid-driven cavity load (Sec. 6.4): the Nitsche right-hand side of
        eq. nitsche_rhs with lid velocity e_1 on x_dim = 1 (velocity part)."""
        f = np.zeros(self.n_u)
        if lib().or_load_cavity(self._h, _p(f)) != 0:
            raise RuntimeError(lib().or_last_error().decode())
        return f

    def manufactured_errors(self, u, p):
        u = np.ascontiguousarray(u, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        out = np.zeros(3)
        lib().or_manufactured_errors(self._h, _p(u), _p(p), _p(out))
        return out

    # --- solvers ------------------------------------------------------------
    def stokes_apply(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        lib().or_stokes_apply(self._h, _p(x), _p(y))
        return y

    def minres(self, b, tol=1e-8, inner_tol=1e-2, max_outer=5000, max_inner=1000, forced=None,
               pressure="diag", forced_q=None, velocity="ic0_pcg", stop="residual"):
        """Preconditioned MINRES from x0 = 0; pressure filtered to zero mean.
        stop: 'residual' (||b - K x|| / ||b|| <= tol, recomputed every step)
        or 'estimate' (|eta| / gamma_1 <= tol).
        velocity: 'ic0_pcg' (IC(0)-PCG on A_h, needs factor()), 'diag'
        (Diag(A_h)) or 'jacobi_pcg' (diagonally preconditioned CG).
        pressure: 'diag' (Diag(Q_nu)), 'pcg' (IC(0)-PCG on Q_nu, needs
        factor_q()) or 'jacobi_pcg'.  Returns (x, info dict with outer,
        relres_est, relres_true, status, counts (inner its per preconditioner
        application), qcounts (pressure CG its per application), hist)."""
        if (velocity == "ic0_pcg" and not self.factored) or (pressure == "pcg" and not self.qfactored):
            raise RuntimeError("factor() (and factor_q() for pressure='pcg') first")
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        info = np.zeros(4)
        fc = None if forced is None else np.ascontiguousarray(forced, dtype=np.int32)
        fq = None if forced_q is None else np.ascontiguousarray(forced_q, dtype=np.int32)
        rc = lib().or_minres(self._h, _p(b), _p(x), tol, inner_tol, max_outer, max_inner,
                             _p(fc), 0 if fc is None else len(fc), PRESSURE_BLOCKS[pressure],
                             _p(fq), 0 if fq is None else len(fq), VELOCITY_BLOCKS[velocity],
                             STOP_RULES[stop], _p(info))
        if rc != 0:
            raise RuntimeError(lib().or_last_error().decode())
        n = lib().or_counts(self._h, None, 0)
        counts = np.zeros(max(n, 1), np.int32)
        lib().or_counts(self._h, _p(counts), n)
        nq = lib().or_qcounts(self._h, None, 0)
        qcounts = np.zeros(max(nq, 1), np.int32)
        lib().or_qcounts(self._h, _p(qcounts), nq)
        nh = lib().or_hist(self._h, 0, None, 0)
        hist = np.zeros(max(nh, 1))
        lib().or_hist(self._h, 0, _p(hist), nh)
        nh2 = lib().or_hist(self._h, 1, None, 0)
        hist2 = np.zeros(max(nh2, 1))
        lib().or_hist(self._h, 1, _p(hist2), nh2)
        lanczos = []
        for which in (2, 3):
            m = lib().or_hist(self._h, which, None, 0)
            arr = np.zeros(max(m, 1))
            lib().or_hist(self._h, which, _p(arr), m)
            lanczos.append(arr[:m].copy())
        return x, dict(outer=int(info[0]), relres_est=float(info[1]), relres_true=float(info[2]),
                       status=int(info[3]), counts=counts[:n].copy(), qcounts=qcounts[:nq].copy(),
                       hist=hist[:nh].copy(), hist_res=hist2[:nh2].copy(), delta=lanczos[0],
                       gamma=lanczos[1])

    def pcg(self, b, inner_tol, max_inner=1000):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        its = lib().or_pcg(self._h, _p(b), _p(x), inner_tol, max_inner)
        return x, int(its)

    def pcg_q(self, b, inner_tol, max_inner=1000):
        """IC(0)-preconditioned CG on Q from x0 = 0 (needs factor_q())."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        its = lib().or_pcg_q(self._h, _p(b), _p(x), inner_tol, max_inner)
        if its < 0:
            raise RuntimeError(lib().or_last_error().decode())
        return x, int(its)

    def precond(self, r, inner_tol, max_inner=1000, pressure="diag"):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        its = lib().or_precond(self._h, _p(r), _p(z), inner_tol, max_inner, PRESSURE_BLOCKS[pressure])
        return z, int(its)

    def filter(self, pres):
        p = np.array(pres, dtype=np.float64)
        lib().or_filter(self._h, _p(p))
        return p

    def dnu(self, lam_u, u):
        lam_u = np.ascontiguousarray(lam_u, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        return float(lib().or_dnu(self._h, _p(lam_u), _p(u)))


def basis(N, q, e, x):
    """Values and derivatives of the q+1 degree-q functions nonzero on element e."""
    v = np.zeros(q + 1)
    d = np.zeros(q + 1)
    lib().or_basis(N, q, e, float(x), _p(v), _p(d))
    return v, d


def gauss(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss(n, _p(x), _p(w))
    return x, w


def manufactured_point(nu, x, y):
    out = np.zeros(5)
    lib().or_manufactured_point(float(nu), float(x), float(y), _p(out))
    return out


def sizes_closed_form(dim, N, p):
    """n_u, n_p from the space definitions (Sec. 3.2)."""
    if dim == 2:
        return 2 * (N + p - 1) * (N + p - 2), (N + p - 1) ** 2
    return 3 * (N + p - 1) ** 2 * (N + p - 2), (N + p - 1) ** 3
