"""Seeded synthetic inputs shared by the CUDA library's callers and the oracle.

This module draws random numbers only; it holds none of the method's
arithmetic.  The forcing family is the one the workloads use:

    f_d(x) = sum_{m=1}^{M} a_{m,d} prod_k sin(pi kappa_{m,k} x_k),
    a_{m,d} ~ N(0, 1),  kappa_{m,k} uniform integers in [1, kmax].
"""
from __future__ import annotations

import numpy as np


def fourier_modes(dim: int, seed: int, nmodes: int = 16, kmax: int = 8):
    """(kappa int32 [nmodes, dim], amp float64 [nmodes, dim]) for one forcing."""
    rng = np.random.default_rng(seed)
    kappa = rng.integers(1, kmax + 1, size=(nmodes, dim)).astype(np.int32)
    amp = rng.standard_normal((nmodes, dim))
    return kappa, amp


def target_velocity(n_u: int, rms: float, seed: int = 1000):
    """u_t ~ N(0, rms^2) for the adjoint loss 1/2 ||u - u_t||^2."""
    return np.random.default_rng(seed).standard_normal(n_u) * rms


def unit_direction(n: int, seed: int):
    """A seeded unit vector (finite-difference direction)."""
    v = np.random.default_rng(seed).standard_normal(n)
    return v / np.linalg.norm(v)
