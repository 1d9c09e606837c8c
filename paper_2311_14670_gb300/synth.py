"""Seeded synthetic inputs with the shapes and distributions of the benchmark workloads.

Plain numpy random draws (PCG64); nothing of the transforms' arithmetic lives here, so both the
GPU tests and the oracle-based checks can use the same arrays.  Index conventions follow
``include/s2gb.h``: coefficients [..., l, m+L-1], valid where max(|m|, |n|) <= l < L.
"""
from __future__ import annotations

import numpy as np


def valid_mask(L: int, n: int) -> np.ndarray:
    """True at the (l, m) entries that carry coefficients for d-index n (= -spin)."""
    ell = np.arange(L)[:, None]
    m = np.arange(-(L - 1), L)[None, :]
    return (np.abs(m) <= ell) & (abs(n) <= ell)


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Real and imaginary parts i.i.d. N(0, 1)."""
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def flm_gaussian(L: int, spin: int, batch: int, seed: int, ell_power: float = 0.0) -> np.ndarray:
    """Sphere coefficients (batch, L, 2L-1): complex Gaussian times (l+1)^-ell_power, zero outside
    the valid domain; f_00 real when spin = 0 (as in the L = 64 workload)."""
    rng = np.random.default_rng(seed)
    a = complex_gaussian(rng, (batch, L, 2 * L - 1))
    a *= (np.arange(L) + 1.0)[:, None] ** (-ell_power)
    a = np.where(valid_mask(L, -spin), a, 0)
    if spin == 0:
        a[:, 0, L - 1] = a[:, 0, L - 1].real
    return a


def flm_real_gaussian(L: int, batch: int, seed: int, ell_power: float = 0.0) -> np.ndarray:
    """Coefficients of a real signal, orders m >= 0 (batch, L, L): complex Gaussian times
    (l+1)^-ell_power where m <= l, real at m = 0."""
    rng = np.random.default_rng(seed)
    a = complex_gaussian(rng, (batch, L, L))
    a *= (np.arange(L) + 1.0)[:, None] ** (-ell_power)
    a = np.where(np.arange(L)[None, :] <= np.arange(L)[:, None], a, 0)
    a[..., 0] = a[..., 0].real
    return a


def signal_real_gaussian(shape, seed: int) -> np.ndarray:
    """Arbitrary real samples, standard Gaussian."""
    return np.random.default_rng(seed).standard_normal(shape)


def flmn_gaussian(L: int, N: int, batch: int, seed: int) -> np.ndarray:
    """Wigner coefficients (batch, 2N-1, L, 2L-1), complex Gaussian where l >= max(|m|, |n|)."""
    rng = np.random.default_rng(seed)
    a = complex_gaussian(rng, (batch, 2 * N - 1, L, 2 * L - 1))
    mask = np.stack([valid_mask(L, n) for n in range(-(N - 1), N)])
    return np.where(mask[None], a, 0)


def signal_gaussian(shape, seed: int) -> np.ndarray:
    """Arbitrary (not bandlimited) samples, complex Gaussian."""
    return complex_gaussian(np.random.default_rng(seed), shape)
