"""Sampling schemes and quadratures of the oracle (test infrastructure only): McEwen-Wiaux (MW),
its symmetric variant (MWSS) and Driscoll-Healy (DH).

Sec. 4.2.2 of the paper:
* MW positions: theta_t = (2t+1) pi / (2L-1), t = 0..L-1;  phi_p = 2 pi p / (2L-1), p = 0..2L-2.
* MW weights: the function equal to sin(theta) on [0, pi] and 0 on (pi, 2pi) is replaced by its
  bandlimited Fourier series w, with coefficients w_hat(m') = int_0^pi sin(theta) e^{i m' theta}
  dtheta (the paper's table: +-i pi/2 at m' = +-1, 0 at other odd m', 2/(1-m'^2) at even m'), and
  contributions on (pi, 2pi) are folded back onto (0, pi).
* For the spherical-harmonic transform the signal is upsampled to bandlimit 2L first, and the
  weights at bandlimit L' = 2L are used.

Readings (the printed formula is ambiguous or inconsistent here):
* The sum over m' runs over |m'| <= L'-1 and T = 2L'-1.
* The Fourier synthesis carries e^{-i m' theta}: with the coefficient definition printed
  (e^{+i m' theta} inside the integral) this is the series that sums back to sin(theta) on [0, pi].
  Only the m' = +-1 terms depend on this sign, and they cancel in the fold below.
* The fold factor is +1.  The integrand of the forward transform, F_m(theta) d^l_{m,-s}(theta),
  is the product of two functions that both change sign by (-1)^{m+s} under theta -> 2pi - theta
  after the torus extension, so it is even; the printed zeta_t (-1)^s would be right only for an
  integrand of parity (-1)^s.  With fold +1 the quadrature is exact for every even integrand.
* theta_{L'-1} = pi is the one unreflected ring (zeta = 0 there), as printed.
* The constant is 1/T per ring for the theta integral; the phi integral contributes 2 pi / (2L-1)
  separately (the printed 2 pi / T^2 is the product of both when phi is sampled like theta).
"""
from __future__ import annotations

import numpy as np

from .wigner import PI_LD


def mw_thetas(L: int, dtype=np.longdouble) -> np.ndarray:
    """MW colatitudes theta_t = (2t+1) pi / (2L-1), t < L (the last one is exactly pi)."""
    t = np.arange(L)
    th = (2 * t + 1).astype(np.longdouble) * PI_LD / np.longdouble(2 * L - 1)
    th[-1] = PI_LD
    return th.astype(dtype)


def mw_torus_thetas(L: int, dtype=np.longdouble) -> np.ndarray:
    """The same formula for t = 0..2L-2: the MW grid extended to the theta torus [0, 2 pi)."""
    t = np.arange(2 * L - 1)
    th = (2 * t + 1).astype(np.longdouble) * PI_LD / np.longdouble(2 * L - 1)
    th[L - 1] = PI_LD
    return th.astype(dtype)


def mw_phis(L: int) -> np.ndarray:
    """MW longitudes phi_p = 2 pi p / (2L-1), p < 2L-1 (extended precision)."""
    p = np.arange(2 * L - 1)
    return (2 * p).astype(np.longdouble) * PI_LD / np.longdouble(2 * L - 1)


def w_hat(mp: np.ndarray) -> np.ndarray:
    """w_hat(m') = int_0^pi sin(theta) e^{i m' theta} dtheta (the paper's closed form), complex."""
    mp = np.asarray(mp)
    out = np.zeros(mp.shape, dtype=np.complex128)
    even = (mp % 2) == 0
    out[even] = 2.0 / (1.0 - mp[even].astype(np.float64) ** 2)
    out[mp == 1] = 1j * np.pi / 2
    out[mp == -1] = -1j * np.pi / 2
    return out


def mw_theta_weights(Lp: int, dtype=np.float64) -> np.ndarray:
    """Theta quadrature weights q_t, t < Lp, of the MW sampling theorem at bandlimit Lp.

    sum_t q_t g(theta_t) = int_0^pi g(theta) sin(theta) dtheta for every g whose torus extension
    is even about pi and has frequencies |k| <= Lp-1 (module readings: fold +1, constant 1/T).
    ``dtype`` float64, or np.longdouble for the extended-precision mode (the same sums, with the
    positions, phases and w_hat in extended precision).
    """
    T = 2 * Lp - 1
    k = np.arange(-(Lp - 1), Lp)
    if dtype == np.longdouble:
        th = mw_torus_thetas(Lp)                          # extended precision
        wk = _w_hat_ld(k)
        E = _expi_ld(-np.outer(th, k.astype(np.longdouble)))
    else:
        th = mw_torus_thetas(Lp, dtype=np.float64)       # theta_t on the torus, t < T
        wk = w_hat(k)
        # w(theta_t) = sum_k w_hat(k) e^{-i k theta_t}   (reading: sign of the synthesis)
        E = np.exp(-1j * np.outer(th, k))
    w = E @ wk
    q = np.empty(Lp, dtype=w.dtype)
    for t in range(Lp):
        zeta = 0.0 if t == Lp - 1 else 1.0
        q[t] = (w[t] + zeta * w[2 * Lp - 2 - t]) / T      # reflect: theta_{2L'-2-t} = 2 pi - theta_t
    assert np.max(np.abs(q.imag)) < 1e-12 * np.max(np.abs(q.real))
    return q.real.copy()


# ----------------------------------------------------------------------------- MWSS (Sec. 4.2.2)
# theta_t = 2 pi t / (2L), t = 0..L (both poles are rings); phi_p = 2 pi p / (2L), p < 2L.  The same
# torus construction as MW with T = 2L torus points: the reflection of theta_t is theta_{2L-t} and
# the rings t = 0 and t = L are their own reflections (zeta = 0 there).  Readings as for MW.
def mwss_thetas(L: int, dtype=np.longdouble) -> np.ndarray:
    """MWSS colatitudes theta_t = pi t / L, t = 0..L (exactly 0 and pi at the ends)."""
    th = np.arange(L + 1).astype(np.longdouble) * PI_LD / np.longdouble(L)
    th[0], th[-1] = 0, PI_LD
    return th.astype(dtype)


def mwss_phis(L: int) -> np.ndarray:
    """MWSS longitudes phi_p = 2 pi p / (2L), p < 2L (extended precision)."""
    return np.arange(2 * L).astype(np.longdouble) * PI_LD / np.longdouble(L)


def _w_hat_ld(k: np.ndarray) -> np.ndarray:
    """w_hat of ``w_hat`` in extended precision (clongdouble)."""
    out = np.zeros(len(k), dtype=np.clongdouble)
    even = (k % 2) == 0
    out[even] = np.longdouble(2) / (np.longdouble(1) - k[even].astype(np.longdouble) ** 2)
    out[k == 1] = 1j * (PI_LD / 2)
    out[k == -1] = -1j * (PI_LD / 2)
    return out


def _expi_ld(ang: np.ndarray) -> np.ndarray:
    """exp(i ang) for extended-precision angles, as clongdouble."""
    E = np.empty(ang.shape, dtype=np.clongdouble)
    E.real = np.cos(ang)
    E.imag = np.sin(ang)
    return E


def mwss_theta_weights(Lp: int, dtype=np.float64) -> np.ndarray:
    """Theta quadrature weights q_t, t = 0..Lp, of the MWSS sampling theorem at bandlimit Lp:
    sum_t q_t g(theta_t) = int_0^pi g sin(theta) dtheta for every g whose torus extension is even
    about pi and has frequencies |k| <= Lp-1 (trapezoid on the 2Lp torus points, exact for the
    product of g with the degree-(Lp-1) truncation of the weight function).  ``dtype`` float64, or
    np.longdouble for the extended-precision mode."""
    T = 2 * Lp
    k = np.arange(-(Lp - 1), Lp)
    if dtype == np.longdouble:
        th = np.arange(T).astype(np.longdouble) * PI_LD / np.longdouble(Lp)
        w = _expi_ld(-np.outer(th, k.astype(np.longdouble))) @ _w_hat_ld(k)
    else:
        th = (np.arange(T).astype(np.longdouble) * PI_LD / np.longdouble(Lp)).astype(np.float64)
        w = np.exp(-1j * np.outer(th, k)) @ w_hat(k)
    q = np.empty(Lp + 1, dtype=w.dtype)
    for t in range(Lp + 1):
        zeta = 0.0 if t in (0, Lp) else 1.0
        q[t] = (w[t] + zeta * w[(T - t) % T]) / T
    assert np.max(np.abs(q.imag)) < 1e-12 * np.max(np.abs(q.real))
    return q.real.copy()


# ----------------------------------------------------------------------------- DH (Sec. 4.2.1)
def dh_thetas(L: int, dtype=np.longdouble) -> np.ndarray:
    """DH colatitudes theta_t = (2t+1) pi / (4L), t < 2L."""
    t = np.arange(2 * L)
    return ((2 * t + 1).astype(np.longdouble) * PI_LD / np.longdouble(4 * L)).astype(dtype)


def dh_theta_weights(L: int, dtype=np.float64) -> np.ndarray:
    """The theta part of the DH weights, (2/L) sin(theta_t) sum_{k<L} sin((2k+1) theta_t)/(2k+1),
    t < 2L (the paper's q(theta, phi) is this times the phi step 2 pi/(2L-1)); evaluated in
    extended precision and rounded to ``dtype``."""
    th = dh_thetas(L)
    k = np.arange(L).astype(np.longdouble)
    S = (np.sin(np.outer(th, 2 * k + 1)) / (2 * k + 1)).sum(axis=1)
    return (np.longdouble(2) / L * np.sin(th) * S).astype(dtype)
