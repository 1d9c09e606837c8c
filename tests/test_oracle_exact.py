"""Pins of the oracle's extended-precision mode (``exact=True``): the sphere transforms on MW, MWSS
and DH sampling and the MW Wigner transform with the d-functions (the recursion over m of
Sec. 3.3), the quadrature weights (Sec. 4.2), the phases and every sum in np.longdouble.

* Round trips land at the rounding level of the extended type (a few hundred units of its
  epsilon), three orders of magnitude below the float64 mode's: any float64 value left in a stage
  would show up at 1e-16.
* The inverse equals a direct synthesis in 40-digit arithmetic (mpmath: the Jacobi form of the
  d-functions of Sec. 3.1 and the phases e^{i m phi}) to that rounding level.
* The float64 and extended modes agree to float64 rounding.
"""
import numpy as np
import pytest

from oracle import transforms as T
from paper_2311_14670_gb300 import synth

EPS_LD = float(np.finfo(np.longdouble).eps)
pytestmark = pytest.mark.skipif(EPS_LD > 1e-17, reason="np.longdouble is not wider than float64 here")


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("L,spin", [(8, 0), (24, 2), (24, -1)])
def test_exact_round_trip_at_extended_rounding_level(L, spin):
    flm = synth.flm_gaussian(L, spin, 1, seed=L + spin)[0]
    f = T.inverse(flm, L, spin, exact=True, keep=True)
    assert f.dtype == np.clongdouble
    back = T.forward(f, L, spin, exact=True, keep=True)
    err = _rel(back, flm)
    assert err < 8 * L * EPS_LD
    # the float64 mode sits at float64 rounding, far above
    back64 = T.forward(T.inverse(flm, L, spin), L, spin)
    assert _rel(back64, flm) > 10 * err


def test_exact_wigner_round_trip_at_extended_rounding_level():
    L, N = 8, 3
    flmn = synth.flmn_gaussian(L, N, 1, seed=4)[0]
    f = T.wigner_inverse(flmn, L, N, exact=True, keep=True)
    back = T.wigner_forward(f, L, N, exact=True, keep=True)
    assert _rel(back, flmn) < 8 * L * EPS_LD


@pytest.mark.parametrize("L,spin", [(4, 0), (4, 1), (5, -2)])
def test_exact_inverse_matches_40_digit_synthesis(L, spin):
    """f(theta_t, phi_p) = sum flm (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta_t) e^{i m phi_p} in mpmath."""
    mpmath = pytest.importorskip("mpmath")
    from oracle.wigner import wigner_d_jacobi
    flm = synth.flm_gaussian(L, spin, 1, seed=11 + L)[0]
    got = T.inverse(flm, L, spin, exact=True, keep=True)
    with mpmath.workdps(40):
        T2 = 2 * L - 1
        th = [mpmath.mpf(2 * t + 1) * mpmath.pi / T2 for t in range(L)]
        th[-1] = mpmath.pi
        ref = np.zeros((L, T2), dtype=object)
        for ell in range(abs(spin), L):
            c = (-1) ** spin * mpmath.sqrt(mpmath.mpf(2 * ell + 1) / (4 * mpmath.pi))
            for m in range(-ell, ell + 1):
                a = mpmath.mpc(flm[ell, m + L - 1].real, flm[ell, m + L - 1].imag)
                for t in range(L):
                    d = wigner_d_jacobi(ell, m, -spin, th[t], dps=40)
                    for p in range(T2):
                        ref[t, p] += a * c * d * mpmath.expjpi(mpmath.mpf(2 * m * p) / T2)
        # the extended values enter mpmath exactly through their decimal expansions
        err = max(abs(mpmath.mpc(mpmath.mpf(np.format_float_scientific(got[t, p].real, precision=40)),
                                 mpmath.mpf(np.format_float_scientific(got[t, p].imag, precision=40))) - ref[t, p])
                  for t in range(L) for p in range(T2))
        scale = max(abs(ref[t, p]) for t in range(L) for p in range(T2))
    assert float(err / scale) < 100 * EPS_LD


@pytest.mark.parametrize("L,spin", [(32, 0), (40, 3)])
def test_exact_and_float64_modes_agree(L, spin):
    flm = synth.flm_gaussian(L, spin, 2, seed=L)
    assert _rel(T.inverse(flm, L, spin, exact=True), T.inverse(flm, L, spin)) < 1e-14
    rng = np.random.default_rng(L)
    f = rng.standard_normal((L, 2 * L - 1)) + 1j * rng.standard_normal((L, 2 * L - 1))
    assert _rel(T.forward(f, L, spin, exact=True), T.forward(f, L, spin)) < 1e-14


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
@pytest.mark.parametrize("L,spin", [(8, 0), (16, 2), (12, -1)])
def test_exact_round_trip_on_mwss_and_dh(sampling, L, spin):
    flm = synth.flm_gaussian(L, spin, 1, seed=3 * L + spin)[0]
    f = T.inverse_s(flm, L, spin, sampling, exact=True, keep=True)
    back = T.forward_s(f, L, spin, sampling, exact=True, keep=True)
    err = _rel(back, flm)
    assert err < 8 * L * EPS_LD
    assert _rel(T.forward_s(T.inverse_s(flm, L, spin, sampling), L, spin, sampling), flm) > 10 * err
    assert _rel(f.astype(np.complex128), T.inverse_s(flm, L, spin, sampling)) < 1e-14
