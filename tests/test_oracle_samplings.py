"""Pins of the oracle's MWSS and DH samplings (Sec. 4.2) against closed forms: exactness of the
quadrature weights, the grids through known spherical harmonics, round trips, agreement of the
forward transforms across samplings, and the dense adjoint against the MW adjoints."""
import os

import numpy as np
import pytest
from numpy.polynomial import legendre

from oracle import transforms as OT
from oracle.sampling import dh_theta_weights, dh_thetas, mwss_theta_weights, mwss_thetas
from paper_2311_14670_gb300 import synth


@pytest.mark.parametrize("L", [1, 2, 3, 8, 17])
def test_dh_weights_integrate_legendre_polynomials_exactly(L):
    """sum_t q_t P_n(cos theta_t) = int_0^pi P_n(cos) sin = 2 delta_n0 for n < 2L (2L rings)."""
    q, x = dh_theta_weights(L), np.cos(dh_thetas(L, np.float64))
    for n in range(2 * L):
        assert abs(q @ legendre.legval(x, [0] * n + [1]) - (2.0 if n == 0 else 0.0)) <= 1e-14
    assert abs(q @ legendre.legval(x, [0] * (2 * L) + [1])) > 1e-6      # and not one degree more


@pytest.mark.parametrize("Lp", [1, 2, 5, 12, 31])
def test_mwss_weights_integrate_even_torus_functions(Lp):
    """cos^n(theta) (n < Lp) is even about pi with torus frequencies <= n: exact integral
    int_0^pi cos^n sin = (1 - (-1)^(n+1)) / (n+1)."""
    q, x = mwss_theta_weights(Lp), np.cos(mwss_thetas(Lp, np.float64))
    for n in range(Lp):
        assert abs(q @ x ** n - (1 - (-1) ** (n + 1)) / (n + 1)) <= 1e-14


def test_grids():
    L = 6
    th = mwss_thetas(L, np.float64)
    assert len(th) == L + 1 and th[0] == 0.0 and th[-1] == np.pi
    th = dh_thetas(L, np.float64)
    assert len(th) == 2 * L and np.allclose(th[::-1], np.pi - th, atol=1e-15)
    assert OT.sampling_shape(L, "mwss") == (L + 1, 2 * L) and OT.sampling_shape(L, "dh") == (2 * L, 2 * L - 1)


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
def test_inverse_reproduces_known_harmonics(sampling):
    """Y_00 = 1/sqrt(4 pi), Y_10 = sqrt(3/(4 pi)) cos theta, Y_11 = -sqrt(3/(8 pi)) sin theta e^{i phi}
    evaluated on the grid (pins theta_t, phi_p and the inverse's normalisation)."""
    L = 4
    R, Tp = OT.sampling_shape(L, sampling)
    th = OT.sampling_thetas(L, sampling).astype(np.float64)[:, None]
    ph = 2 * np.pi * np.arange(Tp)[None, :] / Tp
    for (l, m, ref) in [(0, 0, np.full((R, Tp), 1 / np.sqrt(4 * np.pi))),
                        (1, 0, np.sqrt(3 / (4 * np.pi)) * np.cos(th) * np.ones((1, Tp))),
                        (1, 1, -np.sqrt(3 / (8 * np.pi)) * np.sin(th) * np.exp(1j * ph))]:
        a = np.zeros((L, 2 * L - 1), dtype=np.complex128)
        a[l, m + L - 1] = 1.0
        assert np.abs(OT.inverse_s(a, L, 0, sampling) - ref).max() <= 1e-14


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
@pytest.mark.parametrize("L,spin", [(1, 0), (2, 1), (5, -2), (9, 0), (14, 3)])
def test_round_trip_and_agreement_with_mw(sampling, L, spin):
    """Bandlimited signals: forward(inverse(a)) = a on every sampling, and the forward transform of
    the same function sampled on MW and on this grid agree."""
    a = synth.flm_gaussian(L, spin, 2, seed=L + 3)
    f = OT.inverse_s(a, L, spin, sampling)
    assert f.shape == (2,) + OT.sampling_shape(L, sampling)
    b = OT.forward_s(f, L, spin, sampling)
    assert np.abs(b - a).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(b - OT.forward(OT.inverse(a, L, spin), L, spin)).max() <= 1e-13 * np.abs(a).max()


def test_dense_adjoint_equals_the_mw_adjoints():
    L, spin = 3, 1
    y = synth.signal_gaussian((L, 2 * L - 1), seed=1)
    got = OT.adjoint_dense(lambda x: OT.inverse(x, L, spin), (L, 2 * L - 1), y)
    assert np.abs(np.where(OT.coeff_mask(L, -spin), got, 0) - OT.adjoint_inverse(y, L, spin)).max() <= 1e-13
    c = synth.flm_gaussian(L, spin, 1, seed=2)[0]
    got = OT.adjoint_dense(lambda x: OT.forward(x, L, spin), (L, 2 * L - 1), c)
    assert np.abs(got - OT.adjoint_forward(c, L, spin)).max() <= 1e-13


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
@pytest.mark.parametrize("L,N", [(1, 1), (3, 2), (6, 3), (9, 2)])
def test_wigner_round_trip_and_agreement_with_mw(sampling, L, N):
    """Bandlimited SO(3) signals: forward(inverse(a)) = a on every sampling, and the Wigner
    coefficients of the same function sampled on MW and on this grid agree."""
    a = synth.flmn_gaussian(L, N, 2, seed=L * N + 5)
    f = OT.wigner_inverse_s(a, L, N, sampling)
    R, P = OT.sampling_shape(L, sampling)
    assert f.shape == (2, 2 * N - 1, R, P)
    b = OT.wigner_forward_s(f, L, N, sampling)
    assert np.abs(b - a).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(b - OT.wigner_forward(OT.wigner_inverse(a, L, N), L, N)).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
def test_wigner_n1_is_the_scaled_spin0_transform(sampling):
    """N = 1: the Wigner inverse is the spin-0 inverse with (2l+1)/(8 pi^2) in place of
    sqrt((2l+1)/(4 pi)) (Sec. 2.3: D^l_{m0} is proportional to Y_lm), and it is constant in gamma."""
    L = 7
    a = synth.flmn_gaussian(L, 1, 1, seed=3)[0, 0]                       # [l, m]
    ell = np.arange(L)
    ratio = ((2 * ell + 1) / (8 * np.pi ** 2)) / np.sqrt((2 * ell + 1) / (4 * np.pi))
    f_w = OT.wigner_inverse_s(a[None], L, 1, sampling)[0]
    f_s = OT.inverse_s(a * ratio[:, None], L, 0, sampling)
    assert np.abs(f_w - f_s).max() <= 1e-14 * np.abs(f_s).max()


GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    """The printed values of a golden file: key -> value, the key being every column but the last."""
    out = {}
    with open(os.path.join(GOLDEN_DIR, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                *key, v = line.split()
                out[tuple(key)] = float(v)
    return out


def _valid(L, N):
    return np.stack([OT.coeff_mask(L, n) for n in range(-(N - 1), N)])


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
@pytest.mark.parametrize("L", [8, 16, 32])
def test_round_trip_error_magnitude_matches_paper(sampling, L):
    """The oracle's mean per-coefficient round-trip error on MWSS and DH is at the float64 level the
    paper prints for its on-the-fly transforms (Table sh_error_results; the norm is ambiguous, so
    within a factor 10)."""
    paper = _golden("paper_roundtrip_errors_samplings.txt")[("sht_" + sampling, str(L))]
    rng = np.random.default_rng(L)
    errs = []
    for _ in range(3):
        a = rng.standard_normal((L, 2 * L - 1)) + 1j * rng.standard_normal((L, 2 * L - 1))
        a = np.where(OT.coeff_mask(L, 0), a, 0)
        d = OT.forward_s(OT.inverse_s(a, L, 0, sampling), L, 0, sampling) - a
        errs.append(np.abs(d[OT.coeff_mask(L, 0)]).mean())
    assert np.mean(errs) < 10 * paper


@pytest.mark.parametrize("sampling", ["mw", "mwss"])
@pytest.mark.parametrize("L", [8, 16])
def test_wigner_round_trip_error_magnitude_matches_paper(sampling, L):
    """The same for the Wigner transform with N = 5 on MW and MWSS (Table wig_error_results)."""
    if sampling == "mw":
        paper = _golden("paper_roundtrip_errors_mw.txt")[("W%d" % L,)]
    else:
        paper = _golden("paper_roundtrip_errors_samplings.txt")[("wigner_mwss", str(L))]
    N = 5
    rng = np.random.default_rng(L)
    a = rng.standard_normal((2 * N - 1, L, 2 * L - 1)) + 1j * rng.standard_normal((2 * N - 1, L, 2 * L - 1))
    a = np.where(_valid(L, N), a, 0)
    d = OT.wigner_forward_s(OT.wigner_inverse_s(a, L, N, sampling), L, N, sampling) - a
    assert np.abs(d[_valid(L, N)]).mean() < 10 * paper
