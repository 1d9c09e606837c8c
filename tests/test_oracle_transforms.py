"""Pins for the oracle's spin-s SHT, Wigner transform and adjoints (CPU only).

Independent checks: textbook closed-form Y_lm (l <= 4), the paper's spin operators (Sec. 2.2)
applied by numerical differentiation, the addition theorem, exact round trips, a second exact
quadrature (Gauss-Legendre) for the forward transform, an O(L^4) brute-force inverse from the
Jacobi representation, dense conjugate transposes for the adjoints, the N = 1 reduction of the
Wigner transform, and the paper's printed round-trip error magnitudes.
"""
import os

import numpy as np
import pytest

from oracle import transforms as T
from oracle.sampling import mw_phis, mw_thetas
from oracle.wigner import wigner_d_jacobi, wigner_d_table

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_roundtrip_errors_mw.txt")


def rand_flm(rng, L, n, shape=()):
    a = rng.standard_normal(shape + (L, 2 * L - 1)) + 1j * rng.standard_normal(shape + (L, 2 * L - 1))
    return np.where(T.coeff_mask(L, n), a, 0)


def grid(L):
    th = mw_thetas(L, dtype=np.float64)[:, None]
    ph = mw_phis(L).astype(np.float64)[None, :]
    return th, ph


def closed_Y(ell, m, th, ph):
    """Textbook Y_lm with the Condon-Shortley phase, l <= 4, m >= 0."""
    c, s = np.cos(th), np.sin(th)
    pi = np.pi
    table = {
        (0, 0): 0.5 / np.sqrt(pi) + 0 * th,
        (1, 0): np.sqrt(3 / (4 * pi)) * c,
        (1, 1): -np.sqrt(3 / (8 * pi)) * s,
        (2, 0): np.sqrt(5 / (16 * pi)) * (3 * c ** 2 - 1),
        (2, 1): -np.sqrt(15 / (8 * pi)) * s * c,
        (2, 2): np.sqrt(15 / (32 * pi)) * s ** 2,
        (3, 0): np.sqrt(7 / (16 * pi)) * (5 * c ** 3 - 3 * c),
        (3, 1): -np.sqrt(21 / (64 * pi)) * s * (5 * c ** 2 - 1),
        (3, 2): np.sqrt(105 / (32 * pi)) * s ** 2 * c,
        (3, 3): -np.sqrt(35 / (64 * pi)) * s ** 3,
        (4, 0): 3 / 16 / np.sqrt(pi) * (35 * c ** 4 - 30 * c ** 2 + 3),
        (4, 4): 3 / 16 * np.sqrt(35 / (2 * pi)) * s ** 4,
    }
    return table[(ell, m)] * np.exp(1j * m * ph)


def unit(L, ell, m):
    a = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    a[ell, m + L - 1] = 1
    return a


@pytest.mark.parametrize("ell,m", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1),
                                   (3, 2), (3, 3), (4, 0), (4, 4)])
def test_inverse_gives_closed_form_Ylm(ell, m):
    L = 6
    th, ph = grid(L)
    f = T.inverse(unit(L, ell, m), L, 0)
    assert np.abs(f - closed_Y(ell, m, th, ph)).max() < 1e-14
    # negative m through Y_{l,-m} = (-1)^m Y*_{lm}
    f = T.inverse(unit(L, ell, -m), L, 0)
    assert np.abs(f - (-1) ** m * np.conj(closed_Y(ell, m, th, ph))).max() < 1e-14


@pytest.mark.parametrize("spin", [1, -1])
def test_spin_harmonics_follow_eth_operators(spin):
    """sY_lm from the spin raising/lowering operators of Sec. 2.2 applied to Y_lm.

    For Y = y(theta) e^{i m phi}: eth Y = -(y' - m y / sin) e^{i m phi}, ethbar Y = -(y' + m y / sin) e^{i m phi};
    1Y = eth Y / sqrt(l(l+1)),  -1Y = -ethbar Y / sqrt(l(l+1)).
    y' is a central difference (h = 1e-12) of the Jacobi representation evaluated in 40 digits."""
    mpmath = pytest.importorskip("mpmath")
    L = 5
    th, ph = grid(L)
    for ell in range(1, L):
        for m in range(-ell, ell + 1):
            f = T.inverse(unit(L, ell, m), L, spin)
            for t in range(L - 1):                      # skip the pole ring
                x = mpmath.mpf(float(th[t, 0]))
                with mpmath.workdps(40):
                    y = lambda b: mpmath.sqrt((2 * ell + 1) / (4 * mpmath.pi)) * wigner_d_jacobi(ell, m, 0, b, dps=40)
                    dy = (y(x + mpmath.mpf(10) ** -12) - y(x - mpmath.mpf(10) ** -12)) / (2 * mpmath.mpf(10) ** -12)
                    sx = mpmath.sin(x)
                    if spin == 1:
                        val = -(dy - m * y(x) / sx) / mpmath.sqrt(ell * (ell + 1))
                    else:
                        val = (dy + m * y(x) / sx) / mpmath.sqrt(ell * (ell + 1))
                ref = float(val) * np.exp(1j * m * ph[0])
                assert np.abs(f[t] - ref).max() < 1e-13, (ell, m, t)


@pytest.mark.parametrize("spin", [0, 1, 2, -3])
def test_addition_theorem(spin):
    """sum_m |sY_lm|^2 = (2l+1)/(4 pi) at every sample."""
    L = 9
    for ell in range(abs(spin), L):
        acc = 0
        for m in range(-ell, ell + 1):
            acc = acc + np.abs(T.inverse(unit(L, ell, m), L, spin)) ** 2
        assert np.abs(acc - (2 * ell + 1) / (4 * np.pi)).max() < 1e-13


@pytest.mark.parametrize("L,spin", [(1, 0), (2, 0), (2, 1), (3, -2), (8, 0), (17, 1), (17, -3), (32, 2)])
def test_round_trip(L, spin):
    rng = np.random.default_rng(L * 100 + spin)
    flm = rand_flm(rng, L, -spin)
    f = T.inverse(flm, L, spin)
    back = T.forward(f, L, spin)
    assert np.abs(back - flm).max() < 1e-13 * max(1.0, np.abs(flm).max())


def _forward_gauss_legendre(f, L, spin):
    """Exact forward transform by a second route: torus interpolant in theta integrated with
    L-node Gauss-Legendre quadrature (exact for cos-polynomials of degree <= 2L-1)."""
    x, w = np.polynomial.legendre.leggauss(L)
    thg = np.arccos(x)
    F = np.asarray(f) @ T.phi_dft_matrix(L, -1)                           # F_m(theta_t)
    G = T._extend(F, L, -spin)                                             # torus samples
    tt = np.arange(2 * L - 1)
    thetas_t = (2 * tt + 1) * np.pi / (2 * L - 1)
    k = np.arange(-(L - 1), L)
    coef = np.exp(-1j * np.outer(k, thetas_t)) / (2 * L - 1) @ G          # Fourier coefficients
    Gg = np.exp(1j * np.outer(thg, k)) @ coef                              # interpolant at GL nodes
    D = wigner_d_table(np.arange(L), -spin, thg.astype(np.longdouble))    # [l, m, i]
    qphi = 2 * np.pi / (2 * L - 1)
    out = np.einsum("im,lmi,i->lm", Gg, D, w) * qphi * T.ell_factor(L, spin)[:, None]
    return np.where(T.coeff_mask(L, -spin), out, 0)


@pytest.mark.parametrize("L,spin", [(4, 0), (7, 1), (12, -2), (16, 3)])
def test_forward_equals_gauss_legendre_route_on_arbitrary_data(L, spin):
    """For arbitrary (not bandlimited) MW samples both exact routes define the same linear map."""
    rng = np.random.default_rng(7 + L)
    f = rng.standard_normal((L, 2 * L - 1)) + 1j * rng.standard_normal((L, 2 * L - 1))
    a = T.forward(f, L, spin)
    b = _forward_gauss_legendre(f, L, spin)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("L,spin", [(3, 0), (4, 1), (5, -2)])
def test_inverse_brute_force_from_jacobi(L, spin):
    """O(L^4) direct synthesis f = sum flm sY_lm with sY from the Jacobi representation."""
    rng = np.random.default_rng(3)
    flm = rand_flm(rng, L, -spin)
    th, ph = grid(L)
    ref = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    for ell in range(abs(spin), L):
        for m in range(-ell, ell + 1):
            c = (-1) ** spin * np.sqrt((2 * ell + 1) / (4 * np.pi))
            d = np.array([float(wigner_d_jacobi(ell, m, -spin, float(x))) for x in th[:, 0]])
            ref += flm[ell, m + L - 1] * c * d[:, None] * np.exp(1j * m * ph)
    assert np.abs(T.inverse(flm, L, spin) - ref).max() < 1e-14 * np.abs(ref).max()


def _dense(fn, shape_in):
    n = int(np.prod(shape_in))
    cols = []
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1
        cols.append(np.asarray(fn(e.reshape(shape_in))).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("L,spin", [(3, 0), (4, 1), (5, -2)])
def test_adjoints_are_dense_conjugate_transposes(L, spin):
    shp = (L, 2 * L - 1)
    A_inv = _dense(lambda x: T.inverse(x, L, spin), shp)
    A_fwd = _dense(lambda x: T.forward(x, L, spin), shp)
    rng = np.random.default_rng(11)
    y = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    mask = T.coeff_mask(L, -spin).ravel()
    # inverse ignores coefficients outside the mask, so compare on the masked columns
    got = T.adjoint_inverse(y, L, spin).ravel()
    ref = (A_inv.conj().T @ y.ravel()) * mask
    assert np.abs(got - ref).max() < 1e-13
    got = T.adjoint_forward(np.where(T.coeff_mask(L, -spin), y, 0), L, spin).ravel()
    ref = A_fwd.conj().T @ (y.ravel() * mask)
    assert np.abs(got - ref).max() < 1e-13


@pytest.mark.parametrize("L,N", [(4, 1), (6, 3), (8, 2)])
def test_wigner_round_trip(L, N):
    rng = np.random.default_rng(L + 10 * N)
    flmn = np.stack([rand_flm(rng, L, n) for n in range(-(N - 1), N)])
    f = T.wigner_inverse(flmn, L, N)
    back = T.wigner_forward(f, L, N)
    assert np.abs(back - flmn).max() < 1e-13 * np.abs(flmn).max()


def test_wigner_inverse_of_unit_is_conjugate_D():
    """Inverse Wigner of a unit coefficient is (2l+1)/(8 pi^2) D^{l*}_{mn} = ... e^{i m alpha} d e^{i n gamma}."""
    L, N = 5, 3
    for (ell, m, n) in [(2, 1, -1), (4, -3, 2), (3, 0, 0)]:
        flmn = np.zeros((2 * N - 1, L, 2 * L - 1), dtype=np.complex128)
        flmn[n + N - 1, ell, m + L - 1] = 1
        f = T.wigner_inverse(flmn, L, N)
        th, ph = grid(L)
        gam = 2 * np.pi * np.arange(2 * N - 1) / (2 * N - 1)
        d = np.array([float(wigner_d_jacobi(ell, m, n, float(x))) for x in th[:, 0]])
        ref = ((2 * ell + 1) / (8 * np.pi ** 2) * np.exp(1j * n * gam)[:, None, None]
               * d[None, :, None] * np.exp(1j * m * ph)[None])
        assert np.abs(f - ref).max() < 1e-14


def test_wigner_N1_reduces_to_spin0_sht():
    """With N = 1, flmn^l_{m0} = 2 pi sqrt(4 pi/(2l+1)) flm (Eq. wigner_sht_forward with one gamma sample)."""
    L = 8
    rng = np.random.default_rng(5)
    f = rng.standard_normal((1, L, 2 * L - 1)) + 1j * rng.standard_normal((1, L, 2 * L - 1))
    w = T.wigner_forward(f, L, 1)[0]
    s = T.forward(f[0], L, 0)
    scale = 2 * np.pi * np.sqrt(4 * np.pi / (2 * np.arange(L) + 1))[:, None]
    assert np.abs(w - scale * s).max() < 1e-13 * np.abs(w).max()


def _golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


@pytest.mark.parametrize("L", [8, 16, 32, 64])
def test_round_trip_error_magnitude_matches_paper(L):
    """The oracle's per-coefficient round-trip error is at the paper's printed float64 level
    (Table sh_error_results, MW on-the-fly; the norm is ambiguous, so within a factor 10)."""
    paper = _golden()[str(L)]
    rng = np.random.default_rng(L)
    errs = []
    for _ in range(3):
        flm = rand_flm(rng, L, 0)
        d = T.forward(T.inverse(flm, L, 0), L, 0) - flm
        errs.append(np.abs(d[T.coeff_mask(L, 0)]).mean())
    assert np.mean(errs) < 10 * paper
