"""Pins for the oracle's Wigner small-d functions (CPU only).

Each pin checks the oracle against something other than itself: textbook closed forms, a
library routine (scipy's associated Legendre functions), the Jacobi-polynomial representation
in arbitrary precision, and identities of the rotation group (unitarity, composition, symmetry,
poles).  A dropped term, a wrong sign or a transposed index in the m-recursion breaks several.
"""
import numpy as np
import pytest

from oracle.sampling import mw_thetas
from oracle.wigner import PI_LD, wigner_d_jacobi, wigner_d_table

mpmath = pytest.importorskip("mpmath")

BETAS = np.array([1e-6, 0.05, 0.3, 1.0, np.pi / 2, 2.2, 3.0, np.pi - 1e-5])


def closed_d1_d2(beta):
    """Standard small-d matrices for l = 1, 2 (Wigner's convention; e.g. Varshalovich Sec. 4.16)."""
    c, s = np.cos(beta), np.sin(beta)
    d = {}
    d[(1, 1, 1)] = (1 + c) / 2
    d[(1, 1, 0)] = -s / np.sqrt(2)
    d[(1, 1, -1)] = (1 - c) / 2
    d[(1, 0, 0)] = c
    d[(2, 2, 2)] = ((1 + c) / 2) ** 2
    d[(2, 2, 1)] = -(1 + c) * s / 2
    d[(2, 2, 0)] = np.sqrt(3 / 8) * s ** 2
    d[(2, 2, -1)] = -(1 - c) * s / 2
    d[(2, 2, -2)] = ((1 - c) / 2) ** 2
    d[(2, 1, 1)] = (1 + c) * (2 * c - 1) / 2
    d[(2, 1, 0)] = -np.sqrt(3 / 2) * s * c
    d[(2, 1, -1)] = (1 - c) * (2 * c + 1) / 2
    d[(2, 0, 0)] = (3 * c ** 2 - 1) / 2
    return d


def table_value(ell, m, n, beta):
    D = wigner_d_table([ell], n, np.array([beta], dtype=np.longdouble))
    return D[0, m + ell, 0]


@pytest.mark.parametrize("beta", [0.3, 1.0, 2.2, 3.0])
def test_closed_forms_l1_l2(beta):
    ref = closed_d1_d2(beta)
    for (ell, m, n), v in ref.items():
        # closed forms are listed for m >= |n|-type entries; the symmetries give the rest
        for (mm, nn, sgn) in [(m, n, 1), (n, m, (-1) ** (m - n)), (-n, -m, 1), (-m, -n, (-1) ** (m - n))]:
            got = table_value(ell, mm, nn, beta)
            assert abs(got - sgn * v) < 1e-15, (ell, mm, nn, got, sgn * v)
            jac = float(wigner_d_jacobi(ell, mm, nn, beta))
            assert abs(jac - sgn * v) < 1e-15


@pytest.mark.parametrize("n", [0, 1, -2, 3])
def test_mrecursion_matches_jacobi_small_l(n):
    ells = np.arange(abs(n), 31)
    D = wigner_d_table(ells, n, BETAS.astype(np.longdouble))
    M = ells.max()
    err = 0.0
    for i, ell in enumerate(ells[::3]):
        i = int(np.nonzero(ells == ell)[0][0])
        for m in range(-ell, ell + 1):
            for j, b in enumerate(BETAS):
                ref = float(wigner_d_jacobi(int(ell), m, n, mpmath.mpf(b)))
                err = max(err, abs(D[i, m + M, j] - ref))
    assert err < 5e-15


def test_mrecursion_matches_jacobi_l2047_samples():
    """Spot values at l = 2047 on the MW grid of L = 2048 against arbitrary precision."""
    th = mw_thetas(2048)
    cases = [(0, 0, 0), (3, 0, 0), (3, 5, -2), (700, -300, 2), (700, 40, -2), (1023, 17, 0),
             (2046, 0, 0), (2046, 5, -2), (1500, -1999, 1)]
    for t, m, n in cases:
        with mpmath.workdps(60):
            beta = (2 * t + 1) * mpmath.pi / 4095
            ref = float(wigner_d_jacobi(2047, m, n, beta, dps=60))
        got = wigner_d_table([2047], n, th[[t]])[0, m + 2047, 0]
        assert abs(got - ref) <= 2e-15 + 1e-14 * abs(ref), (t, m, n, got, ref)


@pytest.mark.parametrize("n", [0, -2, 5])
def test_unitarity_large_l(n):
    """sum_m (d^l_{mn})^2 = 1 (unitarity of the rotation matrices) up to l = 2047."""
    th = mw_thetas(2048)[[0, 1, 9, 333, 1023, 1700, 2046]]
    D = wigner_d_table(np.array([abs(n), 64, 511, 2047]), n, th)
    dev = np.abs((D ** 2).sum(axis=1) - 1.0)
    assert dev.max() < 1e-12


def test_composition_law():
    """d(b1 + b2) = d(b1) d(b2) as (2l+1)x(2l+1) matrices, l = 60 (all m and n)."""
    ell = 60
    b1, b2 = 0.7, 1.9
    def full(beta):
        return np.stack([wigner_d_table([ell], n, np.array([beta], dtype=np.longdouble))[0, :, 0]
                         for n in range(-ell, ell + 1)], axis=1)          # [m, n]
    lhs = full(b1 + b2)
    rhs = full(b1) @ full(b2)
    assert np.abs(lhs - rhs).max() < 1e-13


@pytest.mark.parametrize("n", [0, 2, -3])
def test_symmetries(n):
    ell = 40
    b = np.array([0.4, 1.3, 2.9], dtype=np.longdouble)
    Dn = wigner_d_table([ell], n, b)[0]
    for m in range(-ell, ell + 1):
        Dm = wigner_d_table([ell], m, b)[0]
        Dneg = wigner_d_table([ell], -m, b)[0]
        # d_{mn} = (-1)^{m-n} d_{nm} = d_{-n,-m}
        assert np.allclose(Dn[m + ell], (-1) ** (m - n) * Dm[n + ell], atol=1e-14, rtol=0)
        assert np.allclose(Dn[m + ell], Dneg[-n + ell], atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [0, 1, -2])
def test_poles(n):
    ells = np.arange(abs(n), 20)
    D = wigner_d_table(ells, n, np.array([0, PI_LD, 1e-12, PI_LD - np.longdouble(1e-12)]))
    M = ells.max()
    for i, ell in enumerate(ells):
        for m in range(-ell, ell + 1):
            north = 1.0 if m == n else 0.0
            south = (-1.0) ** (ell + m) if m == -n else 0.0
            assert D[i, m + M, 0] == north
            assert D[i, m + M, 1] == south
            assert abs(D[i, m + M, 2] - north) < 1e-9      # continuity near the poles
            assert abs(D[i, m + M, 3] - south) < 1e-9


def test_spin0_against_scipy_legendre():
    """d^l_{m0}(theta) = sqrt((l-m)!/(l+m)!) P_l^m(cos theta) (Condon-Shortley phase, scipy.special.lpmv)."""
    from math import lgamma

    from scipy.special import lpmv
    th = np.array([0.2, 0.9, 1.7, 2.8])
    ells = np.arange(0, 41)
    D = wigner_d_table(ells, 0, th.astype(np.longdouble))
    for i, ell in enumerate(ells):
        for m in range(0, ell + 1):
            norm = np.exp(0.5 * (lgamma(ell - m + 1) - lgamma(ell + m + 1)))
            ref = norm * lpmv(m, ell, np.cos(th))
            assert np.allclose(D[i, m + 40], ref, atol=1e-12, rtol=1e-10)


def test_seed_is_initial_value_formula():
    """m = l entries equal Eq. "initial_values" evaluated in arbitrary precision."""
    for ell, n, b in [(7, 3, 0.8), (300, -2, 0.01), (1200, 0, 2.0), (2047, 1, 1.3)]:
        with mpmath.workdps(50):
            bb = mpmath.mpf(b)
            ref = (mpmath.sqrt(mpmath.factorial(2 * ell) / (mpmath.factorial(ell + n) * mpmath.factorial(ell - n)))
                   * (-mpmath.sin(bb / 2)) ** (ell - n) * mpmath.cos(bb / 2) ** (ell + n))
        got = table_value(ell, ell, n, b)
        assert abs(got - float(ref)) <= 1e-14 * abs(float(ref)) + 1e-300


# ---- a third, independent method: the half-integer recursion over the degree (after Risbo 1996)
def test_halfstep_recursion_matches_jacobi_small_l():
    from oracle.wigner import wigner_d_halfstep, wigner_d_jacobi
    L = 6
    betas = np.array([0.0, 0.3, 1.2, np.pi / 2, 2.9, np.pi])
    H = wigner_d_halfstep(L, betas)
    err = 0.0
    for l in range(L):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                for k, b in enumerate(betas):
                    err = max(err, abs(H[l, m + L - 1, n + L - 1, k] - float(wigner_d_jacobi(l, m, n, float(b)))))
    assert err <= 2e-15


@pytest.mark.parametrize("n", [0, 2, -3, 7])
def test_paper_recursion_over_m_matches_halfstep_recursion_l119(n):
    """The paper's recursion over m (two-sided) and the half-integer recursion over the degree agree
    to L = 120, near both poles and at the equator."""
    from oracle.wigner import wigner_d_halfstep
    L = 120
    betas = np.array([1e-3, 0.05, 0.7, 1.5707, 2.2, 3.1])
    H = wigner_d_halfstep(L, betas)[:, :, n + L - 1, :]                  # [l, m, beta]
    T = wigner_d_table(np.arange(L), n, betas.astype(np.longdouble))       # [l, m, beta]
    assert np.abs(H - T).max() <= 5e-14


def test_halfstep_matrices_are_orthogonal():
    from oracle.wigner import wigner_d_halfstep
    L = 40
    H = wigner_d_halfstep(L, np.array([0.9, 2.5]))
    for l in (1, 17, 39):
        for k in range(2):
            M = H[l, L - 1 - l:L + l, L - 1 - l:L + l, k]
            assert np.abs(M @ M.T - np.eye(2 * l + 1)).max() <= 1e-13
