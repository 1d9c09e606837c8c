"""Pins for the oracle's MW sampling and quadrature weights (CPU only)."""
import numpy as np
import pytest

from oracle.sampling import mw_theta_weights, mw_thetas, mw_torus_thetas, w_hat
from oracle.wigner import wigner_d_table


def test_grid_positions():
    L = 5
    th = mw_thetas(L, dtype=np.float64)
    assert np.allclose(th, (2 * np.arange(L) + 1) * np.pi / (2 * L - 1), rtol=0, atol=1e-15)
    assert th[-1] == np.pi
    tt = mw_torus_thetas(L, dtype=np.float64)
    # reflection theta_{2L-2-t} = 2 pi - theta_t
    assert np.allclose(tt[2 * L - 2 - np.arange(L - 1)], 2 * np.pi - tt[: L - 1], atol=1e-14)


def test_w_hat_is_the_fourier_integral():
    """w_hat(m') equals int_0^pi sin(theta) e^{i m' theta} dtheta (numerical quadrature)."""
    from scipy.integrate import quad
    for mp in range(-6, 7):
        re = quad(lambda x: np.sin(x) * np.cos(mp * x), 0, np.pi, epsabs=1e-14)[0]
        im = quad(lambda x: np.sin(x) * np.sin(mp * x), 0, np.pi, epsabs=1e-14)[0]
        assert abs(w_hat(np.array([mp]))[0] - (re + 1j * im)) < 1e-13


@pytest.mark.parametrize("Lp", [1, 2, 3, 8, 33, 128])
def test_weights_sum_to_two(Lp):
    assert abs(mw_theta_weights(Lp).sum() - 2.0) < 1e-13


@pytest.mark.parametrize("Lp", [4, 9, 64])
def test_weights_integrate_trig_polynomials_exactly(Lp):
    """sum_t q_t cos(k theta_t) = int_0^pi cos(k theta) sin(theta) dtheta for |k| <= Lp-1."""
    q = mw_theta_weights(Lp)
    th = mw_thetas(Lp, dtype=np.float64)
    for k in range(0, Lp):
        exact = 0.0 if k == 1 else (1 + (-1) ** k) / (1 - k * k)
        assert abs(q @ np.cos(k * th) - exact) < 1e-13, k
    # and not beyond the bandlimit (the pin can fail)
    k = 2 * Lp
    exact = (1 + (-1) ** k) / (1 - k * k)
    assert abs(q @ np.cos(k * th) - exact) > 1e-6


@pytest.mark.parametrize("n", [0, 1, -1, 2, 3])
def test_orthogonality_on_upsampled_grid(n):
    """sum_u q_u d^l_{mn} d^l'_{mn} = 2 delta_{ll'}/(2l+1) on the MW grid of bandlimit 2L.

    At odd n this separates the fold readings: a fold factor (-1)^s would break it."""
    L = 12
    q = mw_theta_weights(2 * L)
    th = mw_thetas(2 * L)
    ells = np.arange(abs(n), L)
    D = wigner_d_table(ells, n, th)                       # [l, m, u]
    for mi in range(-(L - 1), L):
        sub = D[:, mi + L - 1, :]
        G = (sub * q) @ sub.T
        valid = ells >= abs(mi)
        exp = np.diag(np.where(valid, 2.0 / (2 * ells + 1), 0.0))
        assert np.abs(G - exp).max() < 1e-14


def test_planted_fold_sign_breaks_orthogonality():
    """The printed fold factor zeta_t (-1)^s, planted into a copy of the weights, fails at odd spin."""
    L, n = 6, 1
    Lp = 2 * L
    T = 2 * Lp - 1
    tt = mw_torus_thetas(Lp, dtype=np.float64)
    k = np.arange(-(Lp - 1), Lp)
    w = np.exp(-1j * np.outer(tt, k)) @ w_hat(k)
    q_bad = np.array([(w[t] + (0 if t == Lp - 1 else -1) * w[2 * Lp - 2 - t]).real / T for t in range(Lp)])
    th = mw_thetas(Lp)
    D = wigner_d_table(np.arange(1, L), n, th)
    sub = D[:, 0 + L - 1, :]
    G = (sub * q_bad) @ sub.T
    assert np.abs(G - np.diag(2.0 / (2 * np.arange(1, L) + 1))).max() > 1e-5
