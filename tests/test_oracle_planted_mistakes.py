"""The oracle's pins catch plausible mistakes: each test plants one mistake in the oracle (on the
CPU, by replacing one of its functions for the duration of the test) and checks that one of the
oracle's pins then fails.  A pin that still passed with the mistake in place would
not be pinning that part of the oracle.

Mistakes planted, with the pin that must catch them:
  * the spin sign (-1)^s dropped from c_l                  -> brute force from the Jacobi form
  * d^l_{n,m} used where d^l_{m,n} belongs (transposed)     -> brute force from the Jacobi form
  * the phi-DFT exponent sign flipped (both directions)     -> closed-form Y_lm (a round trip would
                                                               not notice)
  * the torus-extension parity (-1)^{m+s} dropped           -> round trip
  * uniform theta weights instead of the MW weights         -> round trip
  * the DH-like grid (2t+1) pi/(2L) in place of MW's        -> closed-form Y_lm
  * the gamma-DFT exponent sign flipped (Wigner)            -> inverse of a unit coefficient = D*
  * the Wigner factor (2l+1)/(8 pi^2) replaced by c_l       -> inverse of a unit coefficient = D*
  * ln((k+1)!) for ln(k!) in the seeds                      -> closed-form d^1, d^2
  * the DH weight's sine series one term too long           -> exact integration of P_n, n < 2L
  * the MWSS pole rings counted twice                       -> exact integration of cos^n
  * float64 MW weights inside the extended-precision mode   -> its round trip at extended rounding
The pins of the d-functions, the samplings and the transforms live in ``test_oracle_wigner``,
``test_oracle_samplings`` and ``test_oracle_transforms``.
"""
import numpy as np
import pytest

import oracle.sampling as S
import oracle.transforms as T
import oracle.wigner as W
import test_oracle_samplings as spins
import test_oracle_transforms as pins
import test_oracle_wigner as dpins


def _fails(check, *args):
    with pytest.raises(AssertionError):
        check(*args)


def test_the_pins_pass_without_a_planted_mistake():
    pins.test_inverse_brute_force_from_jacobi(4, 1)
    pins.test_inverse_gives_closed_form_Ylm(2, 1)
    pins.test_round_trip(17, 1)
    pins.test_wigner_inverse_of_unit_is_conjugate_D()


def test_dropped_spin_sign_in_c_l(monkeypatch):
    monkeypatch.setattr(T, "ell_factor", lambda L, spin, dtype=np.float64:
                        np.sqrt((2 * np.arange(L) + 1) / (4 * np.pi)).astype(dtype))
    _fails(pins.test_inverse_brute_force_from_jacobi, 4, 1)


def test_transposed_d_function(monkeypatch):
    orig = T.wigner_d_table

    def transposed(ells, n, thetas, dtype=np.float64):
        D = orig(ells, n, thetas, dtype)                       # [l, m, t], m centred on the middle column
        w = D.shape[1]
        m = np.arange(w) - (w - 1) // 2
        return D * ((-1.0) ** ((m - n) % 2))[None, :, None]    # d^l_{n,m} = (-1)^{m-n} d^l_{m,n}

    monkeypatch.setattr(T, "wigner_d_table", transposed)
    _fails(pins.test_inverse_brute_force_from_jacobi, 4, 1)


def test_flipped_phi_dft_sign(monkeypatch):
    orig = T.phi_dft_matrix
    monkeypatch.setattr(T, "phi_dft_matrix", lambda L, sign, dtype=np.float64: orig(L, -sign, dtype))
    pins.test_round_trip(8, 0)                          # the round trip alone cannot see it
    _fails(pins.test_inverse_gives_closed_form_Ylm, 2, 1)


def test_dropped_torus_extension_parity(monkeypatch):
    def no_parity(F, L, n, orders=None):
        G = np.zeros(F.shape[:-2] + (2 * L - 1, F.shape[-1]), dtype=np.complex128)
        G[..., :L, :] = F
        G[..., L:, :] = F[..., :L - 1, :][..., ::-1, :]
        return G

    monkeypatch.setattr(T, "_extend", no_parity)
    _fails(pins.test_round_trip, 17, 1)


def test_uniform_theta_weights(monkeypatch):
    monkeypatch.setattr(T, "mw_theta_weights", lambda Lp, dtype=np.float64: np.full(Lp, 2.0 / Lp, dtype=dtype))
    _fails(pins.test_round_trip, 17, 1)


def test_wrong_ring_positions(monkeypatch):
    monkeypatch.setattr(T, "mw_thetas", lambda L, dtype=np.longdouble:
                        ((2 * np.arange(L) + 1) * np.pi / (2 * L)).astype(dtype))
    _fails(pins.test_inverse_gives_closed_form_Ylm, 2, 1)


def test_flipped_gamma_dft_sign(monkeypatch):
    orig = T._gamma_matrix
    monkeypatch.setattr(T, "_gamma_matrix", lambda N, sign, dtype=np.float64: orig(N, -sign, dtype))
    _fails(pins.test_wigner_inverse_of_unit_is_conjugate_D)


def test_sphere_factor_in_the_wigner_inverse(monkeypatch):
    orig = T._theta_inverse

    def sphere_scaled(flm, L, n, scale, thetas, dtype=np.float64):
        return orig(flm, L, n, (-1.0) ** n * np.sqrt((2 * np.arange(L) + 1) / (4 * np.pi)), thetas, dtype)

    monkeypatch.setattr(T, "_theta_inverse", sphere_scaled)
    _fails(pins.test_wigner_inverse_of_unit_is_conjugate_D)


# ---------------------------------------------------------------- d-functions and samplings


def test_sampling_and_d_pins_pass_without_a_planted_mistake():
    dpins.test_closed_forms_l1_l2(1.0)
    spins.test_dh_weights_integrate_legendre_polynomials_exactly(8)
    spins.test_mwss_weights_integrate_even_torus_functions(12)


def test_log_factorials_off_by_one(monkeypatch):
    """ln((k+1)!) in place of ln(k!) in the seeds of Eq. initial_values."""
    orig = W._log_factorials
    monkeypatch.setattr(W, "_log_factorials", lambda kmax: orig(kmax + 1)[1:])
    _fails(dpins.test_closed_forms_l1_l2, 1.0)


def test_dh_weight_sum_one_term_too_long(monkeypatch):
    """The DH weight's sine series summed over k <= L instead of k < L."""
    def long_sum(L):
        th = S.dh_thetas(L)
        k = np.arange(L + 1).astype(np.longdouble)
        s = (np.sin(np.outer(th, 2 * k + 1)) / (2 * k + 1)).sum(axis=1)
        return (np.longdouble(2) / L * np.sin(th) * s).astype(np.float64)

    monkeypatch.setattr(spins, "dh_theta_weights", long_sum)
    _fails(spins.test_dh_weights_integrate_legendre_polynomials_exactly, 8)


def test_mwss_poles_counted_twice(monkeypatch):
    """The MWSS pole rings folded with their own reflection (counted twice)."""
    orig = S.mwss_theta_weights

    def doubled(Lp):
        q = orig(Lp).copy()
        q[0] *= 2
        q[-1] *= 2
        return q

    monkeypatch.setattr(spins, "mwss_theta_weights", doubled)
    _fails(spins.test_mwss_weights_integrate_even_torus_functions, 12)


def test_float64_weights_inside_the_extended_mode(monkeypatch):
    """The extended-precision mode fed the float64 MW weights: its round-trip pin must fail."""
    import test_oracle_exact as epins
    if epins.EPS_LD > 1e-17:
        pytest.skip("np.longdouble is not wider than float64 here")
    orig = T.mw_theta_weights
    monkeypatch.setattr(T, "mw_theta_weights", lambda Lp, dtype=np.float64: orig(Lp).astype(dtype))
    _fails(epins.test_exact_round_trip_at_extended_rounding_level, 8, 0)
