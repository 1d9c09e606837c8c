"""Pins of the oracle's real-signal transforms (Sec. 2.2 Hermitian symmetry) against facts that do
not come from the functions under test: the complex oracle transforms, reality of the synthesised
signal, exact round trips and the adjoint identities of real-linear maps."""
import numpy as np
import pytest

from oracle import transforms as OT
from paper_2311_14670_gb300 import synth


def _rdot(a, b):
    return float(np.sum(np.conj(a) * b).real)


@pytest.mark.parametrize("L", [1, 2, 5, 12])
def test_hermitian_coefficients_synthesise_a_real_signal(L):
    """With the (-1)^m sign of Sec. 2.2 the complex inverse of the expanded coefficients is real;
    a wrong sign (or a missing conjugate) leaves an imaginary part of the size of the signal."""
    a = synth.flm_real_gaussian(L, 2, seed=L)
    f = OT.inverse(OT.hermitian_expand(a, L), L, 0)
    assert np.abs(f.imag).max() <= 1e-13 * max(1.0, np.abs(f).max())
    if L >= 2:
        bad = OT.hermitian_expand(a, L)
        bad[..., :L - 1] = -bad[..., :L - 1]                    # plant: drop the (-1)^m pattern
        fb = OT.inverse(bad, L, 0)
        assert np.abs(fb.imag).max() > 1e-3 * np.abs(fb).max()


@pytest.mark.parametrize("L", [3, 8, 13])
def test_forward_of_a_real_signal_is_hermitian(L):
    """The complex oracle forward of arbitrary real samples obeys flm(l,-m) = (-1)^m conj flm(l,m)."""
    f = synth.signal_real_gaussian((2, L, 2 * L - 1), seed=3 * L)
    full = OT.forward(f.astype(np.complex128), L, 0)
    m = np.arange(1, L)
    lhs = full[..., L - 1 - m]
    rhs = ((-1.0) ** m) * np.conj(full[..., L - 1 + m])
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(full).max()
    assert np.abs(full[..., L - 1].imag).max() <= 1e-13 * np.abs(full).max()
    assert np.array_equal(OT.forward_real(f, L), full[..., L - 1:])


@pytest.mark.parametrize("L", [4, 9])
def test_real_round_trip(L):
    a = synth.flm_real_gaussian(L, 3, seed=7 + L)
    back = OT.forward_real(OT.inverse_real(a, L), L)
    assert np.abs(back - a).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("L", [3, 7])
def test_real_adjoint_identities(L):
    """<A x, y> = <x, A^T y> in the real inner product, with nonzero Im flm(l, 0) on the
    coefficient side (which the real maps ignore)."""
    rng = np.random.default_rng(L)
    x = synth.flm_real_gaussian(L, 1, seed=L) + 1j * rng.standard_normal((1, L, L)) * (np.arange(L) == 0)
    x = np.where(np.arange(L)[None, :] <= np.arange(L)[:, None], x, 0)
    y = synth.signal_real_gaussian((1, L, 2 * L - 1), seed=L + 1)
    assert abs(_rdot(OT.inverse_real(x, L), y) - _rdot(x, OT.adjoint_inverse_real(y, L))) <= 1e-12 * (
        np.abs(x).sum() * np.abs(y).sum())
    z = x
    assert abs(_rdot(OT.forward_real(y, L), z) - _rdot(y, OT.adjoint_forward_real(z, L))) <= 1e-12 * (
        np.abs(z).sum() * np.abs(y).sum())
