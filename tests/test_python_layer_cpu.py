"""Host-side pieces of the Python layer that need no GPU: grid shapes per sampling, the domain of
valid coefficients, and the argument checks a captured transform chain makes before it touches the
device."""
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")

from oracle import transforms as OT  # noqa: E402
from paper_2311_14670_gb300 import synth  # noqa: E402
from paper_2311_14670_gb300.transforms import GraphedTransform, sampling_shape  # noqa: E402


@pytest.mark.parametrize("sampling", ["mw", "mwss", "dh"])
@pytest.mark.parametrize("L", [1, 2, 7, 64, 1024])
def test_sampling_shapes_agree_with_the_oracle(sampling, L):
    """(rings, phi samples): MW L x (2L-1), MWSS (L+1) x 2L, DH 2L x (2L-1) (Sec. 4.2)."""
    assert sampling_shape(L, sampling) == OT.sampling_shape(L, sampling)
    R, P = sampling_shape(L, sampling)
    assert R * P == {"mw": L * (2 * L - 1), "mwss": (L + 1) * 2 * L, "dh": 2 * L * (2 * L - 1)}[sampling]


@pytest.mark.parametrize("L", [1, 2, 5, 33])
def test_valid_coefficients_count_l2_minus_n2(L):
    """max(|m|, |n|) <= l < L holds at L^2 - n^2 entries (|n| < L), both in the input generator and
    in the oracle."""
    for n in range(-(L - 1), L):
        assert synth.valid_mask(L, n).sum() == L * L - n * n
        assert (synth.valid_mask(L, n) == OT.coeff_mask(L, n)).all()


def test_graphed_chain_arguments_are_checked_before_any_device_work():
    fake = SimpleNamespace(max_batch=2)                  # no device, no library handle
    with pytest.raises(ValueError):
        GraphedTransform(fake, [], 1)                    # empty chain
    with pytest.raises(ValueError):
        GraphedTransform(fake, ["inverse", "transpose"], 1)   # unknown step
    with pytest.raises(ValueError):
        GraphedTransform(fake, ["inverse", "inverse"], 1)     # a signal fed where coefficients go
    with pytest.raises(ValueError):
        GraphedTransform(fake, ["forward", "adjoint_inverse"], 1)
    with pytest.raises(ValueError):
        GraphedTransform(fake, ["inverse", "forward"], 3)     # batch above max_batch
    with pytest.raises(ValueError):
        GraphedTransform(fake, ["inverse", "forward"], 0)
