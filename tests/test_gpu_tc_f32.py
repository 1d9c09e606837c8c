"""The float32 inverse theta stage with the contraction on the tensor cores (the default for
float32 plans of max_batch >= 16; S2GB_PLAN_FMA_CONTRACTION keeps the FMA-pipe kernel): four exact
base-256 digits per operand, integer level sums.

Against the float64 oracle within the float32 bounds of the mixed-precision path, for every
signal-group size the launcher picks (1, 2, 4, 8, 16 signals per CTA), ragged bandlimits, both
recursion forms (polar-cap tiles) and coefficient magnitudes near float32's range; against the
FMA-pipe float32 kernel on the same inputs; bitwise the same whether a signal is transformed
alone or in a batch of 16 (integer sums, one exponent per column)."""
import numpy as np
import pytest

from gpu_helpers import rel_max, to_gpu, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {5: 2e-6, 16: 2e-6, 33: 4e-6, 64: 5e-6, 130: 1e-5, 257: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def plan(L, spin=0, B=1, **kw):
    """A float32 plan that takes the tensor-core path (max_batch >= 16) for calls on B signals."""
    from paper_2311_14670_gb300 import Plan
    return Plan(L, spin=spin, max_batch=max(B, 16), precision="fp32", **kw)


@pytest.mark.parametrize("L,spin,B", [(5, 0, 1), (16, 1, 2), (33, -2, 3), (64, 0, 5), (130, 2, 8),
                                      (64, 1, 16), (33, 0, 17), (257, -1, 4)])
def test_tc32_inverse_matches_fp64_oracle(L, spin, B):
    p = plan(L, spin, B)
    flm = synth.flm_gaussian(L, spin, B, seed=L * 3 + B)
    got = to_np(p.inverse(to_gpu(flm, torch.complex64)))
    ref = OT.inverse(flm, L, spin)
    assert rel_max(got, ref) <= BOUND[L]


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_tc32_inverse_extreme_coefficient_magnitudes(scale):
    L, B = 33, 2
    p = plan(L, 1, B)
    flm = synth.flm_gaussian(L, 1, B, seed=2) * scale
    got = to_np(p.inverse(to_gpu(flm, torch.complex64)))
    ref = OT.inverse(flm, L, 1)
    assert rel_max(got, ref) <= BOUND[L]


def test_tc32_column_with_wide_dynamic_range():
    """One column's coefficients span 1e-20 .. 1: every degree still contributes at float32 level."""
    L = 64
    flm = synth.flm_gaussian(L, 0, 1, seed=3)
    flm *= np.logspace(0, -20, L)[None, :, None]
    got = to_np(plan(L).inverse(to_gpu(flm, torch.complex64)))
    assert rel_max(got, OT.inverse(flm, L, 0)) <= BOUND[64]


@pytest.mark.parametrize("L,spin,B", [(64, 2, 4), (257, 0, 16)])
def test_tc32_agrees_with_fma_pipe_kernel(L, spin, B):
    flm = synth.flm_gaussian(L, spin, B, seed=7)
    x = to_gpu(flm, torch.complex64)
    a = to_np(plan(L, spin, B).inverse_theta(x))
    b = to_np(plan(L, spin, B, fma_contraction=True).inverse_theta(x))
    assert rel_max(a, b) <= 2 * BOUND[L]


def test_tc32_alone_and_in_a_batch_are_bitwise_equal():
    L, B = 64, 16
    p = plan(L, 2, B)
    flm = synth.flm_gaussian(L, 2, B, seed=11)
    x = to_gpu(flm, torch.complex64)
    batch = p.inverse_theta(x)
    for b in (0, 7, 15):
        alone = p.inverse_theta(x[b:b + 1].contiguous())
        assert torch.equal(alone[0], batch[b])


@pytest.mark.parametrize("kind", ["real", "mwss", "dh"])
def test_tc32_other_plan_kinds(kind):
    L, B = 40, 3
    if kind == "real":
        p = plan(L, 0, B, real=True)
        a = synth.flm_real_gaussian(L, B, seed=5)
        got = to_np(p.inverse(to_gpu(a, torch.complex64)))
        ref = OT.inverse_real(a, L)
    else:
        p = plan(L, 1, B, sampling=kind)
        flm = synth.flm_gaussian(L, 1, B, seed=6)
        got = to_np(p.inverse(to_gpu(flm, torch.complex64)))
        ref = np.stack([OT.inverse_s(flm[b], L, 1, kind) for b in range(B)])
    assert rel_max(got, ref) <= 1e-5


def test_tc32_round_trip_full_size_batch16():
    """The mixed-precision workload's shape at L = 1024: the tensor-core inverse and the float32
    forward on 16 signals."""
    L, B = 1024, 16
    p = plan(L, 0, B)
    flm = synth.flm_gaussian(L, 0, B, seed=21, ell_power=1.0)
    back = to_np(p.forward(p.inverse(to_gpu(flm, torch.complex64))))
    assert rel_max(back, flm) <= 1e-5
