"""The Wigner transform at the size of its benchmark workload (L = 256, N = 8, batch 1, MW),
against the oracle on sampled outputs it computes one by one: rings of the inverse and degrees of
the forward, plus the round trip over every coefficient."""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L, N = 256, 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def plan():
    from paper_2311_14670_gb300 import Plan
    return Plan(L, N=N, max_batch=1)


def test_inverse_sampled_rings(plan):
    flmn = synth.flmn_gaussian(L, N, 1, seed=3001)
    got = to_np(plan.inverse(to_gpu(flmn)))                     # [1][2N-1][L][2L-1]
    rings = [0, 1, 100, 127, 200, 254, 255]
    ref = OT.wigner_inverse(flmn, L, N, rings=rings)
    assert rel_max(got[:, :, rings], ref) <= TOL64


def test_forward_sampled_degrees_on_arbitrary_samples(plan):
    f = synth.signal_gaussian((1, 2 * N - 1, L, 2 * L - 1), seed=3002)
    got = to_np(plan.forward(to_gpu(f)))                        # [1][2N-1][L][2L-1]
    ells = [0, 1, 7, 8, 100, 200, 254, 255]
    ref = OT.wigner_forward(f, L, N, ells=ells)
    assert rel_max(got[:, :, ells], ref) <= TOL64


def test_round_trip(plan):
    flmn = synth.flmn_gaussian(L, N, 1, seed=3003)
    back = to_np(plan.forward(plan.inverse(to_gpu(flmn))))
    assert rel_max(back, flmn) <= TOL64
