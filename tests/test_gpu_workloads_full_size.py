"""Benchmark workloads not covered elsewhere at full size, against the oracle on sampled outputs
it computes one by one:
  * the Wigner transform at L = 256, N = 8, batch 1 (MW): sampled rings of the inverse, sampled
    degrees of the forward, and the round trip over every coefficient;
  * the float32 gradient workload at L = 2048, spin 0, batch 16: the inverse on sampled rings
    against the float64 oracle, and the adjoint of the inverse (the backward pass) against the
    float64 GPU path, which matches the oracle to 1e-12.
The float32 bound is 2e-4 relative max error: the measured errors at this size are about 1e-6
(inverse) and 1.5e-5 (forward-shaped contraction), and the bound grows like L, as
test_gpu_fp32_autograd's per-L bounds do (1e-4 at L = 1024)."""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_BOUND_L2048 = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def wigner_plan():
    from paper_2311_14670_gb300 import Plan
    return Plan(256, N=8, max_batch=1)


def test_wigner_inverse_sampled_rings(wigner_plan):
    L, N = 256, 8
    flmn = synth.flmn_gaussian(L, N, 1, seed=3001)
    got = to_np(wigner_plan.inverse(to_gpu(flmn)))              # [1][2N-1][L][2L-1]
    rings = [0, 1, 100, 127, 200, 254, 255]
    ref = OT.wigner_inverse(flmn, L, N, rings=rings)
    assert rel_max(got[:, :, rings], ref) <= TOL64


def test_wigner_forward_sampled_degrees_on_arbitrary_samples(wigner_plan):
    L, N = 256, 8
    f = synth.signal_gaussian((1, 2 * N - 1, L, 2 * L - 1), seed=3002)
    got = to_np(wigner_plan.forward(to_gpu(f)))                 # [1][2N-1][L][2L-1]
    ells = [0, 1, 7, 8, 100, 200, 254, 255]
    ref = OT.wigner_forward(f, L, N, ells=ells)
    assert rel_max(got[:, :, ells], ref) <= TOL64


def test_wigner_round_trip(wigner_plan):
    L, N = 256, 8
    flmn = synth.flmn_gaussian(L, N, 1, seed=3003)
    back = to_np(wigner_plan.forward(wigner_plan.inverse(to_gpu(flmn))))
    assert rel_max(back, flmn) <= TOL64


def test_fp32_gradient_workload_L2048_batch16():
    from paper_2311_14670_gb300 import Plan
    L, B = 2048, 16
    p32 = Plan(L, max_batch=B, precision="fp32")
    flm = synth.flm_gaussian(L, 0, B, seed=3004, ell_power=1.0)
    f32 = to_np(p32.inverse(to_gpu(flm, torch.complex64)))
    rings = [0, 1, 1023, 2046, 2047]
    ref = OT.inverse(flm, L, 0, rings=rings)
    assert rel_max(f32[:, rings], ref) <= FP32_BOUND_L2048
    del f32
    y = synth.signal_gaussian((B, L, 2 * L - 1), seed=3005)
    got = p32.adjoint_inverse(to_gpu(y, torch.complex64))
    del p32
    p64 = Plan(L, max_batch=B)
    ref64 = p64.adjoint_inverse(to_gpu(y))
    assert rel_max(to_np(got), to_np(ref64)) <= FP32_BOUND_L2048
