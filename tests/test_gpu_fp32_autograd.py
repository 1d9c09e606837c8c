"""Mixed-precision (float32) transforms and the autograd wrappers.

The float32 path has no bit-level parity target: its error against the float64 oracle is measured
and bounded per configuration (recursion and contraction in float32 with float64 starting values
and compensated sums; the error grows with L like sqrt(L) ... L times float32 rounding).
Gradients: torch.autograd.gradcheck (finite differences, float64) at small L, and a directional
finite-difference check of the loss sum |inverse(flm) - target|^2 at L = 32 in both precisions.
"""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# float32 bounds on the relative max error against the float64 oracle, per L (measured values are
# reported by bench.py; these are upper bounds with margin).
FP32_BOUND = {16: 2e-6, 64: 5e-6, 257: 2e-5, 1024: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def plan(L, spin=0, N=0, max_batch=1, precision="fp64"):
    from paper_2311_14670_gb300 import Plan
    return Plan(L, spin=spin, N=N, max_batch=max_batch, precision=precision)


@pytest.mark.parametrize("L,spin", [(16, 0), (64, 2), (257, -1)])
def test_fp32_inverse_and_forward_against_fp64_oracle(L, spin):
    B = 3
    p = plan(L, spin, max_batch=B, precision="fp32")
    flm = synth.flm_gaussian(L, spin, B, seed=L)
    f32 = p.inverse(to_gpu(flm, torch.complex64))
    ref = OT.inverse(flm, L, spin)
    assert rel_max(to_np(f32), ref) <= FP32_BOUND[L]
    f = synth.signal_gaussian((B, L, 2 * L - 1), seed=L + 1)
    got = p.forward(to_gpu(f, torch.complex64))
    assert rel_max(to_np(got), OT.forward(f, L, spin)) <= FP32_BOUND[L]


def test_fp32_theta_kernels_at_L1024_batch16_against_fp64_gpu():
    """The mixed-precision workload shape (batch 16) at L = 1024: float32 theta stages against the
    float64 theta stages (which match the oracle to 1e-12)."""
    L, B = 1024, 16
    p64 = plan(L, 0, max_batch=B)
    p32 = plan(L, 0, max_batch=B, precision="fp32")
    flm = synth.flm_gaussian(L, 0, B, seed=5, ell_power=1.0)
    x = to_gpu(flm)
    ref = p64.inverse_theta(x)
    got = p32.inverse_theta(x.to(torch.complex64))
    assert rel_max(to_np(got), to_np(ref)) <= FP32_BOUND[1024]
    g = to_gpu(synth.signal_gaussian((B, 2 * L - 1, L), seed=6))
    ref = p64.forward_theta(g)
    got = p32.forward_theta(g.to(torch.complex64))
    assert rel_max(to_np(got), to_np(ref)) <= FP32_BOUND[1024]


def test_fp32_wigner_round_trip():
    L, N = 16, 3
    p = plan(L, N=N, precision="fp32")
    flmn = synth.flmn_gaussian(L, N, 1, seed=9)
    back = p.forward(p.inverse(to_gpu(flmn, torch.complex64)))
    assert rel_max(to_np(back), flmn) <= 1e-5


@pytest.mark.parametrize("spin", [0, 1])
def test_gradcheck_float64(spin):
    from paper_2311_14670_gb300 import forward, inverse
    L = 6
    p = plan(L, spin)
    mask = torch.from_numpy(synth.valid_mask(L, -spin)).cuda()
    flm = to_gpu(synth.flm_gaussian(L, spin, 1, seed=3)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a: inverse(a * mask, p), (flm,), eps=1e-6, atol=1e-8, rtol=1e-6)
    f = to_gpu(synth.signal_gaussian((1, L, 2 * L - 1), seed=4)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a: forward(a, p), (f,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_gradcheck_wigner_float64():
    from paper_2311_14670_gb300 import forward, inverse
    L, N = 5, 2
    p = plan(L, N=N)
    mask = torch.from_numpy(np.stack([synth.valid_mask(L, n) for n in range(-(N - 1), N)])).cuda()
    x = to_gpu(synth.flmn_gaussian(L, N, 1, seed=3)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a: inverse(a * mask, p), (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
    f = to_gpu(synth.signal_gaussian((1, 2 * N - 1, L, 2 * L - 1), seed=4)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a: forward(a, p), (f,), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-3)])
def test_loss_gradient_matches_finite_differences_L32(precision, tol):
    """loss = sum |inverse(flm) - target|^2 (the mixed-precision workload's loss, Gaussian random
    field target with C_l ~ (l+1)^-2); its gradient from the hand-written adjoint against central
    differences along random directions."""
    from paper_2311_14670_gb300 import inverse
    L, B = 32, 2
    p = plan(L, 0, max_batch=B, precision=precision)
    dt = p.dtype
    mask = torch.from_numpy(synth.valid_mask(L, 0)).cuda()
    target = inverse(to_gpu(synth.flm_gaussian(L, 0, B, seed=11, ell_power=1.0), dt), p).detach()
    flm = to_gpu(synth.flm_gaussian(L, 0, B, seed=12), dt).requires_grad_(True)

    def loss(a):
        return ((inverse(a * mask, p) - target).abs() ** 2).sum()

    value = loss(flm)
    value.backward()
    grad = flm.grad.detach()
    rng = np.random.default_rng(13)
    for _ in range(3):
        d = to_gpu(synth.complex_gaussian(rng, flm.shape), dt) * mask
        h = 1e-4 if precision == "fp64" else 3e-2
        with torch.no_grad():
            fd = (loss(flm + h * d).double() - loss(flm - h * d).double()) / (2 * h)
        # d loss = Re <grad, d> for PyTorch's conjugate-Wirtinger gradient convention
        an = torch.vdot(grad.flatten(), d.flatten()).real.double()
        assert abs(float(fd - an)) <= tol * abs(float(an)) + 1e-9 * float(value.detach().abs().double())
