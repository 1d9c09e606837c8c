"""Real-signal (Hermitian, spin 0) transforms through the C ABI against the oracle: orders m >= 0
only, real f.  Element by element at small sizes, sampled rings / degrees at L = 1024 and 2048,
adjoints, autograd, order sharding, FP32."""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def rplan(L, max_batch=1, precision="fp64"):
    from paper_2311_14670_gb300 import Plan
    return Plan(L, real=True, max_batch=max_batch, precision=precision)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


SMALL = [1, 2, 3, 16, 17, 64, 130, 257]


@pytest.mark.parametrize("L", SMALL)
@pytest.mark.parametrize("batch", [1, 3])
def test_real_inverse_and_forward_match_oracle(L, batch):
    p = rplan(L, batch)
    a = synth.flm_real_gaussian(L, batch, seed=L + batch)
    f = p.inverse(dev(a))
    assert f.dtype == torch.float64 and tuple(f.shape) == (batch, L, 2 * L - 1)
    assert rel_max(to_np(f), OT.inverse_real(a, L)) <= TOL64
    g = synth.signal_real_gaussian((batch, L, 2 * L - 1), seed=2 * L + batch)
    got = to_np(p.forward(dev(g)))
    assert rel_max(got, OT.forward_real(g, L)) <= TOL64


@pytest.mark.parametrize("L", [2, 9, 40])
def test_real_adjoints_match_oracle(L):
    p = rplan(L, 2)
    y = synth.signal_real_gaussian((2, L, 2 * L - 1), seed=L)
    assert rel_max(to_np(p.adjoint_inverse(dev(y))), OT.adjoint_inverse_real(y, L)) <= TOL64
    z = synth.flm_real_gaussian(L, 2, seed=L + 1)
    z[..., 0] += 1j                                              # ignored by the real maps
    z = np.where(np.arange(L)[None, :] <= np.arange(L)[:, None], z, 0)
    assert rel_max(to_np(p.adjoint_forward(dev(z))), OT.adjoint_forward_real(z, L)) <= TOL64


def test_imaginary_part_of_m0_is_ignored_by_the_inverse():
    L = 20
    p = rplan(L)
    a = synth.flm_real_gaussian(L, 1, seed=5)
    b = a.copy()
    b[..., 0] += 3j
    assert torch.equal(p.inverse(dev(a)), p.inverse(dev(b)))


def test_real_equals_complex_transform_of_the_hermitian_expansion():
    """The real plan against the complex spin-0 plan of the same signal (both on the GPU)."""
    from paper_2311_14670_gb300 import Plan
    L = 300
    p, c = rplan(L), Plan(L)
    a = synth.flm_real_gaussian(L, 1, seed=9, ell_power=1.0)
    fr = p.inverse(dev(a))
    fc = c.inverse(dev(OT.hermitian_expand(a, L)))
    assert rel_max(to_np(fr), to_np(fc).real) <= TOL64
    assert rel_max(to_np(p.forward(fr)), to_np(c.forward(fc))[..., L - 1:]) <= TOL64


@pytest.mark.parametrize("L,B", [(1024, 4), (2048, 1)])
def test_full_size_real_sampled_and_round_trip(L, B):
    p = rplan(L, B)
    a = synth.flm_real_gaussian(L, B, seed=L, ell_power=1.0)
    f = p.inverse(dev(a))
    rings = [0, 1, L // 2, L - 2, L - 1]
    full = OT.hermitian_expand(a, L)
    ref = OT.inverse(full, L, 0, rings=rings).real
    assert rel_max(to_np(f)[:, rings], ref) <= TOL64
    assert rel_max(to_np(p.forward(f)), a) <= TOL64


def test_real_chunked_forward_L2500():
    L = 2500
    p = rplan(L)
    a = synth.flm_real_gaussian(L, 1, seed=1, ell_power=1.0)
    assert rel_max(to_np(p.forward(p.inverse(dev(a)))), a) <= TOL64


def test_real_autograd_matches_finite_differences():
    from paper_2311_14670_gb300 import forward, inverse
    L = 12
    p = rplan(L)
    a = dev(synth.flm_real_gaussian(L, 1, seed=2)).requires_grad_(True)
    w = dev(synth.signal_real_gaussian((1, L, 2 * L - 1), seed=3))
    loss = (inverse(a, p) * w).sum() + (forward(inverse(a, p), p).abs() ** 2).sum()
    loss.backward()
    g = to_np(a.grad)
    a0 = to_np(a.detach())
    h = 1e-6
    for (l, m, part) in [(3, 2, 1.0), (5, 0, 1.0), (7, 4, 1j), (11, 11, 1j)]:
        e = np.zeros_like(a0)
        e[0, l, m] = part
        vals = []
        for s in (+1, -1):
            x = dev(a0 + s * h * e)
            vals.append(float((p.inverse(x) * w).sum() + (p.forward(p.inverse(x)).abs() ** 2).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = g[0, l, m].real if part == 1.0 else g[0, l, m].imag
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def test_real_order_sharding_is_bitwise():
    from paper_2311_14670_gb300.multigpu import order_ranges, sharded_forward, sharded_inverse
    L, world = 200, 3
    p = rplan(L)
    a = dev(synth.flm_real_gaussian(L, 1, seed=4))
    f = p.inverse(a)
    ranges = order_ranges(L, world, 0, real=True)
    for fn, x, ref in ((sharded_inverse, a, f), (sharded_forward, f, p.forward(f))):
        parts = []

        def gather(t):
            parts.append(t.clone())
            return parts + [torch.zeros_like(t)] * (world - len(parts))

        outs = [fn(p, x, ranges, r, gather) for r in range(world)]
        assert torch.equal(outs[-1], ref)


@pytest.mark.parametrize("L", [64, 1024])
def test_real_fp32_error_against_fp64(L):
    p64, p32 = rplan(L), rplan(L, precision="fp32")
    a = synth.flm_real_gaussian(L, 1, seed=L, ell_power=1.0)
    f64 = to_np(p64.inverse(dev(a)))
    f32 = to_np(p32.inverse(dev(a, torch.complex64)))
    assert f32.dtype == np.float32
    # the complex FP32 path measures 6.9e-6 (inverse + forward) at L = 1024: the same bar here
    assert rel_max(f32, f64) <= 1.5e-5
    back = to_np(p32.forward(dev(f32)))
    assert rel_max(back, a) <= 3e-5
