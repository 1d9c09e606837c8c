"""One transform split by order |m| over sequential shards on one GPU (the order-sharded path of
multigpu.py with the exchange played by a list): the assembled result is bitwise equal to the
unsharded transform, for paired (spin 0) and unpaired plans, FP64 and FP32, and for the chunked
forward theta stage above L = 2048."""
import pytest

from gpu_helpers import to_gpu
from paper_2311_14670_gb300 import synth
from paper_2311_14670_gb300.multigpu import order_ranges, sharded_forward, sharded_inverse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def _sequential(plan, x, world, fn):
    """Run every rank's shard in turn; the all-gather returns the shards computed so far."""
    ranges = order_ranges(plan.L, world, abs(plan.spin))
    locals_ = []

    def gather(t):
        locals_.append(t.clone())
        return locals_ + [torch.zeros_like(t)] * (world - len(locals_))

    outs = [fn(plan, x, ranges, r, gather) for r in range(world)]
    return outs[-1]                # the last rank's assembly saw every shard


@pytest.mark.parametrize("L,spin,world,precision", [(64, 0, 2, "fp64"), (64, 2, 3, "fp64"),
                                                    (300, -1, 8, "fp64"), (257, 0, 5, "fp64"),
                                                    (128, 0, 3, "fp32"), (96, 3, 2, "fp32")])
def test_order_sharded_equals_unsharded_bitwise(L, spin, world, precision):
    from paper_2311_14670_gb300 import Plan
    p = Plan(L, spin=spin, max_batch=2, precision=precision)
    flm = to_gpu(synth.flm_gaussian(L, spin, 2, seed=L + world)).to(p.dtype)
    f = p.inverse(flm)
    assert torch.equal(_sequential(p, flm, world, sharded_inverse), f)
    assert torch.equal(_sequential(p, f, world, sharded_forward), p.forward(f))


def test_order_sharded_chunked_forward_L2500():
    from paper_2311_14670_gb300 import Plan
    L = 2500
    p = Plan(L, spin=0)
    f = p.inverse(to_gpu(synth.flm_gaussian(L, 0, 1, seed=3)))
    assert torch.equal(_sequential(p, f, 3, sharded_forward), p.forward(f))


def test_empty_and_out_of_bounds_order_ranges():
    from paper_2311_14670_gb300 import Plan, _native
    L = 32
    p = Plan(L, spin=1)
    flm = to_gpu(synth.flm_gaussian(L, 1, 1, seed=4))
    out = torch.full(p.shape(1), 7.0 + 1j, dtype=p.dtype, device=p.device)
    p.inverse_theta_mrange(flm, 5, 5, out=out)                   # empty: nothing written
    torch.cuda.synchronize()
    assert bool((out == 7.0 + 1j).all())
    p.forward_mrange(p.inverse(flm), 0, 0, out=out)
    torch.cuda.synchronize()
    assert bool((out == 7.0 + 1j).all())
    for lo, hi in [(-1, 3), (4, 3), (0, L + 1)]:
        with pytest.raises(_native.S2GBError):
            p.inverse_theta_mrange(flm, lo, hi, out=out)
        with pytest.raises(_native.S2GBError):
            p.forward_mrange(flm, lo, hi, out=out)
    w = Plan(8, N=2)
    with pytest.raises(_native.S2GBError):
        w.inverse_phi(torch.zeros(w.spectra_shape(1), dtype=w.dtype, device=w.device))
