"""Precompute mode (d-functions kept in device memory, S2GB_PLAN_PRECOMPUTE) against the oracle and
against the on-the-fly plans: every element at small sizes for the sphere (spin 0 paired, spin != 0),
Wigner and real-signal plans, adjoints, sampled outputs at L = 1024 / 2048."""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
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


def pplan(L, spin=0, N=0, max_batch=1, real=False):
    from paper_2311_14670_gb300 import Plan
    return Plan(L, spin=spin, N=N, max_batch=max_batch, real=real, precompute=True)


@pytest.mark.parametrize("L,spin", [(1, 0), (2, 1), (3, -2), (16, 0), (33, -1), (64, 2), (130, 0), (257, 3)])
@pytest.mark.parametrize("batch", [1, 3])
def test_precompute_sphere_matches_oracle(L, spin, batch):
    p = pplan(L, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=L + batch)
    assert rel_max(to_np(p.inverse(to_gpu(flm))), OT.inverse(flm, L, spin)) <= TOL64
    if L <= 96:
        f = synth.signal_gaussian((batch, L, 2 * L - 1), seed=2 * L)
        assert rel_max(to_np(p.forward(to_gpu(f))), OT.forward(f, L, spin)) <= TOL64
    else:
        back = to_np(p.forward(p.inverse(to_gpu(flm))))
        assert rel_max(back, flm) <= TOL64


@pytest.mark.parametrize("L,spin", [(3, 0), (16, -2), (40, 1)])
def test_precompute_adjoints_match_oracle(L, spin):
    p = pplan(L, spin, max_batch=2)
    y = synth.signal_gaussian((2, L, 2 * L - 1), seed=L)
    assert rel_max(to_np(p.adjoint_inverse(to_gpu(y))), OT.adjoint_inverse(y, L, spin)) <= TOL64
    c = synth.flm_gaussian(L, spin, 2, seed=L + 1)
    assert rel_max(to_np(p.adjoint_forward(to_gpu(c))), OT.adjoint_forward(c, L, spin)) <= TOL64


@pytest.mark.parametrize("L,N", [(8, 3), (13, 4)])
def test_precompute_wigner_matches_oracle(L, N):
    p = pplan(L, N=N, max_batch=2)
    flmn = synth.flmn_gaussian(L, N, 2, seed=L)
    assert rel_max(to_np(p.inverse(to_gpu(flmn))), OT.wigner_inverse(flmn, L, N)) <= TOL64
    f = synth.signal_gaussian((2, 2 * N - 1, L, 2 * L - 1), seed=L + 5)
    assert rel_max(to_np(p.forward(to_gpu(f))), OT.wigner_forward(f, L, N)) <= TOL64


@pytest.mark.parametrize("L", [5, 64])
def test_precompute_real_matches_oracle(L):
    p = pplan(L, real=True, max_batch=2)
    a = synth.flm_real_gaussian(L, 2, seed=L)
    assert rel_max(to_np(p.inverse(to_gpu(a))), OT.inverse_real(a, L)) <= TOL64
    g = synth.signal_real_gaussian((2, L, 2 * L - 1), seed=L + 1)
    assert rel_max(to_np(p.forward(to_gpu(g))), OT.forward_real(g, L)) <= TOL64


@pytest.mark.parametrize("L,spin,B", [(1024, 2, 4), (2048, 0, 1)])
def test_precompute_full_size_against_oracle_and_on_the_fly(L, spin, B):
    from paper_2311_14670_gb300 import Plan
    p, q = pplan(L, spin, max_batch=B), Plan(L, spin=spin, max_batch=B)
    nbytes = 8 * L * sum(L - max(abs(m), abs(spin)) for m in range(-(L - 1), L)
                         if (spin != 0 or m >= 0) and max(abs(m), abs(spin)) < L)
    assert p.device_bytes() >= nbytes > q.device_bytes()
    flm = synth.flm_gaussian(L, spin, B, seed=L, ell_power=1.0)
    x = to_gpu(flm)
    f = p.inverse(x)
    rings = [0, 1, L // 2, L - 2, L - 1]
    assert rel_max(to_np(f)[:, rings], OT.inverse(flm, L, spin, rings=rings)) <= TOL64
    assert rel_max(to_np(f), to_np(q.inverse(x))) <= TOL64
    back = p.forward(f)
    assert rel_max(to_np(back), flm) <= TOL64
    assert rel_max(to_np(back), to_np(q.forward(f))) <= TOL64


def test_precompute_order_sharding_is_bitwise():
    from paper_2311_14670_gb300.multigpu import order_ranges, sharded_forward, sharded_inverse
    L, world = 100, 3
    p = pplan(L, 2)
    x = to_gpu(synth.flm_gaussian(L, 2, 1, seed=8))
    f = p.inverse(x)
    ranges = order_ranges(L, world, 2)
    for fn, inp, ref in ((sharded_inverse, x, f), (sharded_forward, f, p.forward(f))):
        parts = []

        def gather(t):
            parts.append(t.clone())
            return parts + [torch.zeros_like(t)] * (world - len(parts))

        outs = [fn(p, inp, ranges, r, gather) for r in range(world)]
        assert torch.equal(outs[-1], ref)
