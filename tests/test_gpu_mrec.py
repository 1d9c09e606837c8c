"""Parity of the theta stages built on the paper's recursion over the order m (plan flag
S2GB_PLAN_MRECURSION, Sec. 3.3) with the CPU oracle and with the default degree-recursion path.

Bar (float64): relative max error max|gpu - oracle| / max|oracle| <= 1e-12 on the same seeded
inputs, as for the default path.  Every element at small L (all three samplings, spins of both
signs, Wigner), the adjoints against the oracle's dense conjugate transposes, sampled rings and
degrees at the full-size workloads, and agreement with the degree recursion.
"""
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


def plan(L, spin=0, N=0, max_batch=1, sampling="mw", mrec=True):
    from paper_2311_14670_gb300 import Plan
    return Plan(L, spin=spin, N=N, max_batch=max_batch, sampling=sampling, mrecursion=mrec)


CASES = [(1, 0), (2, 0), (2, 1), (3, -2), (16, 0), (17, 3), (33, -1), (64, 2), (70, 0), (130, -1)]


@pytest.mark.parametrize("sampling", ["mw", "mwss", "dh"])
@pytest.mark.parametrize("L,spin", CASES)
def test_inverse_and_forward_match_oracle(sampling, L, spin):
    batch = 3
    p = plan(L, spin, max_batch=batch, sampling=sampling)
    flm = synth.flm_gaussian(L, spin, batch, seed=2000 + L)
    got = to_np(p.inverse(to_gpu(flm)))
    assert rel_max(got, OT.inverse_s(flm, L, spin, sampling)) <= TOL64
    if L <= 70:
        R, P = OT.sampling_shape(L, sampling)
        f = synth.signal_gaussian((batch, R, P), seed=2100 + L)
        assert rel_max(to_np(p.forward(to_gpu(f))), OT.forward_s(f, L, spin, sampling)) <= TOL64


@pytest.mark.parametrize("L,spin,batch", [(8, 0, 1), (31, 1, 2), (200, -2, 4), (256, 0, 2)])
def test_round_trip(L, spin, batch):
    p = plan(L, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=2200 + L)
    assert rel_max(to_np(p.forward(p.inverse(to_gpu(flm)))), flm) <= TOL64


@pytest.mark.parametrize("sampling", ["mw", "dh"])
@pytest.mark.parametrize("L,spin", [(2, 0), (4, 1), (5, -2)])
def test_adjoints_match_dense_oracle(sampling, L, spin):
    p = plan(L, spin, sampling=sampling)
    R, P = OT.sampling_shape(L, sampling)
    y = synth.signal_gaussian((R, P), seed=L + 5)
    ref = OT.adjoint_dense(lambda x: OT.inverse_s(x, L, spin, sampling), (L, 2 * L - 1), y)
    ref = np.where(OT.coeff_mask(L, -spin), ref, 0)
    assert rel_max(to_np(p.adjoint_inverse(to_gpu(y[None])))[0], ref) <= TOL64
    c = synth.flm_gaussian(L, spin, 1, seed=L + 6)[0]
    ref = OT.adjoint_dense(lambda x: OT.forward_s(x, L, spin, sampling), (R, P), c)
    assert rel_max(to_np(p.adjoint_forward(to_gpu(c[None])))[0], ref) <= TOL64


@pytest.mark.parametrize("L,N", [(4, 1), (8, 3), (13, 4)])
def test_wigner_matches_oracle(L, N):
    batch = 2
    p = plan(L, N=N, max_batch=batch)
    flmn = synth.flmn_gaussian(L, N, batch, seed=2300 + L)
    assert rel_max(to_np(p.inverse(to_gpu(flmn))), OT.wigner_inverse(flmn, L, N)) <= TOL64
    f = synth.signal_gaussian((batch, 2 * N - 1, L, 2 * L - 1), seed=2400 + L)
    assert rel_max(to_np(p.forward(to_gpu(f))), OT.wigner_forward(f, L, N)) <= TOL64


@pytest.mark.parametrize("L,spin,batch,rings", [
    (1024, 2, 4, [0, 1, 2, 100, 511, 512, 900, 1021, 1022, 1023]),
    (2048, 0, 1, [0, 1, 1023, 2046, 2047]),
])
def test_full_size_sampled_rings_and_agreement_with_degree_recursion(L, spin, batch, rings):
    pm = plan(L, spin, max_batch=batch)
    pl = plan(L, spin, max_batch=batch, mrec=False)
    flm = synth.flm_gaussian(L, spin, batch, seed=2500 + L, ell_power=1.0 if spin else 0.0)
    x = to_gpu(flm)
    f = pm.inverse(x)
    assert rel_max(to_np(f[:, rings]), OT.inverse(flm, L, spin, rings=rings)) <= TOL64
    assert rel_max(to_np(f), to_np(pl.inverse(x))) <= TOL64
    back = pm.forward(f)
    assert rel_max(to_np(back), flm) <= TOL64
    assert rel_max(to_np(back), to_np(pl.forward(f))) <= TOL64


def test_refused_combinations():
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat
    for kw in ({"precision": "fp32"}, {"real": True}, {"precompute": True}):
        with pytest.raises(nat.S2GBError) as e:
            Plan(16, mrecursion=True, **kw)
        assert e.value.code == nat.S2GB_EUNSUPPORTED
    p = plan(16, 1)
    with pytest.raises(nat.S2GBError):
        p.inverse_theta(to_gpu(synth.flm_gaussian(16, 1, 1, seed=1)))
