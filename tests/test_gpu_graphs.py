"""Transforms captured into CUDA graphs (Plan.graphed) give the results of the direct calls, bit for
bit, on every replay with new inputs."""
import pytest

from gpu_helpers import to_gpu
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


@pytest.mark.parametrize("L,spin,N,sampling,precision,batch", [
    (64, 0, 0, "mw", "fp64", 1), (64, 2, 0, "mwss", "fp64", 2), (33, -1, 0, "dh", "fp32", 3),
    (16, 0, 3, "mw", "fp64", 2)])
def test_graphed_round_trip_equals_direct_calls(L, spin, N, sampling, precision, batch):
    from paper_2311_14670_gb300 import Plan
    p = Plan(L, spin=spin, N=N, max_batch=batch, sampling=sampling, precision=precision)
    g = p.graphed(["inverse", "forward"], batch)
    assert g.launches_per_replay >= 1
    for call in range(3):
        coef = (synth.flmn_gaussian(L, N, batch, seed=call) if N else
                synth.flm_gaussian(L, spin, batch, seed=call))
        x = to_gpu(coef, p.dtype)
        ref = p.forward(p.inverse(x))
        got = g(x).clone()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_graphed_adjoint_chain_and_argument_checks():
    from paper_2311_14670_gb300 import Plan
    p = Plan(40, spin=1, max_batch=2)
    g = p.graphed(["adjoint_forward", "adjoint_inverse"], 2)
    x = to_gpu(synth.flm_gaussian(40, 1, 2, seed=7))
    assert torch.equal(g(x).clone(), p.adjoint_inverse(p.adjoint_forward(x)))
    with pytest.raises(ValueError):
        p.graphed(["inverse", "inverse"], 1)
    with pytest.raises(ValueError):
        p.graphed(["forward"], 3)
