"""The continuous-batching server: results equal the same transforms run alone (bit for bit),
admission respects the memory budget, and every request completes."""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max
from oracle import transforms as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def test_results_alone_equal_results_in_the_mix():
    from paper_2311_14670_gb300.serve import Server, make_requests
    srv = Server(device=0, budget_bytes=8 << 30, streams=3, max_batch=4)
    reqs = make_requests(48, float("inf"), seed=3, Ls=(16, 33, 64), spins=(0, 2), distinct=3)
    srv.warm({(r.L, r.spin) for r in reqs})
    stats = srv.run(reqs)
    assert stats["requests"] == 48 and all(r.t_done is not None for r in reqs)
    assert stats["launches"] < 48                      # requests were batched
    for r in reqs:
        p = srv.plan(r.L, r.spin)
        x = r.data.cuda().unsqueeze(0)
        alone = (p.inverse(x) if r.direction == "inverse" else p.forward(x))[0].cpu().numpy()
        # every kernel sums each signal in the same order whatever it is batched with: bit for bit
        assert np.array_equal(r.out.numpy(), alone)
    # and against the oracle for a few of them
    for r in reqs[:6]:
        a = r.data.numpy()
        ref = OT.inverse(a, r.L, r.spin) if r.direction == "inverse" else OT.forward(a, r.L, r.spin)
        assert rel_max(r.out.numpy(), ref) <= TOL64


def test_admission_respects_budget_and_poisson_arrivals_complete():
    from paper_2311_14670_gb300.serve import Server, make_requests
    srv = Server(device=0, budget_bytes=64 << 20, streams=4, max_batch=2)
    reqs = make_requests(30, 2000.0, seed=5, Ls=(32, 64, 128), spins=(0, 1), distinct=2)
    srv.warm({(r.L, r.spin) for r in reqs})
    stats = srv.run(reqs, keep_results=False)
    assert all(r.t_done is not None and r.t_done >= r.arrival for r in reqs)
    biggest = max(srv.footprint(srv.plan(r.L, r.spin), 1) for r in reqs)
    assert stats["peak_in_flight_bytes"] <= max(srv.budget, biggest + srv.plan_bytes)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
