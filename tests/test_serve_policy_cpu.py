"""The server's admission policy (serve.next_admission), host logic only: oldest request first,
batches of one kind up to max_batch, the HBM budget respected while anything runs, a lone
oversized batch still admitted, nothing without a free stream slot."""
import collections
from types import SimpleNamespace

from paper_2311_14670_gb300.serve import next_admission


def _pending(*reqs):
    q = collections.defaultdict(collections.deque)
    for kind, arrival in reqs:
        q[kind].append(SimpleNamespace(arrival=arrival))
    return dict(q)


def _fp(kind, batch):                      # bytes of a batch: proportional to L^2 and the batch
    return batch * kind[0] * kind[0]


def test_oldest_kind_first_and_batched_up_to_max():
    a, b = (128, 0, "inverse"), (256, 2, "forward")
    p = _pending((b, 0.5), (a, 0.1), (a, 0.2), (a, 0.3), (a, 0.9), (a, 1.0))
    assert next_admission(p, 2, 0, 0, 0, 1 << 40, 4, _fp) == (a, 4)
    assert next_admission(p, 2, 0, 0, 0, 1 << 40, 8, _fp) == (a, 5)


def test_budget_respected_while_running_and_lone_batch_admitted():
    a = (1024, 0, "inverse")
    p = _pending((a, 0.0), (a, 0.1))
    need = _fp(a, 2)
    # something runs and the batch does not fit next to it: wait
    assert next_admission(p, 1, 1, 10, 5, need + 14, 4, _fp) is None
    # it fits exactly: admit
    assert next_admission(p, 1, 1, 10, 5, need + 15, 4, _fp) == (a, 2)
    # nothing runs: admitted even beyond the budget (it runs alone)
    assert next_admission(p, 1, 0, 0, 5, 1, 4, _fp) == (a, 2)


def test_no_free_slot_or_nothing_pending():
    a = (64, 0, "forward")
    assert next_admission(_pending((a, 0.0)), 0, 3, 0, 0, 1 << 40, 4, _fp) is None
    assert next_admission({}, 4, 0, 0, 0, 1 << 40, 4, _fp) is None


def test_plan_bytes_read_after_the_footprint():
    """A kind's plan is created while its footprint is taken; the budget check must count it."""
    a = (512, 0, "inverse")
    state = {"plans": 0}

    def fp(kind, batch):
        state["plans"] = 100               # the plan of this kind now exists
        return 10

    p = _pending((a, 0.0))
    assert next_admission(p, 1, 1, 0, lambda: state["plans"], 109, 4, fp) is None
    assert next_admission(p, 1, 1, 0, lambda: state["plans"], 110, 4, fp) == (a, 1)


def test_latency_stats_overall_and_per_bandlimit():
    """Percentiles per L separate small requests from large ones (numpy percentiles on the
    latencies, overall and per group)."""
    import numpy as np

    from paper_2311_14670_gb300.serve import latency_stats
    reqs = [SimpleNamespace(L=128, latency=0.001 * (i + 1)) for i in range(10)]
    reqs += [SimpleNamespace(L=2048, latency=0.1 * (i + 1)) for i in range(4)]
    st = latency_stats(reqs)
    all_lat = np.array([r.latency for r in reqs])
    assert abs(st["p50_ms"] - np.percentile(all_lat, 50) * 1e3) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(all_lat, 99) * 1e3) < 1e-9
    assert set(st["per_L"]) == {128, 2048}
    assert st["per_L"][128]["requests"] == 10 and st["per_L"][2048]["requests"] == 4
    assert abs(st["per_L"][128]["p50_ms"] - 5.5) < 1e-9
    assert abs(st["per_L"][2048]["p99_ms"] - np.percentile([100, 200, 300, 400], 99)) < 1e-9
