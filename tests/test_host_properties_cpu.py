"""Property tests (hypothesis) at random parameters, CPU only (skipped where hypothesis is not
installed): the host logic that decides how work is split and admitted -- the order ranges of a
sharded transform, the column ownership used to assemble the shards, the server's admission
policy -- and the oracle's d-functions against the Jacobi representation."""
import collections
from types import SimpleNamespace

import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from paper_2311_14670_gb300.multigpu import column_owner, order_ranges, order_work  # noqa: E402
from paper_2311_14670_gb300.serve import next_admission  # noqa: E402


@settings(max_examples=300, deadline=None)
@given(L=st.integers(1, 600), world=st.integers(1, 16), n_abs=st.integers(0, 40), real=st.booleans())
def test_order_ranges_partition_and_balance(L, world, n_abs, real):
    n_abs = 0 if real else min(n_abs, L - 1)
    ranges = order_ranges(L, world, n_abs, real)
    assert len(ranges) == world
    assert ranges[0][0] == 0 and ranges[-1][1] == L
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert a <= b == c <= d
    work = order_work(L, n_abs, real)
    loads = [sum(work[a:b]) for a, b in ranges]
    assert sum(loads) == sum(work)
    # no rank carries more than its share plus one order's work
    assert max(loads) <= sum(work) / world + max(work)


@settings(max_examples=300, deadline=None)
@given(L=st.integers(1, 300), world=st.integers(1, 8), mwss=st.booleans())
def test_every_column_has_exactly_the_owner_of_its_order(L, world, mwss):
    ranges = order_ranges(L, world)
    T = 2 * L - 1
    P = 2 * L if mwss else T
    rank_of = {}
    for r, (lo, hi) in enumerate(ranges):
        for a in range(lo, hi):
            rank_of[a] = r
    mod = column_owner(L, ranges, "mod", P)
    centred = column_owner(L, ranges, "centered")
    assert len(mod) == P and len(centred) == T
    for m in range(-(L - 1), L):
        assert mod[m % P] == rank_of[abs(m)]
        assert centred[m + L - 1] == rank_of[abs(m)]
    if mwss:
        assert mod[L] == 0                      # the column of no order
    real = column_owner(L, order_ranges(L, world, real=True), "real")
    assert real == sorted(real) and len(real) == L


_KINDS = [(L, s, d) for L in (64, 128, 256) for s in (0, 2) for d in ("forward", "inverse")]


@settings(max_examples=400, deadline=None)
@given(reqs=st.lists(st.tuples(st.sampled_from(_KINDS), st.floats(0, 100, allow_nan=False)), max_size=30),
       free=st.integers(0, 4), running=st.integers(0, 4), in_flight=st.integers(0, 10 ** 7),
       plan_bytes=st.integers(0, 10 ** 6), budget=st.integers(0, 2 * 10 ** 7), max_batch=st.integers(1, 8))
def test_admission_policy(reqs, free, running, in_flight, plan_bytes, budget, max_batch):
    pending = collections.defaultdict(collections.deque)
    for kind, t in sorted(reqs, key=lambda r: r[1]):
        pending[kind].append(SimpleNamespace(arrival=t))
    pending = dict(pending)

    def footprint(kind, batch):
        return batch * kind[0] * kind[0] * 32

    got = next_admission(pending, free, running, in_flight, plan_bytes, budget, max_batch, footprint)
    if not pending or free <= 0:
        assert got is None
        return
    oldest = min(pending, key=lambda k: pending[k][0].arrival)
    batch = min(len(pending[oldest]), max_batch)
    fits = in_flight + footprint(oldest, batch) + plan_bytes <= budget
    if running and not fits:
        assert got is None
    else:
        assert got == (oldest, batch)


@settings(max_examples=150, deadline=None)
@given(ell=st.integers(0, 60), data=st.data(),
       beta=st.floats(1e-7, 3.14159265358979 - 1e-7, allow_nan=False))
def test_oracle_d_function_matches_the_jacobi_form_anywhere(ell, data, beta):
    """The oracle's d^l_{mn}(beta) (the paper's recursion over m, two-sided) against the Jacobi
    representation in 40-digit arithmetic at random (l, m, n, beta)."""
    import numpy as np

    mpmath = pytest.importorskip("mpmath")
    from oracle.wigner import wigner_d_jacobi, wigner_d_table

    n = data.draw(st.integers(-ell, ell))
    m = data.draw(st.integers(-ell, ell))
    got = wigner_d_table([ell], n, np.array([beta], dtype=np.longdouble))[0, m + ell, 0]
    ref = float(wigner_d_jacobi(ell, m, n, mpmath.mpf(beta), dps=40))
    assert abs(got - ref) <= 1e-14
