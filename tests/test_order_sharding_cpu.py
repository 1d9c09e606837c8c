"""Order (|m|) sharding of one transform: the host logic (balanced ranges, column ownership, the
all-gather exchange and the assembly), checked on CPU with two gloo ranks.  Each rank's theta
stage is played by the oracle restricted to its orders, so what is tested here is only the
splitting and the exchange; the GPU test of the same path is in test_gpu_sharding.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2311_14670_gb300.multigpu import column_owner, order_ranges, order_work  # noqa: E402


@pytest.mark.parametrize("L,world,n_abs", [(1, 1, 0), (2, 2, 0), (7, 2, 0), (64, 3, 2), (1024, 8, 0), (5, 8, 0)])
def test_order_ranges_cover_and_balance(L, world, n_abs):
    ranges = order_ranges(L, world, n_abs)
    assert len(ranges) == world and ranges[0][0] == 0 and ranges[-1][1] == L
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert a <= b == c <= d                                   # contiguous, disjoint, ordered
    work = order_work(L, n_abs)
    loads = [sum(work[a:b]) for a, b in ranges]
    assert sum(loads) == sum(work) == sum(L - max(abs(m), n_abs) for m in range(-(L - 1), L)
                                           if L > max(abs(m), n_abs))
    if L >= world:
        # every cut is within one order's work of the ideal split
        assert max(loads) - sum(work) / world <= max(work)


def test_real_signal_ranges_and_owner():
    L, world = 50, 4
    ranges = order_ranges(L, world, real=True)
    work = order_work(L, real=True)
    assert sum(work) == L * (L + 1) // 2
    loads = [sum(work[a:b]) for a, b in ranges]
    assert max(loads) - sum(work) / world <= max(work)
    owner = column_owner(L, ranges, "real")
    assert len(owner) == L and owner == sorted(owner)


def test_column_owner_layouts():
    L, ranges = 4, [(0, 2), (2, 4)]                 # rank 0: m in {0, +-1}; rank 1: m in {+-2, +-3}
    T = 2 * L - 1
    assert column_owner(L, ranges, "centered") == [1, 1, 0, 0, 0, 1, 1]          # m = -3 .. 3
    mod = column_owner(L, ranges, "mod")                                          # k = m mod T
    assert [mod[m % T] for m in range(-3, 4)] == [1, 1, 0, 0, 0, 1, 1]
    with pytest.raises(ValueError):
        column_owner(L, [(0, 2)], "mod")
    # MWSS ring spectra: P = 2L columns, k = m mod 2L; the column k = L has no order (rank 0)
    ss = column_owner(L, ranges, "mod", 2 * L)
    assert len(ss) == 2 * L and ss[L] == 0
    assert [ss[m % (2 * L)] for m in range(-3, 4)] == [1, 1, 0, 0, 0, 1, 1]


class _OraclePlan:
    """Stands in for a Plan on CPU: the theta stage and the phi stage from the oracle, restricted to
    the orders asked for, with the Plan's layouts."""

    def __init__(self, L, spin):
        self.L, self.spin = L, spin
        self.dtype = torch.complex128

    def coef_shape(self, batch):
        return (batch, self.L, 2 * self.L - 1)

    def spectra_shape(self, batch):
        return (batch, self.L, 2 * self.L - 1)

    def _mask(self, lo, hi):
        m = np.arange(-(self.L - 1), self.L)
        return (np.abs(m) >= lo) & (np.abs(m) < hi)

    def inverse_theta_mrange(self, flm, lo, hi, out):
        from oracle import transforms as OT
        from oracle.sampling import mw_thetas
        L, T = self.L, 2 * self.L - 1
        ref = OT._theta_inverse(flm.numpy(), L, -self.spin, OT.ell_factor(L, self.spin), mw_thetas(L))
        keep = self._mask(lo, hi)
        for c in np.nonzero(keep)[0]:
            m = c - (L - 1)
            out[..., m % T] = torch.from_numpy(np.ascontiguousarray(ref[..., c]))
        return out

    def inverse_phi(self, ft):
        return torch.from_numpy((2 * self.L - 1) * np.fft.ifft(ft.numpy(), axis=-1))

    def forward_mrange(self, f, lo, hi, out):
        from oracle import transforms as OT
        ref = torch.from_numpy(OT.forward(f.numpy(), self.L, self.spin))
        keep = torch.from_numpy(self._mask(lo, hi))
        out[..., keep] = ref[..., keep]
        return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2311_14670_gb300 import synth
        from paper_2311_14670_gb300.multigpu import all_gather_fn, sharded_forward, sharded_inverse
        L, spin = 9, 1
        plan = _OraclePlan(L, spin)
        ranges = order_ranges(L, world, abs(spin))
        flm = torch.from_numpy(synth.flm_gaussian(L, spin, 2, seed=11))
        f = torch.from_numpy(synth.signal_gaussian((2, L, 2 * L - 1), seed=12))
        gather = all_gather_fn()
        inv = sharded_inverse(plan, flm, ranges, rank, gather)
        fwd = sharded_forward(plan, f, ranges, rank, gather)
        q.put((rank, ranges, inv.numpy(), fwd.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_order_sharded_transforms():
    from oracle import transforms as OT
    from paper_2311_14670_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in range(world)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    L, spin = 9, 1
    assert res[0][1] == res[1][1] and res[0][1][0][1] not in (0, L)        # both ranks have orders
    flm = synth.flm_gaussian(L, spin, 2, seed=11)
    f = synth.signal_gaussian((2, L, 2 * L - 1), seed=12)
    ref_inv, ref_fwd = OT.inverse(flm, L, spin), OT.forward(f, L, spin)
    for _, _, inv, fwd in res:
        assert np.abs(inv - ref_inv).max() <= 1e-12 * np.abs(ref_inv).max()
        assert np.array_equal(fwd, ref_fwd)          # assembled by copying: every bit kept
