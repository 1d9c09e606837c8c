"""Multi-process (gloo, world size 2, CPU) checks of the multi-GPU host logic: balanced disjoint
shards that cover every item, distinct per-rank seeds, the max-over-ranks timing reduction and the
weak-scaling throughput.  Each rank transforms its shard with the oracle (no collective on the data
path); the results are gathered here only to verify coverage."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import transforms as OT
        from paper_2311_14670_gb300 import synth
        from paper_2311_14670_gb300.multigpu import (max_over_ranks, rank_seed, shard, weak_scaling_throughput,
                                                     world_info)
        assert world_info() == (world, rank, rank)
        items = list(shard(7, world, rank))
        L = 6
        outs = {}
        for i in items:                      # the data path: independent transforms, no collective
            flm = synth.flm_gaussian(L, 0, 1, seed=i)[0]
            outs[i] = OT.inverse(flm, L, 0)
        t = max_over_ranks([10.0 + rank, 5.0 * (1 - rank)])
        thr = weak_scaling_throughput(4, world, t[0], 3)
        gathered = [None] * world
        dist.all_gather_object(gathered, (items, rank_seed(2, rank), {k: v.tolist() for k, v in outs.items()}))
        if rank == 0:
            q.put((gathered, t, thr))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, t, thr = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [g[0] for g in gathered]
    assert sorted(sum(shards, [])) == list(range(7))          # disjoint and complete
    assert abs(len(shards[0]) - len(shards[1])) <= 1          # balanced
    assert gathered[0][1] != gathered[1][1]                   # distinct seeds
    assert t == [11.0, 5.0]                                   # elementwise max over ranks
    assert thr == pytest.approx(4 * 2 * 3 / 11e-3)
    # every item's transform equals a single-process computation
    from oracle import transforms as OT
    from paper_2311_14670_gb300 import synth
    for items, _, outs in gathered:
        for i in items:
            ref = OT.inverse(synth.flm_gaussian(6, 0, 1, seed=i)[0], 6, 0)
            assert np.allclose(np.array(outs[i]), ref, rtol=0, atol=0)
