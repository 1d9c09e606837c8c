"""Shared helpers of the GPU parity tests (tolerances, tensor conversion)."""
import numpy as np

# float64 bar: relative max error max|gpu - ref| / max|ref|
TOL64 = 1e-12


def rel_max(got, ref) -> float:
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (den if den > 0 else 1.0))


def to_gpu(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_np(t):
    return t.detach().cpu().numpy()


def _oracle_forward_slice(args):
    from oracle import transforms as OT
    f, L, spin, ells, orders = args
    return OT.forward(f, L, spin, ells=ells, orders=orders)


def oracle_forward_parallel(f, L, spin, ells, orders=None, procs=None):
    """OT.forward on the degrees `ells` (and orders `orders`), the degrees split over spawned
    single-threaded oracle processes (the oracle's d-functions cost the same per degree whichever
    orders are kept, so whole columns at L >= 1024 need the host's cores).  Returns [b][ells][orders]."""
    import multiprocessing as mp
    import os
    ells = list(ells)
    procs = max(1, min(procs or os.cpu_count() or 1, len(ells)))
    chunks = [ells[i::procs] for i in range(procs)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        parts = pool.map(_oracle_forward_slice, [(f, L, spin, c, orders) for c in chunks])
    out = None
    for c, part in zip(chunks, parts):
        if out is None:
            out = np.empty(part.shape[:-2] + (len(ells), part.shape[-1]), dtype=part.dtype)
        for k, l in enumerate(c):
            out[..., ells.index(l), :] = part[..., k, :]
    return out
