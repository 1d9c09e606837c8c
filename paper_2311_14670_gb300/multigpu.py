"""Host-side logic of multi-GPU runs: one process per GPU.

Two ways to split work over ranks:
  * whole batches (independent signals; weak scaling, no collective on the data path) -- what
    bench.py times; torch.distributed only lines the ranks up and takes the maximum time;
  * one transform split by order |m| (Sec. 4.4: for a fixed m the theta stage couples degrees and
    rings, never orders).  Each rank runs the theta stage for its contiguous range of |m|, chosen
    so that the number of (l, m) pairs is balanced; the inverse then exchanges the ring spectra
    (one all-gather) before the phi DFT, the forward gathers the coefficients of every range.
    Each rank computes, for its orders, the bits the whole transform computes, and the assembly
    only copies, so the result is bitwise that of the unsharded transform.
"""
from __future__ import annotations

import os


def world_info() -> tuple:
    """(world_size, rank, local_rank) from the torchrun environment (defaults: one process)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, world: int, rank: int) -> range:
    """Contiguous, balanced share of n_items for rank (sizes differ by at most one)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic inputs: distinct per rank, reproducible."""
    return base * 1000 + rank


def max_over_ranks(values, device=None):
    """Elementwise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def weak_scaling_throughput(units_per_rank: int, world: int, ms_max: float, steps: int) -> float:
    """Whole-job units per second: every rank's units divided by the slowest rank's time."""
    return units_per_rank * world * steps / (ms_max * 1e-3)


# ---------------------------------------------------------------------------- order sharding
def order_work(L: int, n_abs: int = 0, real: bool = False) -> list:
    """Theta-stage work of each |m| = a: the (l, +-m) pairs with max(a, |n|) <= l < L (real
    signals: the order m = a alone)."""
    return [max(0, L - max(a, n_abs)) * (1 if (a == 0 or real) else 2) for a in range(L)]


def order_ranges(L: int, world: int, n_abs: int = 0, real: bool = False) -> list:
    """Contiguous |m| ranges [lo, hi), one per rank, covering [0, L) with balanced work (the cut
    after the prefix of work closest to k/world of the total).  A rank may get an empty range
    when world > L."""
    work = order_work(L, n_abs, real)
    total = float(sum(work))
    cuts = [0]
    acc, a = 0.0, 0
    for k in range(1, world):
        target = total * k / world
        while a < L and acc + work[a] / 2.0 <= target:
            acc += work[a]
            a += 1
        cuts.append(max(a, cuts[-1]))
    cuts.append(L)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def column_owner(L: int, ranges, layout: str, P: int | None = None) -> list:
    """Rank owning each column: layout "mod" (P columns, k = m mod P: ring spectra, P = 2L-1 by
    default; on MWSS P = 2L and the column k = L, which no order owns and every rank writes as 0,
    goes to rank 0), "centered" (2L-1 columns, m + L - 1: coefficients) or "real" (L columns,
    m >= 0: both arrays of real-signal plans)."""
    T = 2 * L - 1
    P = T if P is None else P
    owner = [-1] * (L if layout == "real" else (P if layout == "mod" else T))
    for r, (lo, hi) in enumerate(ranges):
        for a in range(lo, hi):
            if layout == "real":
                owner[a] = r
                continue
            for m in ((0,) if a == 0 else (a, -a)):
                owner[(m % P) if layout == "mod" else m + L - 1] = r
    if layout == "mod" and P > T and owner[L] < 0:
        owner[L] = 0
    if min(owner) < 0:
        raise ValueError("the ranges do not cover every order")
    return owner


def assemble_columns(parts, owner):
    """Copy every column (last axis) from the rank that owns it: out[..., k] = parts[owner[k]][..., k]."""
    import torch

    own = torch.as_tensor(owner, device=parts[0].device)
    out = parts[0].clone()
    for r in range(1, len(parts)):
        sel = (own == r).nonzero().flatten()
        if sel.numel():
            out.index_copy_(-1, sel, parts[r].index_select(-1, sel))
    return out


def all_gather_fn(group=None):
    """x -> [x of rank 0, ..., x of rank W-1] through torch.distributed (complex tensors go as
    their real views)."""
    import torch
    import torch.distributed as dist

    def gather(x):
        xr = torch.view_as_real(x) if x.is_complex() else x
        bufs = [torch.empty_like(xr) for _ in range(dist.get_world_size(group))]
        dist.all_gather(bufs, xr.contiguous(), group=group)
        return [torch.view_as_complex(b) if x.is_complex() else b for b in bufs]

    return gather


def sharded_inverse(plan, flm, ranges, rank: int, gather):
    """Inverse transform split by order: the theta stage of this rank's |m| range, the exchange
    of ring spectra, then the phi stage (every rank ends with the whole f)."""
    import torch

    lo, hi = ranges[rank]
    ft = torch.zeros(plan.spectra_shape(flm.shape[0]), dtype=flm.dtype, device=flm.device)
    plan.inverse_theta_mrange(flm, lo, hi, out=ft)
    real = getattr(plan, "real", False)
    ft = assemble_columns(gather(ft), column_owner(plan.L, ranges, "real" if real else "mod", ft.shape[-1]))
    return plan.inverse_phi(ft)


def sharded_forward(plan, f, ranges, rank: int, gather):
    """Forward transform split by order: this rank's |m| range of the theta stage, then the
    coefficients of every range gathered (every rank ends with the whole flm)."""
    import torch

    lo, hi = ranges[rank]
    flm = torch.zeros(plan.coef_shape(f.shape[0]), dtype=plan.dtype, device=f.device)
    plan.forward_mrange(f, lo, hi, out=flm)
    real = getattr(plan, "real", False)
    return assemble_columns(gather(flm), column_owner(plan.L, ranges, "real" if real else "centered"))
