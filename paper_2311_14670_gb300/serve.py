"""Continuous-batching transform server on one GPU.

Requests (forward or inverse spin-s transforms of mixed bandlimit L and spin) arrive over time.
The host loop
  * keeps one plan per (L, spin) on the device (recursion tables and starting-value data stay
    resident; a plan's memory is counted once),
  * groups waiting requests of the same kind into batches (up to ``max_batch``),
  * admits a batch only while the device memory in flight (input + output + workspace of every
    running batch, plus the resident plans) stays under ``budget_bytes``,
  * launches each admitted batch on a free stream of a small stream pool, so that batches overlap
    on the device while newer requests keep arriving and are admitted as slots and memory free up,
  * polls CUDA events (no blocking waits; an iteration that admitted, completed and received
    nothing sleeps for ``poll_s`` while batches run, or until the next arrival when the device is
    idle, so that the host loop does not hold a core at 100 %); on completion the results are in
    the requests' pinned host buffers, the latency (arrival -> result on the host) is recorded and
    memory is released.
Latency percentiles are reported over the whole stream and per bandlimit L, so that small
requests queued behind large batches are visible.
Every kernel computes each signal in the same order whatever batch it is in, so a request's result
does not depend on what it was batched with (checked by ``tests/test_gpu_serve.py``).
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import time

import numpy as np
import torch

from .transforms import Plan


@dataclasses.dataclass
class Request:
    rid: int
    L: int
    spin: int
    direction: str                 # "forward" or "inverse"
    data: torch.Tensor             # pinned host input of shape (L, 2L-1)
    arrival: float                 # seconds since the start of the run
    out: torch.Tensor | None = None   # pinned host result (filled by the server)
    t_done: float | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclasses.dataclass
class _Running:
    reqs: list
    event: torch.cuda.Event
    tensors: tuple
    footprint: int
    stream_idx: int


class _HostPool:
    """Reusable pinned host buffers keyed by (shape, dtype)."""

    def __init__(self):
        self.free = collections.defaultdict(list)

    def get(self, shape, dtype):
        lst = self.free[(tuple(shape), dtype)]
        return lst.pop() if lst else torch.empty(shape, dtype=dtype, pin_memory=True)

    def put(self, t):
        self.free[(tuple(t.shape), t.dtype)].append(t)


def next_admission(pending: dict, free_slots: int, running: int, in_flight: int, plan_bytes: int,
                   budget: int, max_batch: int, footprint):
    """The admission policy of the server loop (host logic only).

    ``pending`` maps a kind (L, spin, direction) to its queue of waiting requests (oldest first;
    each has an ``arrival`` time); ``footprint(kind, batch)`` gives the device bytes of a batch
    (input + output + workspace).  Returns (kind, batch) to launch next, or None to wait: the kind
    of the oldest waiting request, batched up to ``max_batch`` of its requests, when a stream slot
    is free and the batch fits the budget next to everything in flight and the resident plans -- or
    when nothing is running at all (a batch larger than the budget still runs, alone).
    ``plan_bytes`` may be a callable, read after ``footprint`` (which may create the kind's plan).
    """
    if not pending or free_slots <= 0:
        return None
    kind = min(pending, key=lambda k: pending[k][0].arrival)
    batch = min(len(pending[kind]), max_batch)
    fp = footprint(kind, batch)
    pb = plan_bytes() if callable(plan_bytes) else plan_bytes
    if running and in_flight + fp + pb > budget:
        return None
    return kind, batch


def latency_stats(requests) -> dict:
    """p50 / p99 / mean latency (ms) of served requests, overall and per bandlimit L."""
    lat = np.array([r.latency for r in requests])
    out = {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "per_L": {}}
    for L in sorted({r.L for r in requests}):
        sub = np.array([r.latency for r in requests if r.L == L])
        out["per_L"][int(L)] = {"requests": int(sub.size), "p50_ms": float(np.percentile(sub, 50) * 1e3),
                                "p99_ms": float(np.percentile(sub, 99) * 1e3)}
    return out


class Server:
    def __init__(self, device: int = 0, budget_bytes: int = 16 << 30, streams: int = 4,
                 max_batch: int = 4, precision: str = "fp64", poll_s: float = 50e-6):
        self.device = torch.device("cuda", device)
        self.poll_s = float(poll_s)
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.precision = precision
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.busy = [False] * streams
        self.plans: dict = {}
        self.plan_bytes = 0
        self.in_flight = 0
        self.peak_in_flight = 0
        self.launches = 0
        self.host_pool = _HostPool()

    def plan(self, L: int, spin: int) -> Plan:
        key = (L, spin)
        p = self.plans.get(key)
        if p is None:
            p = Plan(L, spin=spin, max_batch=self.max_batch, precision=self.precision, device=self.device)
            self.plans[key] = p
            self.plan_bytes += p.device_bytes()
        return p

    def footprint(self, p: Plan, batch: int) -> int:
        elem = 16 if p.dtype == torch.complex128 else 8
        return 2 * batch * p.L * (2 * p.L - 1) * elem + p.workspace_bytes(batch)

    def warm(self, kinds) -> None:
        """Create the plans of the given (L, spin) kinds before serving (plan creation allocates)."""
        for L, spin in kinds:
            self.plan(L, spin)

    def release(self, req: Request) -> None:
        """Give a consumed result buffer back to the pool."""
        if req.out is not None:
            self.host_pool.put(req.out)
            req.out = None

    def run(self, requests: list, keep_results: bool = True) -> dict:
        """Serve ``requests`` in real time (arrival times relative to the call); returns statistics
        (the latency figures are None for an empty stream)."""
        if not requests:
            return {"requests": 0, "wall_s": 0.0, "throughput_rps": 0.0, "p50_ms": None, "p99_ms": None,
                    "mean_ms": None, "launches": self.launches, "peak_in_flight_bytes": self.peak_in_flight,
                    "plan_bytes": self.plan_bytes, "budget_bytes": self.budget}
        arrivals = [(r.arrival, r.rid, r) for r in requests]
        heapq.heapify(arrivals)
        pending: dict = {}
        running: list = []
        done = 0
        n = len(requests)
        t0 = time.perf_counter()
        idle_sleeps = 0
        while done < n:
            now = time.perf_counter() - t0
            progress = False
            while arrivals and arrivals[0][0] <= now:
                _, _, r = heapq.heappop(arrivals)
                pending.setdefault((r.L, r.spin, r.direction), collections.deque()).append(r)
                progress = True
            still = []
            for job in running:
                if job.event.query():
                    t = time.perf_counter() - t0
                    for r in job.reqs:
                        r.t_done = t
                        if not keep_results:
                            self.release(r)
                    self.in_flight -= job.footprint
                    self.busy[job.stream_idx] = False
                    done += len(job.reqs)
                    progress = True
                else:
                    still.append(job)
            running = still
            while pending:
                free = [i for i, b in enumerate(self.busy) if not b]
                nxt = next_admission(pending, len(free), len(running), self.in_flight, lambda: self.plan_bytes,
                                     self.budget, self.max_batch,
                                     lambda k, b: self.footprint(self.plan(k[0], k[1]), b))
                if nxt is None:
                    break                                  # no free stream, or wait for memory
                kind, batch = nxt
                L, spin, direction = kind
                p = self.plan(L, spin)
                fp = self.footprint(p, batch)
                q = pending[kind]
                reqs = [q.popleft() for _ in range(batch)]
                if not q:
                    del pending[kind]
                running.append(self._launch(p, reqs, direction, fp, free[0]))
                progress = True
            if not progress and done < n:
                # nothing arrived, finished or started: back off instead of spinning
                wait = self.poll_s if running else max(0.0, arrivals[0][0] - now) if arrivals else self.poll_s
                time.sleep(min(wait, 0.002))
                idle_sleeps += 1
        wall = time.perf_counter() - t0
        stats = {"requests": n, "wall_s": wall, "throughput_rps": n / wall}
        stats.update(latency_stats(requests))
        stats.update({"launches": self.launches, "peak_in_flight_bytes": self.peak_in_flight,
                      "plan_bytes": self.plan_bytes, "budget_bytes": self.budget, "idle_sleeps": idle_sleeps})
        return stats

    def _launch(self, p: Plan, reqs, direction: str, fp: int, si: int) -> _Running:
        st = self.streams[si]
        self.busy[si] = True
        self.in_flight += fp
        self.peak_in_flight = max(self.peak_in_flight, self.in_flight + self.plan_bytes)
        self.launches += 1
        batch = len(reqs)
        shape = p.shape(batch)
        with torch.cuda.stream(st):
            x = torch.empty(shape, dtype=p.dtype, device=self.device)
            for i, r in enumerate(reqs):
                x[i].copy_(r.data, non_blocking=True)
            ws = torch.empty(p.workspace_bytes(batch), dtype=torch.uint8, device=self.device)
            out = torch.empty(shape, dtype=p.dtype, device=self.device)
            if direction == "inverse":
                p.inverse(x, out=out, ws=ws)
            else:
                p.forward(x, out=out, ws=ws)
            for i, r in enumerate(reqs):
                r.out = self.host_pool.get(shape[1:], p.dtype)
                r.out.copy_(out[i], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        for t in (x, ws, out):
            t.record_stream(st)
        return _Running(reqs, ev, (x, ws, out), fp, si)


def make_requests(n: int, rate: float, seed: int, Ls=(128, 256, 512, 1024, 2048), spins=(0, 2),
                  dtype=torch.complex128, distinct: int = 4) -> list:
    """Poisson arrivals at ``rate`` requests/s (rate = inf: all at t = 0); L, spin and direction
    uniform.  Inputs are complex Gaussian (coefficients restricted to l >= max(|m|, |spin|) for
    inverse requests); ``distinct`` different pinned inputs per kind are reused round-robin so that
    host memory stays bounded for long streams."""
    rng = np.random.default_rng(seed)
    inputs: dict = {}
    t = 0.0
    out = []
    for i in range(n):
        if np.isfinite(rate):
            t += rng.exponential(1.0 / rate)
        L = int(rng.choice(Ls))
        spin = int(rng.choice(spins))
        direction = "inverse" if rng.random() < 0.5 else "forward"
        key = (L, spin, direction)
        lst = inputs.setdefault(key, [])
        if len(lst) < distinct:
            a = rng.standard_normal((L, 2 * L - 1)) + 1j * rng.standard_normal((L, 2 * L - 1))
            if direction == "inverse":
                ell = np.arange(L)[:, None]
                m = np.arange(-(L - 1), L)[None, :]
                a = np.where((np.abs(m) <= ell) & (ell >= abs(spin)), a, 0)
            lst.append(torch.from_numpy(a).to(dtype).pin_memory())
            data = lst[-1]
        else:
            data = lst[i % distinct]
        out.append(Request(i, L, spin, direction, data, t))
    return out
