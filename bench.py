#!/usr/bin/env python3
"""Benchmark of the MW spin-s spherical-harmonic transform on GB300 (one JSON line on stdout).

A step is one pass of the whole transform path over one batch: the inverse transform of B signals
(theta-stage kernel + phi inverse DFT) followed by the forward transform of the result (phi DFT,
theta torus extension and quadrature FFTs, theta-stage kernel).  Default workload: L = 1024,
spin 2, batch 4, float64, coefficients complex Gaussian / (l+1) -- 2B = 8 transforms per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) shard independent batches over the ranks with no
collective on the data path (weak scaling); the barrier and the max-over-ranks timing use NCCL.
``--impl reference`` times the CPU oracle (plain numpy, test infrastructure) on bounded samples of
the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# The CPU oracle legs run single-threaded so that the reported core count is exact.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (L, spin, N, batch, ell_power, description)
    "l1024s2b4": (1024, 2, 0, 4, 1.0, "spin-2 SHT round trip, L=1024, MW 1024x2047, batch 4, FP64"),
    "l2048s0b1": (2048, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=2048, MW 2048x4095, batch 1, FP64"),
    "l2048s0b4": (2048, 0, 0, 4, 0.0, "spin-0 SHT round trip, L=2048, MW 2048x4095, batch 4, FP64"),
    "l64s0b1": (64, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=64, MW 64x127, batch 1, FP64"),
    "l64s0b1graph": (64, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=64, MW 64x127, batch 1, FP64, the round "
                     "trip captured once into a CUDA graph and replayed"),
    "l4096s0b1": (4096, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=4096, MW 4096x8191, batch 1, FP64"),
    "l8192s0b1": (8192, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=8192, MW 8192x16383, batch 1, FP64"),
    "wigner256n8": (256, 0, 8, 1, 0.0, "Wigner round trip, L=256, N=8, MW 256x511x15, batch 1, FP64"),
    "l2048realb1": (2048, 0, 0, 1, 0.0, "real-signal SHT round trip (orders m >= 0), L=2048, MW 2048x4095, "
                    "batch 1, FP64"),
    "l1024realb4": (1024, 0, 0, 4, 1.0, "real-signal SHT round trip (orders m >= 0), L=1024, MW 1024x2047, "
                    "batch 4, FP64"),
    "l1024s2b4pre": (1024, 2, 0, 4, 1.0, "spin-2 SHT round trip, L=1024, batch 4, FP64, precompute mode "
                     "(d-table 8.6 GB in HBM)"),
    "l1024s0b1pre": (1024, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=1024, batch 1, FP64, precompute mode "
                     "(d-table 4.3 GB in HBM)"),
    "l2048s0b1pre": (2048, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=2048, batch 1, FP64, precompute mode "
                     "(d-table 34 GB in HBM)"),
    "l2048realb1pre": (2048, 0, 0, 1, 0.0, "real-signal SHT round trip, L=2048, batch 1, FP64, precompute "
                       "mode (d-table 34 GB in HBM)"),
    "l2048s0b16f32grad": (2048, 0, 0, 16, 1.0, "differentiable FP32 SHT, L=2048, spin 0, batch 16: "
                          "loss = sum |inverse(flm) - target|^2 and its gradient via the adjoint"),
    "l1024s0b1dh": (1024, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=1024, DH 2048x2047, batch 1, FP64"),
    "l2048s0b1dh": (2048, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=2048, DH 4096x4095, batch 1, FP64"),
    "l1024s0b1mwss": (1024, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=1024, MWSS 1025x2048, batch 1, FP64"),
    "l2048s0b1mwss": (2048, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=2048, MWSS 2049x4096, batch 1, FP64"),
    "l1024s2b4dh": (1024, 2, 0, 4, 1.0, "spin-2 SHT round trip, L=1024, DH 2048x2047, batch 4, FP64"),
    "l1024s2b4mrec": (1024, 2, 0, 4, 1.0, "spin-2 SHT round trip, L=1024, MW, batch 4, FP64, theta stages by "
                      "the paper's recursion over the order m"),
    "l2048s0b1mrec": (2048, 0, 0, 1, 0.0, "spin-0 SHT round trip, L=2048, MW, batch 1, FP64, theta stages by "
                      "the paper's recursion over the order m"),
    "l2048s2b1mrec": (2048, 2, 0, 1, 0.0, "spin-2 SHT round trip, L=2048, MW, batch 1, FP64, theta stages by "
                      "the paper's recursion over the order m"),
    "l2048s2b1": (2048, 2, 0, 1, 0.0, "spin-2 SHT round trip, L=2048, MW 2048x4095, batch 1, FP64"),
    "l1024s0b4f32": (1024, 0, 0, 4, 1.0, "spin-0 SHT round trip, L=1024, MW 1024x2047, batch 4, FP32 mixed "
                     "precision (float64 starting values)"),
    "l1024s0b16f32": (1024, 0, 0, 16, 1.0, "spin-0 SHT round trip, L=1024, MW 1024x2047, batch 16, FP32 mixed "
                      "precision (float64 starting values)"),
}
PRECISION = {"l2048s0b16f32grad": "fp32", "l1024s0b4f32": "fp32", "l1024s0b16f32": "fp32"}
REAL = {"l2048realb1", "l1024realb4", "l2048realb1pre"}
PRECOMPUTE = {"l1024s2b4pre", "l1024s0b1pre", "l2048s0b1pre", "l2048realb1pre"}
GRAD = {"l2048s0b16f32grad"}
MREC = {"l1024s2b4mrec", "l2048s0b1mrec", "l2048s2b1mrec"}
GRAPH = {"l64s0b1graph"}
SAMPLING = {"l1024s0b1dh": "dh", "l2048s0b1dh": "dh", "l1024s0b1mwss": "mwss", "l2048s0b1mwss": "mwss",
            "l1024s2b4dh": "dh"}
METRIC = "transforms/sec"
# nominal FMA lanes per SM per clock (GB300), for the nominal peak printed beside the measured one
FP64_LANES_PER_SM_CLK = 2
FP32_LANES_PER_SM_CLK = 128


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "theta_traffic.json")
KERNEL_SOURCES = ["theta_kernels.cu", "theta_common.cuh", "s2gb_internal.h", "dd.cuh", "theta_tc.cu",
                  "tc_common.cuh"]


def kernel_source_hash() -> str:
    """sha256 over the sources of the float64 theta kernels (ties profiled counters to a version)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2311_14670_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, if it was taken on this
    workload with the current kernel sources; otherwise None."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("workload") != workload or rec.get("source_sha256") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch", {}).get(kernel)


def algorithmic_flops(L: int, n_list, R: int, batch: int, real: bool = False, paired: bool = False) -> float:
    """Per launch of one theta kernel: every element (l, m, theta) costs 4B flops of contraction
    (a real d times B complex values, FMA = 2) and every recursion chain 5 flops per step.  Real
    signals have the orders m >= 0 only, L (L + 1) / 2 pairs (l, m).  Paired plans (spin-0 sphere
    and Wigner: d^l_{-m,-n} = (-1)^{m-n} d^l_{m,n}) run one recursion for the columns (m, n) and
    (-m, -n), so the recursion is counted once per pair: (P + L00) / 2 chains per ring, L00 = L
    self-paired (l, 0, 0) elements when n = 0 is in the plan."""
    pairs = L * (L + 1) // 2 if real else sum(L * L - n * n for n in n_list)
    chains = (pairs + (L if 0 in n_list else 0)) // 2 if paired else pairs
    return float(R) * (5.0 * chains + 4.0 * batch * pairs)


def recursion_flops(L: int, n_list, R: int, real: bool = False, paired: bool = False) -> float:
    """Per launch of one theta kernel: the recursion alone, 5 flops (FMA = 2) per chain step.
    With the contraction on the tensor cores this is the work left to the float64 pipe."""
    pairs = L * (L + 1) // 2 if real else sum(L * L - n * n for n in n_list)
    chains = (pairs + (L if 0 in n_list else 0)) // 2 if paired else pairs
    return float(R) * 5.0 * chains


def measured_fma_peak(precision: str, dev) -> dict:
    """The FMA pipe's throughput on this GPU, measured with the library's FMA-chain kernel
    (s2gb_fma_chain: independent chains, 4 CTAs of 256 threads per SM): best of three launches of
    about 20 ms, CUDA events on the launching stream."""
    import torch

    from paper_2311_14670_gb300 import _native as nat
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 4 * sms, 256
    f64 = precision == "fp64"
    iters = 10_000 if f64 else 400_000
    out = torch.empty(blocks * threads, dtype=torch.float64 if f64 else torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    prec = nat.S2GB_FP64 if f64 else nat.S2GB_FP32
    flops = 2.0 * blocks * threads * nat.fma_chain_lanes() * iters
    nat.fma_chain(prec, blocks, threads, iters, out, stream.cuda_stream)
    best = None
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nat.fma_chain(prec, blocks, threads, iters, out, stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return {"tflops": flops / (best * 1e-3) / 1e12, "ms": best, "sms": sms,
            "how": f"s2gb_fma_chain: {blocks} CTAs x {threads} threads x {nat.fma_chain_lanes()} independent "
                   f"{precision.upper()} FMA chains x {iters} steps, best of 3 launches (CUDA events)"}


def workload_config(workload: str, world: int) -> dict:
    """The `config` of a bench line: the same dict for the GPU arm and the oracle (reference) arm."""
    L, spin, N, B, ellp, desc = WORKLOADS[workload]
    nN = 2 * N - 1 if N else 1
    cols = L if workload in REAL else 2 * L - 1
    es = 8 if PRECISION.get(workload, "fp64") == "fp32" else 16
    coef_mb = B * nN * L * cols * es / 1e6
    l2 = (f"inputs larger than L2: {coef_mb:.0f} MB of coefficients and as many of samples per step "
          "(no flush between steps)" if coef_mb > 129 else
          f"working set fits in L2 ({coef_mb:.2f} MB of coefficients per step; latency-bound size, not flushed)")
    return {"workload": workload, "description": desc, "L": L, "spin": spin, "N": N,
            "sampling": SAMPLING.get(workload, "mw"), "batch_per_gpu": B, "transforms_per_step": 2 * B * world * nN,
            "step": ("loss forward (inverse) + backward (adjoint inverse) of the batch" if workload in GRAD
                     else "inverse + forward of every signal in the batch"),
            "l2": l2, "parallelism": f"dp{world} (independent batches, no data-path collective)"}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[2:6]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    from paper_2311_14670_gb300.multigpu import world_info
    return world_info()


def run_ours(args, world, rank, local):
    import torch

    from paper_2311_14670_gb300 import Plan, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    L, spin, N, B, ellp, desc = WORKLOADS[args.workload]
    precision = PRECISION.get(args.workload, "fp64")
    grad_mode = args.workload in GRAD
    real = args.workload in REAL
    tp0 = time.perf_counter()
    sampling = SAMPLING.get(args.workload, "mw")
    plan = Plan(L, spin=spin, N=N, max_batch=B, device=local, precision=precision, real=real,
                precompute=args.workload in PRECOMPUTE, sampling=sampling, mrecursion=args.workload in MREC)
    torch.cuda.synchronize(dev)
    plan_ms = (time.perf_counter() - tp0) * 1e3
    cdt = plan.dtype
    from paper_2311_14670_gb300.multigpu import max_over_ranks, rank_seed, weak_scaling_throughput
    if N:
        coef = synth.flmn_gaussian(L, N, B, seed=rank_seed(3, rank))
        n_list = list(range(-(N - 1), N))
    elif real:
        coef = synth.flm_real_gaussian(L, B, seed=rank_seed(2, rank), ell_power=ellp)
        n_list = [0]
    else:
        coef = synth.flm_gaussian(L, spin, B, seed=rank_seed(2, rank), ell_power=0.0 if grad_mode else ellp)
        n_list = [-spin]
    x = torch.from_numpy(coef).to(dev).to(cdt)
    f = torch.empty(plan.shape(B), dtype=plan.signal_dtype, device=dev)
    y = torch.empty_like(x)
    ws = plan.workspace(B)
    stream = torch.cuda.current_stream(dev)
    if grad_mode:
        from paper_2311_14670_gb300 import inverse as inverse_ad
        # Gaussian random-field target: a_lm ~ sqrt(C_l) (N(0,1) + i N(0,1)), C_l = (l+1)^-2
        a = synth.flm_gaussian(L, spin, B, seed=4242 + rank, ell_power=ellp)
        target = plan.inverse(torch.from_numpy(a).to(dev).to(cdt))
        xg = x.clone().requires_grad_(True)

        def step():
            xg.grad = None
            loss = ((inverse_ad(xg, plan) - target).abs() ** 2).sum()
            loss.backward()
            y.copy_(xg.grad)
    elif args.workload in GRAPH:
        gr = plan.graphed(["inverse", "forward"], B)
        gr.input.copy_(x)

        def step():
            gr.replay()
            y.copy_(gr.output)
    else:
        def step():
            plan.inverse(x, out=f, ws=ws)
            plan.forward(f, out=y, ws=ws)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    from paper_2311_14670_gb300 import _native
    with ClockSampler(local) as clocks:
        k0 = _native.kernels_launched()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        k1 = _native.kernels_launched()
        barrier()
    ms = e0.elapsed_time(e1)
    err = None if grad_mode else float((y - x).abs().max() / x.abs().max())
    # the three figures of the round-trip error: relative max (above), relative RMS, mean |diff|
    err_rms = None if grad_mode else float(torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x))
    err_mean = None if grad_mode else float((y - x).abs().mean())

    # end to end through the public API: pinned host input -> device -> step -> host result, every
    # step.  The transforms run on the launch stream; the copies run on a second stream with two
    # buffers each way, so that the input of step k+1 and the result of step k move while step k
    # computes (every copy still lies between the two timing events).
    hx = x.detach().cpu().pin_memory()
    hy = [torch.empty_like(hx).pin_memory() for _ in range(2)]
    cstream = torch.cuda.Stream(dev)
    xin = [torch.empty_like(x) for _ in range(2)]
    yout = [torch.empty_like(y) for _ in range(2)]
    in_ready = [torch.cuda.Event() for _ in range(2)]
    in_free = [torch.cuda.Event() for _ in range(2)]
    out_ready = [torch.cuda.Event() for _ in range(2)]
    out_free = [torch.cuda.Event() for _ in range(2)]

    def h2d(slot):
        with torch.cuda.stream(cstream):
            cstream.wait_event(in_free[slot])
            xin[slot].copy_(hx, non_blocking=True)
            in_ready[slot].record(cstream)

    def e2e_run(nsteps, start):
        for e in in_free + out_free:
            e.record(stream)
        cstream.wait_event(start)
        h2d(0)
        for k in range(nsteps):
            sl = k & 1
            if k + 1 < nsteps:
                h2d(1 - sl)                                   # prefetch the next step's input
            stream.wait_event(in_ready[sl])
            stream.wait_event(out_free[sl])
            if grad_mode:
                with torch.no_grad():
                    xg.copy_(xin[sl])
                in_free[sl].record(stream)
                step()
                yout[sl].copy_(y)
            elif args.workload in GRAPH:
                gr.input.copy_(xin[sl])
                in_free[sl].record(stream)
                gr.replay()
                yout[sl].copy_(gr.output)
            else:
                plan.inverse(xin[sl], out=f, ws=ws)
                in_free[sl].record(stream)
                plan.forward(f, out=yout[sl], ws=ws)
            out_ready[sl].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(out_ready[sl])
                hy[sl].copy_(yout[sl], non_blocking=True)
                out_free[sl].record(cstream)
        stream.wait_stream(cstream)

    w0 = torch.cuda.Event()
    w0.record(stream)
    e2e_run(max(1, args.warmup // 2), w0)
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    e2e_run(args.steps, t0)
    t1.record(stream)
    barrier()
    ms_e2e = t0.elapsed_time(t1)
    e2e_check = float((yout[(args.steps - 1) & 1] - y).abs().max()) if not grad_mode else None

    # the theta-stage kernels alone, on the launch stream, same workload
    kern = {}
    if not N:
        R = plan.R
        g = torch.from_numpy(synth.signal_gaussian((B, L if real else 2 * L - 1, R), seed=77)).to(dev).to(cdt)
        ft = torch.empty(plan.spectra_shape(B), dtype=cdt, device=dev)
        fl = torch.empty(plan.coef_shape(B), dtype=cdt, device=dev)
        xd_ = x.detach()
        stages = [("theta_inverse", lambda: plan.inverse_theta(xd_, out=ft))]
        if R <= 2048:    # above, the forward theta stage runs in ring chunks inside forward() only
            stages.append(("theta_forward", lambda: plan.forward_theta(g, out=fl)))
        if plan.mrecursion:
            # the order-recursion theta stages write partial sums into the workspace, so they run
            # only inside the transforms: time the whole inverse and forward (the theta stage plus
            # the phi DFTs and, in the forward, the theta-direction quadrature operator)
            stages = [("inverse_transform", lambda: plan.inverse(xd_, out=f, ws=ws)),
                      ("forward_transform", lambda: plan.forward(f, out=y, ws=ws))]
        for name, fn in stages:
            fn()
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(2, args.steps)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            kms = a.elapsed_time(b) / reps
            flops = algorithmic_flops(L, n_list, R, B, real, paired=plan.paired)
            rflops = recursion_flops(L, n_list, R, real, paired=plan.paired)
            kern[name] = {"ms": kms, "flops": flops, "tflops": flops / (kms * 1e-3) / 1e12,
                          "recursion_flops": rflops, "recursion_tflops": rflops / (kms * 1e-3) / 1e12}

    # the step split into the two theta kernels and everything else (phi / theta-direction FFTs on
    # cuFFT, glue kernels): per step, from the separately timed theta kernels
    stage_split = None
    if "theta_inverse" in kern and "theta_forward" in kern:
        th = kern["theta_inverse"]["ms"] + kern["theta_forward"]["ms"]
        stage_split = {"theta_kernels_ms": round(th, 3),
                       "fft_and_glue_ms": round(max(0.0, ms / args.steps - th), 3),
                       # this GPU's transforms per second if the step were the theta kernels alone
                       "theta_stage_transforms_per_s": round(2 * B * (2 * N - 1 if N else 1) / (th * 1e-3), 3)}
    ms, ms_e2e = max_over_ranks([ms, ms_e2e], device=dev)
    # a gradient step is one inverse transform plus its adjoint: 2 transforms per signal, as a round trip
    transforms_per_step = 2 * B * world * (2 * N - 1 if N else 1)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return None
    ck = clocks.summary()
    sm_max = ck["sm_max_mhz"] or 2070.0
    lanes = FP64_LANES_PER_SM_CLK if precision == "fp64" else FP32_LANES_PER_SM_CLK
    meas = measured_fma_peak(precision, dev)
    nominal = meas["sms"] * lanes * 2 * sm_max * 1e6 / 1e12    # TFLOP/s
    peak = meas["tflops"]
    roof = None
    # float64 plans whose contraction runs on the tensor cores: the float64 pipe runs the recursion
    # only, so the roofline counts the recursion's flops against it; otherwise the whole (5 + 4B)
    tensor = precision == "fp64" and not plan.precompute and not plan.mrecursion and not plan.fma_contraction
    if kern:
        dom = max(kern, key=lambda k: kern[k]["ms"])
        ach = kern[dom]["recursion_tflops"] if tensor else kern[dom]["tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 4), "peak": round(peak, 4),
                "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                "work": ("recursion: 5 flops per (l, m, theta) chain step on the float64 pipe; the "
                         "contraction (4B flops per element) runs on the tensor cores as exact float16 "
                         "digit products" if tensor else "(5 + 4B) flops per (l, m, theta) element"),
                "algorithmic_tflops_5_plus_4B": round(kern[dom]["tflops"], 4),
                "traffic": profiled_traffic(args.workload, dom) if precision == "fp64" else None,
                "peak_basis": f"{precision.upper()} FMA pipe, measured on this GPU: {meas['how']}",
                "peak_nominal": round(nominal, 4),
                "peak_nominal_basis": f"{meas['sms']} SMs x {lanes} lanes x 2 flop x {sm_max:.0f} MHz",
                "frac_of_nominal": round(ach / nominal, 4)}
    value = weak_scaling_throughput(transforms_per_step // world, world, ms, args.steps)
    in_bytes = x.numel() * x.element_size()
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "transforms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == "fp64" else "f32 (f64 starting values)",
        "data": "synthetic (seeded complex Gaussian coefficients)",
        "config": workload_config(args.workload, world),
        "plan": {"create_ms": round(plan_ms, 1), "device_bytes": plan.device_bytes(),
                 "workspace_bytes": ws.numel()},
        "roundtrip_rel_max_err": err,
        "roundtrip_rel_rms_err": err_rms,
        "roundtrip_mean_abs_err": err_mean,
        "e2e": {"value": round(weak_scaling_throughput(transforms_per_step // world, world, ms_e2e, args.steps), 3),
                "unit": "transforms/s",
                "copies": "pinned host <-> device every step on a second stream, double-buffered, "
                          "overlapping the transforms",
                "result_max_abs_diff_vs_device_path": e2e_check,
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": in_bytes},
        # graph replays launch the captured kernels without the host-side counter: count them at capture
        "gpu_launches": (gr.launches_per_replay * args.steps if args.workload in GRAPH else k1 - k0),
        "kernels": kern,
        "stages": stage_split,
        "roofline": roof,
        "clocks": {k: ck[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    if args.workload == "l1024s2b4" and not args.no_l2048 and world == 1 and precision == "fp64":
        out["l2048"] = l2048_records(dev, peak)
        out["l2048"]["peak_tflops_measured"] = round(peak, 4)
    if not args.no_cpu_baseline and world == 1 and not grad_mode:
        out["cpu_baseline"] = cpu_baseline_parallel(args.workload, sampling, args.cpu_rings, args.cpu_procs)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def l2048_records(dev, peak_tflops: float, steps: int = 5, warmup: int = 3) -> dict:
    """The L = 2048 round trips (MW, FP64, batch 1) beside the default line: spin 2 (unpaired
    theta kernels) and spin 0 (paired).  Per configuration: the theta kernels' CUDA-event times and
    their fraction of the measured FP64 peak, and the round trip's ms / transforms per second."""
    import torch

    from paper_2311_14670_gb300 import Plan, synth
    out = {}
    stream = torch.cuda.current_stream(dev)
    for spin in (2, 0):
        L = 2048
        plan = Plan(L, spin=spin, max_batch=1, device=dev.index)
        x = torch.from_numpy(synth.flm_gaussian(L, spin, 1, seed=2048 + spin)).to(dev)
        f = torch.empty(plan.shape(1), dtype=plan.signal_dtype, device=dev)
        y = torch.empty_like(x)
        ws = plan.workspace(1)
        g = torch.from_numpy(synth.signal_gaussian((1, 2 * L - 1, L), seed=77)).to(dev)
        ft = torch.empty(plan.spectra_shape(1), dtype=plan.dtype, device=dev)
        fl = torch.empty(plan.coef_shape(1), dtype=plan.dtype, device=dev)

        def timed(fn, reps):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            return a.elapsed_time(b) / reps

        def rt():
            plan.inverse(x, out=f, ws=ws)
            plan.forward(f, out=y, ws=ws)

        ms = timed(rt, steps)
        err = float((y - x).abs().max() / x.abs().max())
        flops = algorithmic_flops(L, [-spin], L, 1, paired=plan.paired)
        rflops = recursion_flops(L, [-spin], L, paired=plan.paired)
        ti = timed(lambda: plan.inverse_theta(x, out=ft), steps)
        tf = timed(lambda: plan.forward_theta(g, out=fl), steps)
        out[f"s{spin}b1"] = {
            "roundtrip_ms": round(ms, 3), "transforms_per_s": round(2 / (ms * 1e-3), 3),
            "theta_inverse_ms": round(ti, 3), "theta_forward_ms": round(tf, 3),
            "theta_flops_per_launch": flops, "recursion_flops_per_launch": rflops, "paired": plan.paired,
            # the float64 pipe runs the recursion (the contraction is on the tensor cores)
            "frac_theta_inverse": round(rflops / (ti * 1e-3) / 1e12 / peak_tflops, 4),
            "frac_theta_forward": round(rflops / (tf * 1e-3) / 1e12 / peak_tflops, 4),
            "algorithmic_tflops_inverse": round(flops / (ti * 1e-3) / 1e12, 4),
            "algorithmic_tflops_forward": round(flops / (tf * 1e-3) / 1e12, 4),
            "roundtrip_rel_max_err": err}
        del plan, ws
        torch.cuda.empty_cache()
    return out


def run_serve(args, world, rank, local):
    """Served stream (mixed L in {128..2048}, spin in {0, 2}, forward/inverse): saturated throughput,
    then Poisson arrivals at rho x that rate; p50/p99 latency per rho.  Rank 0 only."""
    import torch

    from paper_2311_14670_gb300.serve import Server, make_requests

    if rank != 0:
        return None
    torch.cuda.set_device(local)
    precision = "fp32" if args.workload == "serve_fp32" else "fp64"
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    srv = Server(device=local, budget_bytes=args.budget_gib << 30, streams=4, max_batch=4, precision=precision)
    kinds = {(L, s) for L in (128, 256, 512, 1024, 2048) for s in (0, 2)}
    srv.warm(kinds)
    warm = make_requests(40, float("inf"), seed=1, dtype=dt)
    srv.run(warm, keep_results=False)
    sat = srv.run(make_requests(args.requests, float("inf"), seed=2, dtype=dt), keep_results=False)
    out = {"saturated": sat}
    for rho in (0.5, 0.8, 0.95):
        st = srv.run(make_requests(args.requests, rho * sat["throughput_rps"], seed=3, dtype=dt),
                     keep_results=False)
        out[f"rho_{rho}"] = st
    res = {"metric": "served transforms/sec", "value": round(sat["throughput_rps"], 3), "unit": "transforms/s",
           "n_gpus": 1, "steps": args.requests, "warmup": 40, "ms_per_step": round(1e3 / sat["throughput_rps"], 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if precision == "fp64" else "f32 (f64 starting values)",
           "data": "synthetic (seeded complex Gaussian inputs, Poisson arrivals)",
           "config": {"workload": args.workload, "requests": args.requests,
                      "mix": "L uniform {128,256,512,1024,2048}, spin uniform {0,2}, forward/inverse uniform",
                      "budget_gib": args.budget_gib, "streams": 4, "max_batch": 4},
           "serving": {k: {q: (round(v, 3) if isinstance(v, float) else v) for q, v in st.items()}
                       for k, st in out.items()}}
    return res


_SETUP_CACHE = {}


def _cached(key, fn):
    """Inputs and oracle matrices of a bounded sample, built once per process (a pool worker times
    several samples of the same workload; only the timed stages count)."""
    if key not in _SETUP_CACHE:
        _SETUP_CACHE[key] = fn()
    return _SETUP_CACHE[key]


def cpu_baseline(workload: str, rings: int = 4) -> dict:
    """The oracle (plain numpy, single thread) on a bounded sample of the workload, scaled to
    transforms/s.  The oracle's stages are timed on `rings`-sized slices and scaled by the size
    they are linear in: the inverse (d-table + synthesis) per ring; the forward's phi-DFT, torus
    extension and upsampling per order m; its quadrature against the d-table per degree l.  A
    Wigner transform is 2N-1 such stages (timed for one n) plus the gamma DFT."""
    from oracle import transforms as OT
    from paper_2311_14670_gb300 import synth

    L, spin, N, B, ellp, _ = WORKLOADS[workload]
    T = 2 * L - 1
    n = 0 if N else -spin
    nn = 2 * N - 1 if N else 1
    coef = _cached(("coef", workload), lambda: synth.flm_gaussian(L, -n, B, seed=1, ell_power=ellp))
    f = _cached(("f", workload), lambda: synth.signal_gaussian((B, L, T), seed=2))
    k = max(2, min(L, rings))
    k2 = k // 2

    def fit(fn, full):
        """Time fn(k/2) and fn(k); extrapolate t(x) = a + b x (per-call overhead + per-unit cost)."""
        t0 = time.perf_counter()
        fn(k2)
        ta = time.perf_counter() - t0
        t0 = time.perf_counter()
        fn(k)
        tb = time.perf_counter() - t0
        b = max(0.0, (tb - ta) / (k - k2))
        a = max(0.0, tb - b * k)
        return a + b * full

    scale = OT.ell_factor(L, -n)
    thetas = OT.mw_thetas(L)
    t_start = time.perf_counter()

    def inv(j):                                                # inverse: per ring
        sel = np.linspace(0, L - 1, j).astype(int)
        OT._theta_inverse(coef, L, n, scale, thetas[sel]) @ OT.phi_dft_matrix(L, +1).T

    cmat, up = _cached(("up", L), lambda: OT._upsample_matrices(L))

    def fft(j):                                                # forward DFT/upsampling: per order
        sel = np.linspace(-(L - 1), L - 1, j).astype(int)
        up @ (cmat @ OT._extend(OT._phi_forward(f, L, sel), L, n, sel))

    Gu = _cached(("Gu", workload), lambda: synth.signal_gaussian((B, 2 * L, T), seed=3))   # same shape

    def quad(j):                                               # forward quadrature: per degree
        OT._theta_forward_upsampled(Gu, L, n, scale, np.linspace(abs(n), L - 1, j).astype(int))

    t_inv = fit(inv, L)
    t_fft = fit(fft, T)
    t_quad = fit(quad, L)
    t_gam = 0.0
    if N:
        fw = synth.signal_gaussian((B, nn, L, T), seed=4)
        t0 = time.perf_counter()
        np.einsum("kn,...ktp->...ntp", OT._gamma_matrix(N, -1), fw)
        t_gam = 2 * (time.perf_counter() - t0)
    total = nn * (t_inv + t_fft + t_quad) + t_gam
    per = 2 * B * nn
    return {"value": round(per / total, 6), "unit": "transforms/s", "cores": 1, "kind": "oracle",
            "sample": f"{workload}: oracle stages timed on {k2} and {k} of {L} rings / {T} orders / {L} "
                      f"degrees (all {B} signals{', one of %d n' % nn if N else ''}), single thread, "
                      f"extrapolated as overhead + linear cost to the full round trip",
            "seconds_measured": round(time.perf_counter() - t_start, 2),
            "seconds_full_round_trip_est": round(total, 1)}


def cpu_baseline_sampled(workload: str, sampling: str, rings: int = 4) -> dict:
    """cpu_baseline for the MWSS and DH workloads (spin-s sphere transforms): the oracle's inverse
    timed per ring, its forward phi DFT (and, on MWSS, theta upsampling) per order and its
    quadrature per degree, each on two slice sizes and extrapolated as overhead + linear cost."""
    from oracle import transforms as OT
    from paper_2311_14670_gb300 import synth

    L, spin, N, B, ellp, _ = WORKLOADS[workload]
    R, P = OT.sampling_shape(L, sampling)
    T = 2 * L - 1
    coef = _cached(("coef", workload), lambda: synth.flm_gaussian(L, spin, B, seed=1, ell_power=ellp))
    f = _cached(("f", workload), lambda: synth.signal_gaussian((B, R, P), seed=2))
    k = max(2, min(L, rings))
    k2 = k // 2

    def fit(fn, full):
        t0 = time.perf_counter()
        fn(k2)
        ta = time.perf_counter() - t0
        t0 = time.perf_counter()
        fn(k)
        tb = time.perf_counter() - t0
        b = max(0.0, (tb - ta) / (k - k2))
        return max(0.0, tb - b * k) + b * full

    t_start = time.perf_counter()
    scale = OT.ell_factor(L, spin)

    def inv(j):                                                # inverse: per ring
        OT.inverse_s(coef, L, spin, sampling, rings=np.linspace(0, R - 1, j).astype(int))

    E = OT._phi_matrix(L, P, -1)
    up = cm = None
    if sampling == "mwss":
        kk = np.arange(-(L - 1), L)
        cm = OT._expi_pi(-np.outer(kk, 2 * np.arange(2 * L)), 2 * L) / (2 * L)
        up = OT._expi_pi(np.outer(np.arange(2 * L + 1), kk), 2 * L)

    def dft(j):                                                # phi DFT (+ upsampling): per order
        F = f @ E[:, np.linspace(0, T - 1, j).astype(int)]
        if up is not None:
            up @ (cm @ np.concatenate([F, F[..., 1:L, :]], axis=-2))

    Rq = 2 * L + 1 if sampling == "mwss" else R
    W = synth.signal_gaussian((B, Rq, T), seed=3)                # stand-in of the weighted spectra
    thq = OT.mwss_thetas(2 * L) if sampling == "mwss" else OT.dh_thetas(L)

    def quad(j):                                               # quadrature: per degree
        OT._quadrature(W, thq, L, -spin, scale, np.linspace(abs(spin), L - 1, j).astype(int))

    total = fit(inv, R) + fit(dft, T) + fit(quad, L)
    return {"value": round(2 * B / total, 6), "unit": "transforms/s", "cores": 1, "kind": "oracle",
            "sample": f"{workload}: oracle stages timed on {k2} and {k} of {R} rings / {T} orders / {L} "
                      f"degrees (all {B} signals), single thread, extrapolated as overhead + linear cost",
            "seconds_measured": round(time.perf_counter() - t_start, 2),
            "seconds_full_round_trip_est": round(total, 1)}


def _baseline_task(args) -> dict:
    """One single-threaded oracle sample in a pool worker (spawned: no CUDA state)."""
    workload, sampling, rings = args
    try:
        return (cpu_baseline_sampled(workload, sampling, rings=rings) if sampling != "mw"
                else cpu_baseline(workload, rings=rings))
    except Exception as exc:   # reported to the parent, which raises
        return {"error": repr(exc)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """`procs` spawned single-threaded oracle processes, kept for several samples.  One sample: every
    process times the same bounded slice of the workload concurrently and extrapolates its own full
    round trip under the others' load; the throughputs add up (independent transforms, one per
    core).  The GPU arm's cpu_baseline is one such sample; each step of the reference arm is one."""

    def __init__(self, procs: int):
        import multiprocessing as mp
        self.procs = max(1, procs)
        self.pool = mp.get_context("spawn").Pool(self.procs) if self.procs > 1 else None

    def sample(self, workload: str, sampling: str, rings: int) -> dict:
        task = (workload, sampling, rings)
        res = self.pool.map(_baseline_task, [task] * self.procs, chunksize=1) if self.pool else [_baseline_task(task)]
        bad = [r["error"] for r in res if "error" in r]
        if bad:
            raise RuntimeError(f"oracle baseline process failed: {bad[0]}")
        total = sum(r["value"] for r in res)
        return {"value": round(total, 6), "unit": res[0]["unit"], "cores": self.procs, "kind": "oracle",
                "sample": f"{self.procs} concurrent single-threaded oracle processes, one per host core; each: "
                          + res[0]["sample"],
                "per_process_value": round(total / self.procs, 6),
                "seconds_measured": max(r["seconds_measured"] for r in res),
                "seconds_full_round_trip_est": round(statistics.median(r["seconds_full_round_trip_est"] for r in res), 1)}

    def close(self):
        if self.pool:
            self.pool.close()
            self.pool.join()


def cpu_baseline_parallel(workload: str, sampling: str, rings: int, procs: int) -> dict:
    """cpu_baseline on all host cores: one OraclePool sample."""
    pool = OraclePool(procs)
    try:
        return pool.sample(workload, sampling, rings)
    finally:
        pool.close()


def run_reference(args, world, rank):
    """The oracle arm: each step is one OraclePool sample of the workload (the same procedure as the
    GPU arm's cpu_baseline).  `value` is the median over the timed steps of the extrapolated
    transforms/s; `ms_per_step` is the measured wall time of a step (a bounded sample, not a whole
    round trip), and the extrapolated time of a whole step is reported beside it."""
    if rank != 0:
        return None
    L, spin, N, B, ellp, desc = WORKLOADS[args.workload]
    sampling = SAMPLING.get(args.workload, "mw")
    pool = OraclePool(args.cpu_procs)
    try:
        for _ in range(args.warmup):
            pool.sample(args.workload, sampling, args.cpu_rings)
        samples, walls = [], []
        last = None
        for _ in range(args.steps):
            t0 = time.perf_counter()
            last = pool.sample(args.workload, sampling, args.cpu_rings)
            walls.append(time.perf_counter() - t0)
            samples.append(last["value"])
    finally:
        pool.close()
    value = statistics.median(samples)
    cfg = workload_config(args.workload, world)
    per = cfg["transforms_per_step"]
    cb = {"value": value, "unit": "transforms/s", "cores": pool.procs, "kind": "oracle",
          "sample": "each step: " + last["sample"]}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(walls), 3),
            "ms_per_step_basis": "measured wall time of one step (one bounded oracle sample on all host cores)",
            "ms_per_full_step_extrapolated": round(per / value * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded complex Gaussian coefficients)",
            "config": cfg, "cpu_baseline": cb, "wall_s": round(sum(walls), 3),
            "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="l1024s2b4", choices=sorted(WORKLOADS) + ["serve_fp64", "serve_fp32"])
    ap.add_argument("--requests", type=int, default=512, help="served-stream length (serve_* workloads)")
    ap.add_argument("--budget-gib", type=int, default=16, help="HBM admission budget (serve_* workloads)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l2048", action="store_true",
                    help="skip the L = 2048 records beside the default workload's line")
    ap.add_argument("--cpu-rings", type=int, default=4,
                    help="rings / orders / degrees of one oracle sample (timed at half and at this size)")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes for the CPU baseline (0: one per host core)")
    args = ap.parse_args()
    if args.cpu_procs <= 0:
        args.cpu_procs = host_cores()
    world, rank, local = dist_setup()
    if args.workload.startswith("serve_"):
        out = None if args.impl == "reference" else run_serve(args, world, rank, local)
        if args.impl == "reference" and rank == 0:
            out = {"impl": "reference", "unavailable": "the oracle has no served mode"}
    elif args.impl == "reference":
        out = run_reference(args, world, rank)
    else:
        out = run_ours(args, world, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
