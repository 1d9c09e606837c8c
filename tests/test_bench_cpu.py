"""bench.py's host-side contract, without a GPU: the reference arm (the oracle timed on host cores)
prints one JSON line with the contract's keys, and the helpers count algorithmic work and read
the profiled traffic as stated."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "l64s0b1", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "l64s0b1"
    # the same config dict as the GPU arm's line, so that the two lines describe one workload
    import bench
    assert d["config"] == bench.workload_config("l64s0b1", 1)
    # ms_per_step is the measured wall time of a step, which fits inside the run
    assert d["ms_per_step"] * d["steps"] <= 1e3 * d["wall_s"] + 10.0


def test_algorithmic_flops_and_traffic_lookup():
    import bench
    # (L^2 - n^2) R (5 + 4B): L = 1024, spin 2, R = L, B = 4
    assert bench.algorithmic_flops(1024, [-2], 1024, 4) == (1024 ** 2 - 4) * 1024 * 21
    # real signals: orders m >= 0, L (L + 1) / 2 pairs
    assert bench.algorithmic_flops(8, [0], 8, 1, real=True) == 36 * 8 * 9
    # paired plans (spin 0): one recursion per (m, -m) pair, (L^2 + L) / 2 chains per ring
    L = 2048
    assert bench.algorithmic_flops(L, [0], L, 1, paired=True) == L * (5 * (L * L + L) // 2 + 4 * L * L)
    # Wigner n = -1, 0, 1: pairs sum (L^2 - n^2), chains (pairs + L) / 2
    pairs = 3 * 16 * 16 - 2
    assert bench.algorithmic_flops(16, [-1, 0, 1], 16, 2, paired=True) == 16 * (5 * ((pairs + 16) // 2) + 8 * pairs)
    assert bench.profiled_traffic("no-such-workload", "theta_forward") is None
    assert len(bench.kernel_source_hash()) == 64
    for name, (L, spin, N, B, ellp, desc) in bench.WORKLOADS.items():
        assert L >= 1 and B >= 1 and desc
