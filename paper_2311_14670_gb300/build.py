"""Build libs2gb.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled in its own nvcc process (in parallel) and the
objects are linked into ``paper_2311_14670_gb300/libs2gb.so`` against cuFFT.  No CMake, no
torch extension machinery: the library has a plain C ABI (``include/s2gb.h``).
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libs2gb.so")
SOURCES = ["api.cu", "plan.cu", "theta_kernels.cu", "theta_kernels_f32.cu", "theta_precompute.cu", "glue.cu",
           "poles.cu", "theta_mrec.cu", "peak.cu", "theta_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


STAMP = os.path.join(BUILD, "host")


def _host_tag() -> str:
    """The machine the objects are built for: objects of another host architecture are rebuilt."""
    return platform.machine()


def _stamp_matches(stamp: str = STAMP) -> bool:
    try:
        with open(stamp) as fh:
            return fh.read().strip() == _host_tag()
    except OSError:
        return False


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libs2gb.so")
    return cand


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "s2gb.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libs2gb.so."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    force = force or not _stamp_matches()
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        if force or _stale(obj, src):
            cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if verbose or ptxas_verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcufft"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed: " + " ".join(cmd))
        with open(STAMP, "w") as fh:
            fh.write(_host_tag() + "\n")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv))
