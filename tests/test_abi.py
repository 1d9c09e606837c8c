"""The C ABI library builds, loads and exports every entry point that include/s2gb.h declares.
No compute call is made (these tests run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "s2gb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(s2gb_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_14670_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["s2gb_plan_create", "s2gb_plan_destroy", "s2gb_workspace_bytes", "s2gb_forward",
              "s2gb_inverse", "s2gb_adjoint_forward", "s2gb_adjoint_inverse", "s2gb_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_argument_rejection_without_gpu(libpath):
    from paper_2311_14670_gb300 import _native as nat
    assert nat.strerror(0) == "success"
    assert nat.strerror(-6).startswith("workspace")
    assert nat.strerror(12345) == "unknown error code"
    h = ctypes.c_void_p(1)
    lib = nat.lib()
    # invalid sizes are rejected before any device is touched, and *out is cleared
    for args in [(0, 0, 0), (8, 8, 0), (8, -8, 0), (8, 0, -1), (8, 0, 9)]:
        L, spin, N = args
        assert lib.s2gb_plan_create(ctypes.byref(h), L, spin, N, 0, 0, 1, 0) == nat.S2GB_EINVAL
        assert h.value is None
    assert lib.s2gb_plan_create(ctypes.byref(h), 8, 0, 0, 7, 0, 1, 0) == nat.S2GB_EINVAL   # sampling
    assert lib.s2gb_plan_create(ctypes.byref(h), 8, 0, 0, 0, 9, 1, 0) == nat.S2GB_EINVAL   # precision
    assert lib.s2gb_plan_create(ctypes.byref(h), 8, 0, 0, 0, 0, 0, 0) == nat.S2GB_EINVAL   # max_batch
    assert lib.s2gb_plan_create(None, 8, 0, 0, 0, 0, 1, 0) == nat.S2GB_EINVAL
    # max_batch x (2N-1) x rows beyond the 32-bit FFT batch counts: refused before any device work
    assert lib.s2gb_plan_create(ctypes.byref(h), 1024, 0, 0, 0, 0, 1 << 21, 0) == nat.S2GB_EUNSUPPORTED
    assert h.value is None
    assert lib.s2gb_plan_create(ctypes.byref(h), 64, 0, 32, 2, 0, 1 << 19, 0) == nat.S2GB_EUNSUPPORTED
    # null plans
    assert lib.s2gb_workspace_bytes(None, 1) == 0
    assert lib.s2gb_forward(None, None, None, 1, None, 0, None) == nat.S2GB_EINVAL
    lib.s2gb_plan_destroy(None)


def test_kernel_launch_counter_starts_at_zero_without_gpu(libpath):
    from paper_2311_14670_gb300 import _native as nat
    n = nat.kernels_launched()
    assert isinstance(n, int) and n >= 0
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert n == 0                       # nothing in the CPU suite launches a kernel


def test_plan_flags_are_checked_before_any_device_work(libpath):
    from paper_2311_14670_gb300 import _native as nat
    lib = nat.lib()
    h = ctypes.c_void_p(1)
    # unknown flag bits, a real plan with spin or N, precompute in FP32 or above L = 2048
    assert lib.s2gb_plan_create_flags(ctypes.byref(h), 8, 0, 0, 0, 0, 1, 0, 8) == nat.S2GB_EINVAL
    assert h.value is None
    assert lib.s2gb_plan_create_flags(ctypes.byref(h), 8, 1, 0, 0, 0, 1, 0, nat.S2GB_PLAN_REAL) == nat.S2GB_EINVAL
    assert lib.s2gb_plan_create_flags(ctypes.byref(h), 8, 0, 2, 0, 0, 1, 0, nat.S2GB_PLAN_REAL) == nat.S2GB_EINVAL
    assert lib.s2gb_plan_create_flags(ctypes.byref(h), 8, 0, 0, 0, nat.S2GB_FP32, 1, 0,
                                      nat.S2GB_PLAN_PRECOMPUTE) == nat.S2GB_EUNSUPPORTED
    assert lib.s2gb_plan_create_flags(ctypes.byref(h), 4096, 0, 0, 0, 0, 1, 0,
                                      nat.S2GB_PLAN_PRECOMPUTE) == nat.S2GB_EUNSUPPORTED
    assert h.value is None


def test_build_rebuilds_objects_of_another_host_architecture(tmp_path, libpath):
    from paper_2311_14670_gb300 import build
    assert build._stamp_matches()                      # written by the build of this host
    other = tmp_path / "host"
    other.write_text("some-other-machine\n")
    assert not build._stamp_matches(str(other))
    assert not build._stamp_matches(str(tmp_path / "missing"))


def test_fma_chain_rejects_bad_sizes_without_gpu(libpath):
    """The peak-measurement helper checks its launch shape before touching a device."""
    from paper_2311_14670_gb300 import _native as nat
    lib = nat.lib()
    buf = ctypes.c_void_p(16)
    assert lib.s2gb_fma_chain_lanes() >= 1
    for prec, blocks, threads, iters, out in [(0, 0, 256, 10, buf), (0, 4, 300, 10, buf), (0, 4, 48, 10, buf),
                                              (1, 4, 256, 0, buf), (0, 4, 256, 10, None), (7, 4, 256, 10, buf)]:
        assert lib.s2gb_fma_chain(prec, blocks, threads, iters, out, None) == nat.S2GB_EINVAL
