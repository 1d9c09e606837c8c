"""ctypes binding of libs2gb.so: argument marshalling only.

Every function here has the name of the C entry point in ``include/s2gb.h`` without the
``s2gb_`` prefix and passes its arguments straight through.  Data arguments are CUDA tensors
(their ``data_ptr()`` is passed), ``stream`` defaults to PyTorch's current stream on the plan's
device.  A negative return code raises ``S2GBError``.  There is no fallback: if the library is
missing, importing any transform raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libs2gb.so")

S2GB_OK = 0
S2GB_EINVAL = -1
S2GB_EUNSUPPORTED = -2
S2GB_ENOMEM = -3
S2GB_ECUDA = -4
S2GB_ECUFFT = -5
S2GB_EWORKSPACE = -6
S2GB_MW = 0
S2GB_MWSS = 1
S2GB_DH = 2
S2GB_FP64 = 0
S2GB_FP32 = 1
S2GB_PLAN_REAL = 1
S2GB_PLAN_PRECOMPUTE = 2
S2GB_PLAN_MRECURSION = 4
S2GB_PLAN_FMA_CONTRACTION = 8

_lib = None


class S2GBError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libs2gb.so (built in-tree by ``paper_2311_14670_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.s2gb_plan_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, i]
        L.s2gb_plan_create.restype = i
        L.s2gb_plan_create_real.argtypes = [ctypes.POINTER(vp), i, i, i, i, i]
        L.s2gb_plan_create_real.restype = i
        L.s2gb_plan_create_flags.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, i, ctypes.c_uint]
        L.s2gb_plan_create_flags.restype = i
        L.s2gb_plan_destroy.argtypes = [vp]
        L.s2gb_plan_destroy.restype = None
        L.s2gb_workspace_bytes.argtypes = [vp, i]
        L.s2gb_workspace_bytes.restype = sz
        L.s2gb_kernels_launched.argtypes = []
        L.s2gb_kernels_launched.restype = ctypes.c_ulonglong
        L.s2gb_plan_device_bytes.argtypes = [vp]
        L.s2gb_plan_device_bytes.restype = sz
        for name in ("s2gb_forward", "s2gb_inverse", "s2gb_adjoint_forward", "s2gb_adjoint_inverse"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp, i, vp, sz, vp]
            fn.restype = i
        L.s2gb_inverse_noalloc.argtypes = [vp, vp, vp, i, vp]
        L.s2gb_inverse_noalloc.restype = i
        for name in ("s2gb_inverse_theta", "s2gb_forward_theta"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp, i, vp]
            fn.restype = i
        L.s2gb_inverse_theta_mrange.argtypes = [vp, vp, vp, i, i, i, vp]
        L.s2gb_inverse_theta_mrange.restype = i
        L.s2gb_inverse_phi.argtypes = [vp, vp, vp, i, vp, sz, vp]
        L.s2gb_inverse_phi.restype = i
        L.s2gb_forward_mrange.argtypes = [vp, vp, vp, i, i, i, vp, sz, vp]
        L.s2gb_forward_mrange.restype = i
        L.s2gb_device_status.argtypes = [i, i]
        L.s2gb_device_status.restype = i
        L.s2gb_fma_chain.argtypes = [i, i, i, ctypes.c_longlong, vp, vp]
        L.s2gb_fma_chain.restype = i
        L.s2gb_fma_chain_lanes.argtypes = []
        L.s2gb_fma_chain_lanes.restype = i
        L.s2gb_strerror.argtypes = [i]
        L.s2gb_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().s2gb_strerror(int(code)).decode()


def _check(rc: int, where: str) -> None:
    if rc != S2GB_OK:
        raise S2GBError(rc, where)


def plan_create(L: int, spin: int, N: int, sampling: int, precision: int, max_batch: int, device: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().s2gb_plan_create(ctypes.byref(h), L, spin, N, sampling, precision, max_batch, device),
           "s2gb_plan_create")
    return h.value


def plan_create_real(L: int, sampling: int, precision: int, max_batch: int, device: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().s2gb_plan_create_real(ctypes.byref(h), L, sampling, precision, max_batch, device),
           "s2gb_plan_create_real")
    return h.value


def plan_create_flags(L: int, spin: int, N: int, sampling: int, precision: int, max_batch: int,
                      device: int, flags: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().s2gb_plan_create_flags(ctypes.byref(h), L, spin, N, sampling, precision, max_batch, device,
                                        flags), "s2gb_plan_create_flags")
    return h.value


def plan_destroy(plan: int) -> None:
    lib().s2gb_plan_destroy(ctypes.c_void_p(plan))


def workspace_bytes(plan: int, batch: int) -> int:
    return int(lib().s2gb_workspace_bytes(ctypes.c_void_p(plan), batch))


def kernels_launched() -> int:
    """Launches of this library's own kernels so far in this process (host-side counter)."""
    return int(lib().s2gb_kernels_launched())


def plan_device_bytes(plan: int) -> int:
    return int(lib().s2gb_plan_device_bytes(ctypes.c_void_p(plan)))


def _ptr(x) -> int:
    return x if isinstance(x, int) else x.data_ptr()


def _call(name: str, plan: int, src, dst, batch: int, ws, ws_bytes: int, stream: int) -> None:
    fn = getattr(lib(), "s2gb_" + name)
    _check(fn(ctypes.c_void_p(plan), ctypes.c_void_p(_ptr(src)), ctypes.c_void_p(_ptr(dst)), batch,
              ctypes.c_void_p(_ptr(ws) if ws is not None else 0), ws_bytes, ctypes.c_void_p(stream)),
           "s2gb_" + name)


def forward(plan, f, flm, batch, ws, ws_bytes, stream):
    _call("forward", plan, f, flm, batch, ws, ws_bytes, stream)


def inverse(plan, flm, f, batch, ws, ws_bytes, stream):
    _call("inverse", plan, flm, f, batch, ws, ws_bytes, stream)


def adjoint_forward(plan, flm_bar, f_bar, batch, ws, ws_bytes, stream):
    _call("adjoint_forward", plan, flm_bar, f_bar, batch, ws, ws_bytes, stream)


def adjoint_inverse(plan, f_bar, flm_bar, batch, ws, ws_bytes, stream):
    _call("adjoint_inverse", plan, f_bar, flm_bar, batch, ws, ws_bytes, stream)


def inverse_theta(plan, flm, ftilde, batch, stream):
    _check(lib().s2gb_inverse_theta(ctypes.c_void_p(plan), ctypes.c_void_p(_ptr(flm)),
                                    ctypes.c_void_p(_ptr(ftilde)), batch, ctypes.c_void_p(stream)),
           "s2gb_inverse_theta")


def forward_theta(plan, g, flm, batch, stream):
    _check(lib().s2gb_forward_theta(ctypes.c_void_p(plan), ctypes.c_void_p(_ptr(g)),
                                    ctypes.c_void_p(_ptr(flm)), batch, ctypes.c_void_p(stream)),
           "s2gb_forward_theta")


def inverse_theta_mrange(plan, flm, ftilde, batch, m_lo, m_hi, stream):
    _check(lib().s2gb_inverse_theta_mrange(ctypes.c_void_p(plan), ctypes.c_void_p(_ptr(flm)),
                                           ctypes.c_void_p(_ptr(ftilde)), batch, m_lo, m_hi,
                                           ctypes.c_void_p(stream)),
           "s2gb_inverse_theta_mrange")


def inverse_phi(plan, ftilde, f, batch, ws, ws_bytes, stream):
    _call("inverse_phi", plan, ftilde, f, batch, ws, ws_bytes, stream)


def forward_mrange(plan, f, flm, batch, m_lo, m_hi, ws, ws_bytes, stream):
    _check(lib().s2gb_forward_mrange(ctypes.c_void_p(plan), ctypes.c_void_p(_ptr(f)),
                                     ctypes.c_void_p(_ptr(flm)), batch, m_lo, m_hi,
                                     ctypes.c_void_p(_ptr(ws) if ws is not None else 0), ws_bytes,
                                     ctypes.c_void_p(stream)),
           "s2gb_forward_mrange")


def inverse_noalloc(plan, flm, f, batch, stream):
    """s2gb_inverse_noalloc: the inverse transform with the library's static scratch (no workspace)."""
    _check(lib().s2gb_inverse_noalloc(ctypes.c_void_p(plan), ctypes.c_void_p(_ptr(flm)),
                                      ctypes.c_void_p(_ptr(f)), batch, ctypes.c_void_p(stream)),
           "s2gb_inverse_noalloc")


def fma_chain(precision, blocks, threads, iters, out, stream):
    """s2gb_fma_chain: one launch of independent FMA chains (the FMA pipe's measured peak)."""
    _check(lib().s2gb_fma_chain(precision, blocks, threads, iters, ctypes.c_void_p(_ptr(out)),
                                ctypes.c_void_p(stream)), "s2gb_fma_chain")


def fma_chain_lanes():
    """Independent FMA chains per thread of s2gb_fma_chain."""
    return lib().s2gb_fma_chain_lanes()


def device_status(device, clear=True):
    """s2gb_device_status: 0, or the code of a tensor-core kernel whose bounded wait ran out."""
    rc = lib().s2gb_device_status(int(device), 1 if clear else 0)
    if rc < 0:
        raise S2GBError(rc, "s2gb_device_status")
    return rc
