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
