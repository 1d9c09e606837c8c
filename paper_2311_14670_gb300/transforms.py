"""PyTorch-facing wrappers of libs2gb.so: plans, transforms on CUDA tensors, autograd.

Tensors are CUDA tensors laid out as in ``include/s2gb.h``, with (R, P) the rings and phi samples
of the sampling -- (L, 2L-1) for "mw", (L+1, 2L) for "mwss", (2L, 2L-1) for "dh":
  sphere:  f of shape (batch, R, P), flm of shape (batch, L, 2L-1), complex
  Wigner:  f of shape (batch, 2N-1, R, P), flmn of shape (batch, 2N-1, L, 2L-1), complex
  real signals (``real=True``, spin 0; "mw" and "dh"): f real of shape (batch, R, P), flm complex
           of shape (batch, L, L) holding the orders m >= 0
complex128 / float64 for ``precision="fp64"`` plans, complex64 / float32 for ``"fp32"``.  Every call enqueues on
PyTorch's current stream of the plan's device.  The autograd functions use the hand-written adjoint
transforms for the backward pass (Sec. 5.2), which recompute the Wigner d-functions instead of
storing anything.
"""
from __future__ import annotations

import threading

import torch

from . import _native as nat

_PRECISIONS = {"fp64": (nat.S2GB_FP64, torch.complex128), "fp32": (nat.S2GB_FP32, torch.complex64)}
_SAMPLINGS = {"mw": nat.S2GB_MW, "mwss": nat.S2GB_MWSS, "dh": nat.S2GB_DH}


def sampling_shape(L: int, sampling: str) -> tuple:
    """(rings R, phi samples P) of a sampling scheme (Sec. 4.2)."""
    return {"mw": (L, 2 * L - 1), "mwss": (L + 1, 2 * L), "dh": (2 * L, 2 * L - 1)}[sampling]


_REAL_OF = {torch.complex128: torch.float64, torch.complex64: torch.float32}


class Plan:
    """A transform plan (``s2gb_plan_create``) plus a per-batch-size workspace cache.

    Calls that take no ``ws`` share the cached workspace of their batch size, so they must not
    overlap on the device: calls on one stream are fine, and concurrent streams pass a workspace
    each (``ws=torch.empty(plan.workspace_bytes(batch), dtype=torch.uint8, device=...)``)."""

    def __init__(self, L: int, spin: int = 0, N: int = 0, precision: str = "fp64", max_batch: int = 1,
                 device: int | torch.device | None = None, sampling: str = "mw", real: bool = False,
                 precompute: bool = False, mrecursion: bool = False, fma_contraction: bool = False):
        if sampling not in _SAMPLINGS:
            raise ValueError(f"sampling must be one of {list(_SAMPLINGS)}")
        if precision not in _PRECISIONS:
            raise ValueError(f"precision must be one of {list(_PRECISIONS)}")
        if device is None:
            device = torch.cuda.current_device()
        if isinstance(device, torch.device):
            device = device.index if device.index is not None else torch.cuda.current_device()
        self.L, self.spin, self.N, self.precision, self.max_batch = int(L), int(spin), int(N), precision, int(max_batch)
        self.device = torch.device("cuda", int(device))
        self.dtype = _PRECISIONS[precision][1]          # coefficients (and complex signals)
        self.real = bool(real)
        self.precompute = bool(precompute)
        self.mrecursion = bool(mrecursion)      # theta stages by the paper's recursion over m
        # float64 on-the-fly plans contract on the tensor cores unless this asks for the FMA pipe
        self.fma_contraction = bool(fma_contraction)
        self.sampling = sampling
        self.R, self.P = sampling_shape(self.L, sampling)
        if self.real and (self.spin != 0 or self.N != 0):
            raise ValueError("real-signal plans are spin-0 sphere transforms (spin = 0, N = 0)")
        flags = ((nat.S2GB_PLAN_REAL if self.real else 0) | (nat.S2GB_PLAN_PRECOMPUTE if self.precompute else 0)
                 | (nat.S2GB_PLAN_MRECURSION if self.mrecursion else 0)
                 | (nat.S2GB_PLAN_FMA_CONTRACTION if self.fma_contraction else 0))
        self._h = nat.plan_create_flags(self.L, self.spin, self.N, _SAMPLINGS[sampling], _PRECISIONS[precision][0],
                                        self.max_batch, int(device), flags)
        self.signal_dtype = _REAL_OF[self.dtype] if self.real else self.dtype
        self._ws = {}
        self._lock = threading.Lock()

    # ---------------------------------------------------------------- shapes
    @property
    def wigner(self) -> bool:
        return self.N >= 1

    @property
    def paired(self) -> bool:
        """The theta kernels pair the columns (m, n) and (-m, -n) (one recursion for both, by
        d^l_{-m,-n} = (-1)^{m-n} d^l_{m,n}): complex spin-0 sphere plans and Wigner plans."""
        return not self.real and (self.wigner or self.spin == 0)

    def shape(self, batch: int) -> tuple:
        """Shape of f."""
        return (batch, 2 * self.N - 1, self.R, self.P) if self.wigner else (batch, self.R, self.P)

    def coef_shape(self, batch: int) -> tuple:
        """Shape of flm."""
        T = 2 * self.L - 1
        if self.real:
            return (batch, self.L, self.L)
        return (batch, 2 * self.N - 1, self.L, T) if self.wigner else (batch, self.L, T)

    def spectra_shape(self, batch: int) -> tuple:
        """Shape of the theta stage's ring spectra ftilde[b][t][k] (k = m mod P; real: k = m)."""
        return (batch, self.R, self.L if self.real else self.P)

    def _spec(self, kind: str):
        if kind == "signal":
            return self.shape, self.signal_dtype
        if kind == "spectra":
            return self.spectra_shape, self.dtype
        return self.coef_shape, self.dtype

    def workspace_bytes(self, batch: int) -> int:
        return nat.workspace_bytes(self._h, batch)

    def device_bytes(self) -> int:
        return nat.plan_device_bytes(self._h)

    def workspace(self, batch: int) -> torch.Tensor:
        with self._lock:
            ws = self._ws.get(batch)
            if ws is None:
                ws = torch.empty(self.workspace_bytes(batch), dtype=torch.uint8, device=self.device)
                self._ws[batch] = ws
            return ws

    def _check(self, x: torch.Tensor, name: str, kind: str = "coef") -> int:
        shape_of, dtype = self._spec(kind)
        if not isinstance(x, torch.Tensor) or x.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if x.dtype != dtype:
            raise TypeError(f"{name} must have dtype {dtype}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        batch = x.shape[0] if x.dim() == len(shape_of(1)) else None
        if batch is None or tuple(x.shape) != shape_of(batch):
            raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {shape_of(batch or 1)}")
        if not 1 <= batch <= self.max_batch:
            raise ValueError(f"batch {batch} outside [1, {self.max_batch}]")
        return batch

    def _out(self, out, batch: int, kind: str):
        shape_of, dtype = self._spec(kind)
        if out is None:
            return torch.empty(shape_of(batch), dtype=dtype, device=self.device)
        if self._check(out, "out", kind) != batch:
            raise ValueError("out must have the batch size of the input")
        return out

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _run(self, name: str, x: torch.Tensor, out: torch.Tensor | None, ws: torch.Tensor | None,
             src: str, dst: str):
        batch = self._check(x, "input", src)
        out = self._out(out, batch, dst)
        if ws is None:
            ws = self.workspace(batch)
        getattr(nat, name)(self._h, x, out, batch, ws, ws.numel(), self._stream())
        return out

    # ---------------------------------------------------------------- transforms (no autograd)
    def forward(self, f, out=None, ws=None):
        """Forward transform f -> flm (s2gb_forward)."""
        return self._run("forward", f, out, ws, "signal", "coef")

    def inverse(self, flm, out=None, ws=None):
        """Inverse transform flm -> f (s2gb_inverse)."""
        return self._run("inverse", flm, out, ws, "coef", "signal")

    def adjoint_forward(self, flm_bar, out=None, ws=None):
        return self._run("adjoint_forward", flm_bar, out, ws, "coef", "signal")

    def adjoint_inverse(self, f_bar, out=None, ws=None):
        return self._run("adjoint_inverse", f_bar, out, ws, "signal", "coef")

    def inverse_theta(self, flm, out=None):
        """Theta stage of the inverse alone (s2gb_inverse_theta): ring spectra ftilde[b][t][k],
        k = m mod P (real plans: k = m >= 0)."""
        return self.inverse_theta_mrange(flm, 0, self.L, out=out)

    def inverse_theta_mrange(self, flm, m_lo: int, m_hi: int, out=None):
        """Theta stage of the inverse for the orders with |m| in [m_lo, m_hi)
        (s2gb_inverse_theta_mrange); columns of other orders in ``out`` are left as they are."""
        batch = self._check(flm, "flm")
        out = self._out(out, batch, "spectra")
        nat.inverse_theta_mrange(self._h, flm, out, batch, int(m_lo), int(m_hi), self._stream())
        return out

    def inverse_phi(self, ftilde, out=None, ws=None):
        """The phi stage of the sphere inverse: ring spectra -> f (s2gb_inverse_phi)."""
        return self._run("inverse_phi", ftilde, out, ws, "spectra", "signal")

    def forward_mrange(self, f, m_lo: int, m_hi: int, out=None, ws=None):
        """Forward transform whose theta stage covers the orders with |m| in [m_lo, m_hi) only
        (s2gb_forward_mrange); flm entries of other orders in ``out`` are left as they are."""
        batch = self._check(f, "f", "signal")
        out = self._out(out, batch, "coef")
        if ws is None:
            ws = self.workspace(batch)
        nat.forward_mrange(self._h, f, out, batch, int(m_lo), int(m_hi), ws, ws.numel(), self._stream())
        return out

    def forward_theta(self, g, out=None):
        """Theta stage of the forward alone (s2gb_forward_theta): g[b][r][t] -> flm, r = m + L - 1
        (real plans: r = m >= 0), t < R rings."""
        rows = self.L if self.real else 2 * self.L - 1
        if g.dim() != 3 or tuple(g.shape[1:]) != (rows, self.R):
            raise ValueError(f"g must have shape (batch, {rows}, {self.R})")
        if g.dtype != self.dtype or g.device != self.device or not g.is_contiguous():
            raise ValueError("g must be a contiguous tensor of the plan's dtype and device")
        batch = g.shape[0]
        out = self._out(out, batch, "coef")
        nat.forward_theta(self._h, g, out, batch, self._stream())
        return out

    def graphed(self, steps, batch: int) -> "GraphedTransform":
        """The transforms ``steps`` (names of Plan methods, e.g. ["inverse", "forward"], each
        feeding the next) on ``batch`` signals, captured once into a CUDA graph; see
        GraphedTransform."""
        return GraphedTransform(self, list(steps), int(batch))

    def close(self):
        if getattr(self, "_h", None):
            nat.plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_KINDS = {"forward": ("signal", "coef"), "inverse": ("coef", "signal"),
          "adjoint_forward": ("coef", "signal"), "adjoint_inverse": ("signal", "coef")}


class GraphedTransform:
    """A chain of transforms on a fixed batch, captured into one CUDA graph and replayed.

    For small bandlimits a transform is a handful of short kernel and cuFFT launches whose launch
    overhead exceeds their run time; replaying the captured graph issues them as one graph launch.
    The input, the intermediate results, the output and the workspace are static buffers owned by
    this object: ``__call__`` copies its argument into the input buffer, replays, and returns the
    output buffer (overwritten by the next call).  The transforms run once before capture (so the
    library's one-time kernel settings are made outside the capture).  Replays do not advance the
    library's launch counter (``launches_per_replay`` holds the count taken at capture).
    """

    def __init__(self, plan: Plan, steps, batch: int):
        if not steps or any(st not in _KINDS for st in steps):
            raise ValueError(f"steps must be names among {list(_KINDS)}")
        for a, b in zip(steps, steps[1:]):
            if _KINDS[a][1] != _KINDS[b][0]:
                raise ValueError(f"{a} produces a {_KINDS[a][1]} array, {b} takes a {_KINDS[b][0]} array")
        if not 1 <= batch <= plan.max_batch:
            raise ValueError(f"batch {batch} outside [1, {plan.max_batch}]")
        self.plan, self.steps, self.batch = plan, steps, batch

        def buf(kind):
            shape_of, dtype = plan._spec(kind)
            return torch.zeros(shape_of(batch), dtype=dtype, device=plan.device)

        self.bufs = [buf(_KINDS[steps[0]][0])] + [buf(_KINDS[st][1]) for st in steps]
        self.ws = torch.empty(plan.workspace_bytes(batch), dtype=torch.uint8, device=plan.device)
        side = torch.cuda.Stream(plan.device)
        side.wait_stream(torch.cuda.current_stream(plan.device))
        with torch.cuda.stream(side):
            self._run()                               # outside the capture: one-time settings
        torch.cuda.synchronize(plan.device)
        k0 = nat.kernels_launched()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            self._run()
        self.launches_per_replay = nat.kernels_launched() - k0
        torch.cuda.synchronize(plan.device)

    def _run(self):
        for i, st in enumerate(self.steps):
            getattr(self.plan, st)(self.bufs[i], out=self.bufs[i + 1], ws=self.ws)

    @property
    def input(self) -> torch.Tensor:
        return self.bufs[0]

    @property
    def output(self) -> torch.Tensor:
        return self.bufs[-1]

    def replay(self) -> torch.Tensor:
        """Replay on the current stream with the input buffer as it is."""
        self.graph.replay()
        return self.bufs[-1]

    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        self.bufs[0].copy_(x)
        return self.replay()


class _Forward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, plan):
        ctx.plan = plan
        return plan.forward(f.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint_forward(g.contiguous()), None


class _Inverse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, flm, plan):
        ctx.plan = plan
        return plan.inverse(flm.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint_inverse(g.contiguous()), None


def forward(f: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable forward transform; its backward is the adjoint forward transform."""
    return _Forward.apply(f, plan)


def inverse(flm: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable inverse transform; its backward is the adjoint inverse transform."""
    return _Inverse.apply(flm, plan)
