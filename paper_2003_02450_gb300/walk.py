"""A small object API over the C ABI, shaped like the paper's `LQSW` walk
class (Section 4): build the superoperator once, set an initial state, then
`step` / `series`, and read populations.  PyTorch supplies device memory and
the CUDA stream; the computation is the library's.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qsw as _c
from . import workloads as _w


class Context:
    """A library context bound to one device and torch's current stream there."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        self.handle = _c.qsw_create(device, self.stream.cuda_stream)

    def close(self):
        if self.handle is not None:
            _c.qsw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LQSW:
    """An L-QSW on a digraph G (row = destination, column = source)."""

    def __init__(self, G, omega: float, H=None, sources=(), sinks=(), precision: str = "c128",
                 ctx: Context | None = None, operator: str = "matfree"):
        self.ctx = ctx or Context()
        self.precision = precision
        self.operator = operator
        self.op = _c.qsw_build_superoperator(self.ctx.handle, G, H, omega, sources, sinks,
                                             precision, operator)
        info = _c.qsw_op_info(self.ctx.handle, self.op)
        self.n_tilde = info["n_tilde"]
        self.n = info["n"]
        self.nnz = info["nnz"]
        self.norms = info["norms"]
        self.omega = omega
        self.rho0 = None
        self.last_stats: dict = {}

    @property
    def _dev(self):
        return torch.device("cuda", self.ctx.device)

    def set_omega(self, omega: float) -> None:
        _c.qsw_set_omega(self.ctx.handle, self.op, omega)
        info = _c.qsw_op_info(self.ctx.handle, self.op)
        self.nnz, self.norms, self.omega = info["nnz"], info["norms"], omega

    def initial_state(self, rho0=None, populations=None) -> torch.Tensor:
        state = torch.empty(self.n, dtype=torch.complex128, device=self._dev)
        _c.qsw_initial_state(self.ctx.handle, self.op, state, rho0=rho0, populations=populations)
        self.rho0 = state
        return state

    def series(self, t0: float, dt: float, steps: int, rho0: torch.Tensor | None = None,
               states: bool = True, pops: bool = True):
        rho0 = self.rho0 if rho0 is None else rho0
        if rho0 is None:
            raise ValueError("no initial state")
        out = torch.empty((steps + 1, self.n), dtype=torch.complex128, device=self._dev) if states else None
        p = torch.empty((steps + 1, self.n_tilde), dtype=torch.float64, device=self._dev) if pops else None
        self.last_stats = _c.qsw_expmv_series(self.ctx.handle, self.op, rho0, t0, dt, steps, out, p)
        return out, p

    def step(self, t: float, rho0: torch.Tensor | None = None) -> torch.Tensor:
        out, _ = self.series(t, 0.0, 0, rho0, states=True, pops=False)
        return out[0]

    def apply(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty_like(x)
        _c.qsw_apply(self.ctx.handle, self.op, x, y)
        return y

    def populations(self, states: torch.Tensor) -> torch.Tensor:
        states = states.reshape(-1, self.n)
        p = torch.empty((states.shape[0], self.n_tilde), dtype=torch.float64, device=self._dev)
        _c.qsw_populations(self.ctx.handle, self.op, states, states.shape[0], p)
        return p

    def export_csr(self):
        rowptr = torch.empty(self.n + 1, dtype=torch.int32, device=self._dev)
        col = torch.empty(max(1, self.nnz), dtype=torch.int32, device=self._dev)
        val = torch.empty(max(1, self.nnz), dtype=torch.complex128, device=self._dev)
        _c.qsw_op_export_csr(self.ctx.handle, self.op, rowptr, col, val)
        return rowptr, col[: self.nnz], val[: self.nnz]

    def close(self):
        if self.op is not None:
            _c.qsw_op_destroy(self.op)
            self.op = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def walk_from_config(cfg: _w.WalkConfig, ctx: Context | None = None) -> LQSW:
    w = LQSW(cfg.graph, cfg.omega, sources=cfg.sources, sinks=cfg.sinks,
             precision=cfg.precision, ctx=ctx)
    w.initial_state(rho0=cfg.rho0)
    return w
