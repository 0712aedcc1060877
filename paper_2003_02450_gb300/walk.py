"""A small object API over the C ABI, shaped like the paper's walk classes
(Section 4: `LQSW`, `GQSW`, and the GQSW with vertex subspaces for the
non-moralising walk): build the operator once, set an initial state, then
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


class _Walk:
    """What every walk object shares: one operator handle and its state dimension."""

    def _init(self, ctx: Context | None, precision: str, omega: float):
        self.ctx = ctx or Context()
        self.precision = precision
        self.omega = omega
        self.rho0 = None
        self.last_stats: dict = {}

    def _info(self):
        info = _c.qsw_op_info(self.ctx.handle, self.op)
        self.n_tilde = info["n_tilde"]
        self.n = info["n"]
        self.nnz = info["nnz"]
        self.norms = info["norms"]

    @property
    def _dev(self):
        return torch.device("cuda", self.ctx.device)

    def set_omega(self, omega: float) -> None:
        _c.qsw_set_omega(self.ctx.handle, self.op, omega)
        self._info()
        self.omega = omega

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

    def survival_time(self, t_end: float, q: int, sink: int, rho0: torch.Tensor | None = None):
        """Expected survival time: Simpson over 1 - p_sink on q + 1 times of [0, t_end]."""
        rho0 = self.rho0 if rho0 is None else rho0
        if rho0 is None:
            raise ValueError("no initial state")
        eta, self.last_stats = _c.qsw_survival_time(self.ctx.handle, self.op, rho0, t_end, q, sink)
        return eta

    def close(self):
        if getattr(self, "op", None) is not None:
            _c.qsw_op_destroy(self.op)
            self.op = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LQSW(_Walk):
    """An L-QSW on a digraph G (row = destination, column = source)."""

    def __init__(self, G, omega: float, H=None, sources=(), sinks=(), precision: str = "c128",
                 ctx: Context | None = None, operator: str = "matfree"):
        self._init(ctx, precision, omega)
        self.operator = operator
        self.op = _c.qsw_build_superoperator(self.ctx.handle, G, H, omega, sources, sinks,
                                             precision, operator)
        self._info()

    def export_csr(self):
        rowptr = torch.empty(self.n + 1, dtype=torch.int32, device=self._dev)
        col = torch.empty(max(1, self.nnz), dtype=torch.int32, device=self._dev)
        val = torch.empty(max(1, self.nnz), dtype=torch.complex128, device=self._dev)
        _c.qsw_op_export_csr(self.ctx.handle, self.op, rowptr, col, val)
        return rowptr, col[: self.nnz], val[: self.nnz]


class GQSW(_Walk):
    """A global-interaction walk (Section 2.5.2): by default the G-QSW of
    digraph G (L = G, H = Laplacian of G^u); with `Ls` (and optionally `H_rot`)
    the walk of those explicit operators on G's vertices, H required then."""

    def __init__(self, G, omega: float, H=None, Ls=None, H_rot=None, sources=(), sinks=(),
                 precision: str = "c128", ctx: Context | None = None):
        self._init(ctx, precision, omega)
        if Ls is None and H_rot is None:
            self.op = _c.qsw_build_gqsw(self.ctx.handle, G, H, omega, sources, sinks, precision)
        else:
            if H is None:
                raise ValueError("explicit Lindblad operators need an explicit H")
            n = G.n if hasattr(G, "n") else np.asarray(G).shape[0]
            self.op = _c.qsw_build_global(self.ctx.handle, n, H, list(Ls or []), H_rot, omega,
                                          sources, sinks, precision)
        self._info()


class NMGQSW(_Walk):
    """The non-moralising G-QSW of digraph G (Eq. nm_gqsw) on its demoralised
    vertex copies.  `initial_state(populations=...)` and `vertex_populations`
    work with the N original vertices (Eq. nm_rho_map); `series` returns the
    copies' populations, `series_vertices` the vertices'."""

    def __init__(self, G, omega: float, precision: str = "c128", ctx: Context | None = None):
        self._init(ctx, precision, omega)
        self.N = G.n if hasattr(G, "n") else np.asarray(G).shape[0]
        self.op = _c.qsw_build_nm_gqsw(self.ctx.handle, G, omega, precision)
        self._info()
        self.vsets = _c.qsw_nm_vsets(self.ctx.handle, self.op, self.N)

    def initial_state(self, rho0=None, populations=None) -> torch.Tensor:
        if populations is not None and len(populations) == self.N and rho0 is None:
            state = torch.empty(self.n, dtype=torch.complex128, device=self._dev)
            _c.qsw_nm_initial_state(self.ctx.handle, self.op, populations, state)
            self.rho0 = state
            return state
        return super().initial_state(rho0=rho0, populations=populations)

    def vertex_populations(self, pops_copies: torch.Tensor) -> torch.Tensor:
        pops_copies = pops_copies.reshape(-1, self.n_tilde)
        p = torch.empty((pops_copies.shape[0], self.N), dtype=torch.float64, device=self._dev)
        _c.qsw_nm_populations(self.ctx.handle, self.op, pops_copies, pops_copies.shape[0], p)
        return p

    def series_vertices(self, t0: float, dt: float, steps: int, rho0: torch.Tensor | None = None):
        _, p = self.series(t0, dt, steps, rho0, states=False, pops=True)
        return self.vertex_populations(p)


def walk_from_config(cfg: _w.WalkConfig, ctx: Context | None = None) -> LQSW:
    w = LQSW(cfg.graph, cfg.omega, sources=cfg.sources, sinks=cfg.sinks,
             precision=cfg.precision, ctx=ctx)
    w.initial_state(rho0=cfg.rho0)
    return w
