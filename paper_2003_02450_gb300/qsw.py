"""ctypes binding of libqsw.so (include/qsw.h), one Python function per C entry
point with the same name.  Argument marshalling only: every step of the
computation runs in the library's CUDA kernels.  Device buffers are passed as
integer device pointers (e.g. ``torch.Tensor.data_ptr()``).

If the library has not been built the first call raises ``QswUnavailable``;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqsw.so")

QSW_C128 = 0
QSW_C64_BULK = 1
PRECISIONS = {"c128": QSW_C128, "c64": QSW_C64_BULK}
QSW_OPERATOR_MATRIX_FREE = 0
QSW_OPERATOR_CSR = 1
OPERATORS = {"matfree": QSW_OPERATOR_MATRIX_FREE, "csr": QSW_OPERATOR_CSR}

STATUS = {0: "QSW_OK", 1: "QSW_ERR_INVALID_ARG", 2: "QSW_ERR_NOT_SIMPLE",
          3: "QSW_ERR_OMEGA_RANGE", 4: "QSW_ERR_OOM", 5: "QSW_ERR_NOT_CONVERGED",
          6: "QSW_ERR_CUDA", 7: "QSW_ERR_TOO_LARGE", 8: "QSW_ERR_NOT_HERMITIAN"}


class QswUnavailable(RuntimeError):
    """libqsw.so is missing or cannot be loaded."""


class QswError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.message = message


class qsw_csr(ctypes.Structure):
    _fields_ = [("n", c_int32), ("nnz", c_int32), ("rowptr", POINTER(c_int32)),
                ("col", POINTER(c_int32)), ("w", POINTER(c_double))]


class qsw_port(ctypes.Structure):
    _fields_ = [("vertex", c_int32), ("rate", c_double)]


class qsw_series_stats(ctypes.Structure):
    _fields_ = [("m0", c_int32), ("s0", c_int32), ("m_star", c_int32), ("s", c_int32),
                ("step_m", c_int32), ("step_s", c_int32), ("outputs_per_block", c_int32),
                ("jobs", c_int32), ("matvecs", c_int64), ("bytes_per_matvec", c_double),
                ("kernel_ms", c_double), ("fupdates", c_int64), ("algorithmic_bytes", c_double),
                ("algorithmic_flops", c_double), ("hermitian", c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class qsw_zcsr(ctypes.Structure):
    _fields_ = [("n", c_int32), ("nnz", c_int32), ("rowptr", POINTER(c_int32)),
                ("col", POINTER(c_int32)), ("re", POINTER(c_double)), ("im", POINTER(c_double))]


class qsw_batch_stats(ctypes.Structure):
    _fields_ = [("walks", c_int32), ("clusters", c_int32), ("norms_ms", c_double),
                ("series_ms", c_double), ("matvecs", c_int64), ("fupdates", c_int64),
                ("small_walks", c_int32), ("algorithmic_flops", c_double),
                ("algorithmic_bytes", c_double), ("cluster_size", c_int32),
                ("small_limit", c_int32), ("tuned", c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


QSW_BUILD_DEFER_NORMS = 0x100
QSW_BUILD_FIXED_SCHEDULE = 0x200
QSW_BUILD_FP64_RANKING = 0x400
NOALLOC_SCRATCH_BYTES = 16 << 20   # QSW_NOALLOC_SCRATCH_BYTES


class qsw_server_config(ctypes.Structure):
    _fields_ = [("workers", c_int32), ("max_batch", c_int32), ("memory_budget_bytes", c_double)]


class qsw_request(ctypes.Structure):
    _fields_ = [("graph", qsw_csr), ("omega", c_double), ("precision", c_int32),
                ("rho0", c_void_p), ("populations", c_void_p), ("t0", c_double),
                ("dt", c_double), ("steps", c_int32), ("pops_out", c_void_p)]


class qsw_request_result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("latency_ms", c_double), ("queue_ms", c_double),
                ("error", ctypes.c_char * 256)]

_lib = None

_SIGNATURES = {
    "qsw_create": ([POINTER(c_void_p), c_int32, c_void_p], c_int32),
    "qsw_destroy": ([c_void_p], None),
    "qsw_last_error": ([c_void_p], ctypes.c_char_p),
    "qsw_build_superoperator": ([c_void_p, POINTER(qsw_csr), POINTER(qsw_csr), c_double,
                                 POINTER(qsw_port), c_int32, POINTER(qsw_port), c_int32, c_int32,
                                 c_int32, POINTER(c_void_p)], c_int32),
    "qsw_set_omega": ([c_void_p, c_double], c_int32),
    "qsw_op_info": ([c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64),
                     POINTER(c_double)], c_int32),
    "qsw_op_export_csr": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "qsw_op_destroy": ([c_void_p], None),
    "qsw_initial_state": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "qsw_apply": ([c_void_p, c_void_p, c_void_p], c_int32),
    "qsw_expmv_series": ([c_void_p, c_void_p, c_double, c_double, c_int32, c_void_p, c_void_p,
                          POINTER(qsw_series_stats)], c_int32),
    "qsw_expmv_series_noalloc": ([c_void_p, c_void_p, c_double, c_double, c_int32, c_void_p,
                                  c_void_p, POINTER(qsw_series_stats)], c_int32),
    "qsw_expmv_series_host": ([c_void_p, c_void_p, c_double, c_double, c_int32, c_void_p,
                               c_void_p, POINTER(qsw_series_stats)], c_int32),
    "qsw_populations": ([c_void_p, c_void_p, c_int32, c_void_p], c_int32),
    "qsw_build_global": ([c_void_p, c_int32, POINTER(qsw_zcsr), POINTER(qsw_zcsr), c_int32,
                          POINTER(qsw_zcsr), c_double, POINTER(qsw_port), c_int32,
                          POINTER(qsw_port), c_int32, c_int32, c_int32, POINTER(c_void_p)], c_int32),
    "qsw_build_gqsw": ([c_void_p, POINTER(qsw_csr), POINTER(qsw_csr), c_double, POINTER(qsw_port),
                        c_int32, POINTER(qsw_port), c_int32, c_int32, POINTER(c_void_p)], c_int32),
    "qsw_build_nm_gqsw": ([c_void_p, POINTER(qsw_csr), c_double, c_int32, POINTER(c_void_p)],
                          c_int32),
    "qsw_nm_vsets": ([c_void_p, POINTER(c_int32)], c_int32),
    "qsw_nm_populations": ([c_void_p, c_void_p, c_int32, c_void_p], c_int32),
    "qsw_nm_initial_state": ([c_void_p, POINTER(c_double), c_void_p], c_int32),
    "qsw_survival_time": ([c_void_p, c_void_p, c_double, c_int32, c_int32, POINTER(c_double),
                           c_void_p, POINTER(qsw_series_stats)], c_int32),
    "qsw_batch_survival_time": ([c_void_p, c_int32, POINTER(c_void_p), POINTER(c_void_p),
                                 POINTER(c_double), POINTER(c_int32), POINTER(c_int32),
                                 POINTER(c_double), POINTER(qsw_batch_stats)], c_int32),
    "qsw_probe_wait_limit": ([c_void_p, POINTER(c_double)], c_int32),
    "qsw_theta_table": ([c_int32, POINTER(c_double)], c_int32),
    "qsw_kernel_launches": ([], c_int64),
    "qsw_device_allocations": ([], c_int64),
    "qsw_tune_measurements": ([], c_int64),
    "qsw_tune_reset": ([], None),
    "qsw_batch_set_schedule": ([c_void_p, c_int32, c_int32], c_int32),
    "qsw_op_set_csr_schedule": ([c_void_p, c_int32, c_int32], c_int32),
    "qsw_op_schedule": ([c_void_p, POINTER(c_int32), POINTER(c_int32)], c_int32),
    "qsw_server_create": ([c_int32, POINTER(qsw_server_config), POINTER(c_void_p)], c_int32),
    "qsw_server_submit": ([c_void_p, POINTER(qsw_request), POINTER(c_int64)], c_int32),
    "qsw_server_wait": ([c_void_p, c_int64, c_double, POINTER(qsw_request_result)], c_int32),
    "qsw_server_stats": ([c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_double)], c_int32),
    "qsw_server_destroy": ([c_void_p], None),
    "qsw_batch_series": ([c_void_p, c_int32, POINTER(c_void_p), POINTER(c_void_p), c_int32,
                          POINTER(c_double), POINTER(c_double), POINTER(c_int32),
                          POINTER(c_void_p), POINTER(qsw_batch_stats)], c_int32),
    "qsw_select_params": ([POINTER(c_double), c_double, c_int32, c_int32, POINTER(c_int32),
                           POINTER(c_int32)], c_int32),
}


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QswUnavailable(f"{LIB_PATH} is not built; run `python -m "
                                 "paper_2003_02450_gb300.build`")
        try:
            handle = ctypes.CDLL(LIB_PATH)
        except OSError as exc:
            raise QswUnavailable(str(exc)) from exc
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _check(status: int, ctx=None):
    if status != 0:
        msg = lib().qsw_last_error(ctx)
        raise QswError(status, msg.decode() if msg else "")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return c_void_p(x)
    if hasattr(x, "data_ptr"):
        return c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(c_void_p)
    raise TypeError(f"cannot pass {type(x)} as a pointer")


class _Csr:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, n, rowptr, col, w):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.c = qsw_csr(int(n), int(self.col.size),
                         self.rowptr.ctypes.data_as(POINTER(c_int32)),
                         self.col.ctypes.data_as(POINTER(c_int32)),
                         self.w.ctypes.data_as(POINTER(c_double)))


class _ZCsr:
    """A complex CSR view of any scipy-convertible matrix (arrays kept alive)."""

    def __init__(self, m):
        import scipy.sparse as sp
        m = sp.csr_matrix(m, dtype=np.complex128)
        m.sort_indices()
        self.rowptr = np.ascontiguousarray(m.indptr, dtype=np.int32)
        self.col = np.ascontiguousarray(m.indices, dtype=np.int32)
        self.re = np.ascontiguousarray(m.data.real, dtype=np.float64)
        self.im = np.ascontiguousarray(m.data.imag, dtype=np.float64)
        self.c = qsw_zcsr(int(m.shape[0]), int(self.col.size),
                          self.rowptr.ctypes.data_as(POINTER(c_int32)),
                          self.col.ctypes.data_as(POINTER(c_int32)),
                          self.re.ctypes.data_as(POINTER(c_double)),
                          self.im.ctypes.data_as(POINTER(c_double)))


def _as_csr(g):
    if g is None:
        return None
    if hasattr(g, "rowptr"):   # workloads.Digraph
        return _Csr(g.n, g.rowptr, g.col, g.w)
    import scipy.sparse as sp
    m = sp.csr_matrix(g)
    m.sort_indices()
    return _Csr(m.shape[0], m.indptr, m.indices, m.data)


def _ports(ports):
    ports = list(ports or [])
    arr = (qsw_port * max(1, len(ports)))()
    for k, (v, r) in enumerate(ports):
        arr[k].vertex = int(v)
        arr[k].rate = float(r)
    return arr, len(ports)


# ------------------------------------------------------------------ calls --

def qsw_create(device: int = 0, stream: int | None = None):
    h = c_void_p()
    st = lib().qsw_create(byref(h), int(device), c_void_p(stream) if stream else None)
    _check(st)
    return h


def qsw_destroy(ctx) -> None:
    lib().qsw_destroy(ctx)


def qsw_last_error(ctx) -> str:
    msg = lib().qsw_last_error(ctx)
    return msg.decode() if msg else ""


def qsw_build_superoperator(ctx, G, H=None, omega: float = 0.5, sources=(), sinks=(),
                            precision="c128", operator="matfree", defer_norms: bool = False,
                            fixed_schedule: bool = False, fp64_ranking: bool = False):
    g = _as_csr(G)
    h = _as_csr(H)
    src, nsrc = _ports(sources)
    snk, nsnk = _ports(sinks)
    prec = PRECISIONS.get(precision, precision)
    kind = (OPERATORS.get(operator, operator) | (QSW_BUILD_DEFER_NORMS if defer_norms else 0)
            | (QSW_BUILD_FIXED_SCHEDULE if fixed_schedule else 0)
            | (QSW_BUILD_FP64_RANKING if fp64_ranking else 0))
    op = c_void_p()
    st = lib().qsw_build_superoperator(ctx, byref(g.c), byref(h.c) if h else None, float(omega),
                                       src, nsrc, snk, nsnk, int(prec), int(kind), byref(op))
    _check(st, ctx)
    return op


def qsw_build_global(ctx, n_vertices: int, H, Ls=(), H_rot=None, omega: float = 0.5, sources=(),
                     sinks=(), precision="c128", defer_norms: bool = False):
    """Global-interaction walk (G-QSW / NM-G-QSW) from explicit operators:
    H (Hermitian), Lindblad operators Ls, optional rotating Hamiltonian H_rot."""
    h = _ZCsr(H)
    ls = [_ZCsr(L) for L in Ls]
    arr = (qsw_zcsr * max(1, len(ls)))(*[z.c for z in ls])
    rot = _ZCsr(H_rot) if H_rot is not None else None
    src, nsrc = _ports(sources)
    snk, nsnk = _ports(sinks)
    op = c_void_p()
    st = lib().qsw_build_global(ctx, int(n_vertices), byref(h.c), arr, len(ls),
                                byref(rot.c) if rot else None, float(omega), src, nsrc, snk, nsnk,
                                int(PRECISIONS.get(precision, precision)),
                                QSW_BUILD_DEFER_NORMS if defer_norms else 0, byref(op))
    _check(st, ctx)
    return op


def qsw_build_gqsw(ctx, G, H=None, omega: float = 0.5, sources=(), sinks=(), precision="c128"):
    """G-QSW of digraph G: L = [G], H as passed or the Laplacian of G^u."""
    g = _as_csr(G)
    h = _as_csr(H)
    src, nsrc = _ports(sources)
    snk, nsnk = _ports(sinks)
    op = c_void_p()
    st = lib().qsw_build_gqsw(ctx, byref(g.c), byref(h.c) if h else None, float(omega), src, nsrc,
                              snk, nsnk, int(PRECISIONS.get(precision, precision)), byref(op))
    _check(st, ctx)
    return op


def qsw_build_nm_gqsw(ctx, G, omega: float = 0.5, precision="c128"):
    """Non-moralising G-QSW of digraph G on its demoralised vertex copies."""
    g = _as_csr(G)
    op = c_void_p()
    _check(lib().qsw_build_nm_gqsw(ctx, byref(g.c), float(omega),
                                   int(PRECISIONS.get(precision, precision)), byref(op)), ctx)
    return op


def qsw_nm_vsets(ctx, op, n_vertices: int) -> np.ndarray:
    off = np.zeros(n_vertices + 1, dtype=np.int32)
    _check(lib().qsw_nm_vsets(op, off.ctypes.data_as(POINTER(c_int32))), ctx)
    return off


def qsw_nm_populations(ctx, op, d_pops_expanded, count: int, d_pops) -> None:
    _check(lib().qsw_nm_populations(op, _ptr(d_pops_expanded), int(count), _ptr(d_pops)), ctx)


def qsw_nm_initial_state(ctx, op, pops, d_state) -> None:
    p = np.ascontiguousarray(pops, dtype=np.float64)
    _check(lib().qsw_nm_initial_state(op, p.ctypes.data_as(POINTER(c_double)), _ptr(d_state)), ctx)


def qsw_set_omega(ctx, op, omega: float) -> None:
    _check(lib().qsw_set_omega(op, float(omega)), ctx)


def qsw_op_info(ctx, op) -> dict:
    nt, n, nnz = c_int64(), c_int64(), c_int64()
    norms = (c_double * 9)()
    _check(lib().qsw_op_info(op, byref(nt), byref(n), byref(nnz), norms), ctx)
    return {"n_tilde": nt.value, "n": n.value, "nnz": nnz.value, "norms": list(norms)}


def qsw_op_export_csr(ctx, op, d_rowptr, d_col, d_val) -> None:
    _check(lib().qsw_op_export_csr(op, _ptr(d_rowptr), _ptr(d_col), _ptr(d_val)), ctx)


def qsw_op_destroy(op) -> None:
    lib().qsw_op_destroy(op)


def qsw_initial_state(ctx, op, d_state, rho0=None, populations=None) -> None:
    r = None if rho0 is None else np.asfortranarray(np.asarray(rho0, dtype=np.complex128))
    p = None if populations is None else np.ascontiguousarray(populations, dtype=np.float64)
    _check(lib().qsw_initial_state(op, _ptr(r), _ptr(p), _ptr(d_state)), ctx)


def qsw_apply(ctx, op, d_x, d_y) -> None:
    _check(lib().qsw_apply(op, _ptr(d_x), _ptr(d_y)), ctx)


def qsw_expmv_series(ctx, op, d_rho0, t0: float, dt: float, steps: int, d_out=None,
                     d_pops=None) -> dict:
    stats = qsw_series_stats()
    _check(lib().qsw_expmv_series(op, _ptr(d_rho0), float(t0), float(dt), int(steps),
                                  _ptr(d_out), _ptr(d_pops), byref(stats)), ctx)
    return stats.as_dict()


def qsw_expmv_series_noalloc(ctx, op, d_rho0, t0: float, dt: float, steps: int, d_out=None,
                             d_pops=None) -> dict:
    """qsw_expmv_series with its workspace in the library's fixed device array
    (NOALLOC_SCRATCH_BYTES per device); no device allocation in the call."""
    stats = qsw_series_stats()
    _check(lib().qsw_expmv_series_noalloc(op, _ptr(d_rho0), float(t0), float(dt), int(steps),
                                          _ptr(d_out), _ptr(d_pops), byref(stats)), ctx)
    return stats.as_dict()


def qsw_expmv_series_host(ctx, op, h_rho0, t0: float, dt: float, steps: int, h_out=None,
                          h_pops=None) -> dict:
    stats = qsw_series_stats()
    _check(lib().qsw_expmv_series_host(op, _ptr(h_rho0), float(t0), float(dt), int(steps),
                                       _ptr(h_out), _ptr(h_pops), byref(stats)), ctx)
    return stats.as_dict()


def qsw_populations(ctx, op, d_rho_series, count: int, d_pops) -> None:
    _check(lib().qsw_populations(op, _ptr(d_rho_series), int(count), _ptr(d_pops)), ctx)


def qsw_batch_series(ctx, ops, d_rho0s, n0: int, t0s, dts, steps, d_pops) -> dict:
    """Many walks in one launch; lists of per-walk operators / device buffers."""
    k = len(ops)
    arr = lambda T, xs: (T * k)(*xs)
    stats = qsw_batch_stats()
    _check(lib().qsw_batch_series(ctx, k, arr(c_void_p, [o.value if isinstance(o, c_void_p) else o for o in ops]),
                                  arr(c_void_p, [_ptr(x).value for x in d_rho0s]), int(n0),
                                  arr(c_double, [float(x) for x in t0s]),
                                  arr(c_double, [float(x) for x in dts]),
                                  arr(c_int32, [int(x) for x in steps]),
                                  arr(c_void_p, [_ptr(x).value for x in d_pops]), byref(stats)), ctx)
    return stats.as_dict()


def qsw_survival_time(ctx, op, d_rho0, t_end: float, q: int, sink: int, d_pops=None):
    """Expected survival time (Simpson over the sink population); returns
    (eta, series stats)."""
    eta = c_double()
    stats = qsw_series_stats()
    _check(lib().qsw_survival_time(op, _ptr(d_rho0), float(t_end), int(q), int(sink), byref(eta),
                                   _ptr(d_pops), byref(stats)), ctx)
    return eta.value, stats.as_dict()


def qsw_batch_survival_time(ctx, ops, d_rho0s, t_ends, qs, sinks):
    """Expected survival times of many walks in one batched launch; returns
    (list of eta, batch stats)."""
    k = len(ops)
    eta = (c_double * k)()
    stats = qsw_batch_stats()
    _check(lib().qsw_batch_survival_time(
        ctx, k, (c_void_p * k)(*[o.value if isinstance(o, c_void_p) else o for o in ops]),
        (c_void_p * k)(*[_ptr(x).value for x in d_rho0s]),
        (c_double * k)(*[float(x) for x in t_ends]), (c_int32 * k)(*[int(x) for x in qs]),
        (c_int32 * k)(*[int(x) for x in sinks]), eta, byref(stats)), ctx)
    return list(eta), stats.as_dict()


def qsw_probe_wait_limit(ctx) -> float:
    """Run the grid barrier with one block absent; seconds until it gave up."""
    sec = c_double()
    _check(lib().qsw_probe_wait_limit(ctx, byref(sec)), ctx)
    return sec.value


def qsw_server_create(device: int = 0, workers: int = 2, max_batch: int = 64,
                      memory_budget_bytes: float = 0.0):
    h = c_void_p()
    cfg = qsw_server_config(int(workers), int(max_batch), float(memory_budget_bytes))
    _check(lib().qsw_server_create(int(device), byref(cfg), byref(h)))
    return h


class Request:
    """Host-side request; keeps every buffer the server reads or writes alive."""

    def __init__(self, G, omega, t0, dt, steps, precision="c128", rho0=None, populations=None):
        self.g = _as_csr(G)
        self.n = self.g.c.n
        self.rho0 = None if rho0 is None else np.asfortranarray(np.asarray(rho0, np.complex128))
        self.pops0 = None if populations is None else np.ascontiguousarray(populations, np.float64)
        self.pops = np.zeros((steps + 1, self.n))
        self.c = qsw_request(self.g.c, float(omega), int(PRECISIONS.get(precision, precision)),
                             _ptr(self.rho0), _ptr(self.pops0), float(t0), float(dt), int(steps),
                             _ptr(self.pops))
        self.id = None


def qsw_server_submit(server, req: "Request") -> int:
    i = c_int64()
    _check(lib().qsw_server_submit(server, byref(req.c), byref(i)))
    req.id = i.value
    return i.value


def qsw_server_wait(server, req: "Request", timeout_s: float = 600.0) -> dict:
    res = qsw_request_result()
    st = lib().qsw_server_wait(server, int(req.id), float(timeout_s), byref(res))
    if st != 0:
        raise QswError(st, res.error.decode(errors="replace"))
    return {"latency_ms": res.latency_ms, "queue_ms": res.queue_ms}


def qsw_server_stats(server) -> dict:
    q, b, m = c_int64(), c_int64(), c_double()
    _check(lib().qsw_server_stats(server, byref(q), byref(b), byref(m)))
    return {"queued": q.value, "batches": b.value, "bytes_in_use": m.value}


def qsw_server_destroy(server) -> None:
    lib().qsw_server_destroy(server)


def qsw_kernel_launches() -> int:
    return int(lib().qsw_kernel_launches())


def qsw_device_allocations() -> int:
    return int(lib().qsw_device_allocations())


def qsw_tune_measurements() -> int:
    return int(lib().qsw_tune_measurements())


def qsw_tune_reset() -> None:
    lib().qsw_tune_reset()


def qsw_batch_set_schedule(ctx, cluster_size: int = 0, small_limit: int = -1) -> None:
    """Fix the batched series phase's schedule for this context (0 / -1: tuned)."""
    _check(lib().qsw_batch_set_schedule(ctx, int(cluster_size), int(small_limit)), ctx)


def qsw_op_set_csr_schedule(op, lanes_per_row: int, unroll: int = 2, ctx=None) -> None:
    """Fix a CSR operator's schedule (-1: the sliced form)."""
    _check(lib().qsw_op_set_csr_schedule(op, int(lanes_per_row), int(unroll)), ctx)


def qsw_op_schedule(op, with_unroll: bool = False):
    """CSR lanes per row (0 for matrix-free); with_unroll: (lanes, unroll depth)."""
    v, u = c_int32(), c_int32()
    _check(lib().qsw_op_schedule(op, byref(v), byref(u)))
    return (v.value, u.value) if with_unroll else v.value


def qsw_theta_table(precision="c128") -> np.ndarray:
    out = (c_double * 55)()
    _check(lib().qsw_theta_table(int(PRECISIONS.get(precision, precision)), out))
    return np.array(out[:])


def qsw_select_params(norms9, t: float, n0: int = 1, precision="c128"):
    arr = (c_double * 9)(*[float(x) for x in norms9])
    m, s = c_int32(), c_int32()
    _check(lib().qsw_select_params(arr, float(t), int(n0), int(PRECISIONS.get(precision, precision)),
                                   byref(m), byref(s)))
    return m.value, s.value
