"""qsw_expmv_series_noalloc against qsw_expmv_series, through the C ABI.

The no-allocation entry point runs the same kernels with its workspace in the
library's fixed device array; its results must match the allocating entry
point's within the complex128 parity tolerance, on two calls in a row (the
second call finds the array dirty from the first and must clear what has to
start at zero).  This file is named to be collected last, so that it also runs
after every other GPU test in the same process.
"""
import numpy as np
import pytest

from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu

TOL_C128 = 1e-10     # max |rho| difference, as the parity tests
TOL_C64_POP = 1e-4   # populations, complex64 bulk


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    import torch
    from paper_2003_02450_gb300.walk import Context
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return Context(0)


def _walk(ctx, g, omega, precision="c128", operator="matfree", sources=(), sinks=()):
    from paper_2003_02450_gb300.walk import LQSW
    return LQSW(g, omega, sources=sources, sinks=sinks, precision=precision, ctx=ctx,
                operator=operator)


def _rho0(w, seed):
    import torch
    rho = W.random_density_matrix(w.n_tilde, seed)
    return torch.from_numpy(W.vec(rho)).to("cuda:0")


def _run(ctx, w, fn, rho0, t0, dt, steps, with_out=True):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    out = (torch.full((steps + 1, w.n, 2), np.nan, dtype=torch.float64, device="cuda:0")
           if with_out else None)
    pops = torch.full((steps + 1, w.n_tilde), np.nan, dtype=torch.float64, device="cuda:0")
    allocs0 = C.qsw_device_allocations()
    stats = getattr(C, fn)(ctx.handle, w.op, rho0, t0, dt, steps, out, pops)
    stats["device_allocations"] = C.qsw_device_allocations() - allocs0
    torch.cuda.synchronize()
    return (None if out is None else out.cpu().numpy()), pops.cpu().numpy(), stats


CASES = [
    # (graph, omega, precision, operator, sources, sinks, t0, dt, steps, with_out)
    ("cycle16", 0.5, "c128", "matfree", (), (), 0.0, 0.5, 20, True),
    ("er40", 0.37, "c128", "matfree", ((0, 0.5),), ((39, 0.5),), 0.3, 0.25, 33, True),
    ("er40", 0.6, "c128", "csr", (), (), 0.0, 1.0, 12, True),
    ("grid6", 0.1, "c128", "matfree", (), (), 0.2, 0.5, 40, False),
    ("grid6", 0.1, "c64", "matfree", (), (), 0.0, 0.5, 40, False),
]


def _graph(name):
    if name == "cycle16":
        return W.cycle_graph(16)
    if name == "er40":
        return W.erdos_renyi_digraph(40, 0.1, 7)
    return W.grid_graph(6, 6)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[2]}-{c[3]}-{'out' if c[9] else 'ring'}"
                                              for c in CASES])
def test_noalloc_matches_series_twice(ctx, case):
    gname, omega, prec, opk, src, snk, t0, dt, steps, with_out = case
    w = _walk(ctx, _graph(gname), omega, prec, opk, src, snk)
    rho0 = _rho0(w, 11)
    ref_out, ref_pops, ref_stats = _run(ctx, w, "qsw_expmv_series", rho0, t0, dt, steps, with_out)
    # positive control: the allocating entry point's first call on a fresh
    # operator allocates its workspace, and the counter sees it
    assert ref_stats["device_allocations"] > 0
    for call in range(2):
        out, pops, stats = _run(ctx, w, "qsw_expmv_series_noalloc", rho0, t0, dt, steps, with_out)
        # the property the entry point exists for: the library allocated nothing
        assert stats["device_allocations"] == 0, f"call {call}"
        assert np.all(np.isfinite(pops)), f"call {call}: unwritten populations"
        tol = TOL_C128 if prec == "c128" else TOL_C64_POP
        assert np.max(np.abs(pops - ref_pops)) <= tol, f"call {call}"
        if with_out:
            assert np.all(np.isfinite(out)), f"call {call}: unwritten states"
            assert np.max(np.abs(out - ref_out)) <= TOL_C128, f"call {call}"
        for key in ("m0", "s0", "m_star", "s", "jobs", "matvecs", "fupdates", "hermitian"):
            assert stats[key] == ref_stats[key], (call, key)
        assert stats["algorithmic_bytes"] == pytest.approx(ref_stats["algorithmic_bytes"], rel=1e-12)
        assert stats["kernel_ms"] == 0.0
    w.close()


def test_noalloc_rejects_oversize(ctx):
    """A walk whose two Taylor-term vectors alone exceed the fixed array is
    refused on the host, before any work is issued, and the context stays
    usable."""
    import torch
    from paper_2003_02450_gb300 import qsw as C
    n_tilde = 800   # 2 x 800^2 x 16 bytes = 20.5 MB > 16 MiB
    assert 2 * n_tilde ** 2 * 16 > C.NOALLOC_SCRATCH_BYTES
    w = _walk(ctx, W.cycle_graph(n_tilde), 0.5)
    rho0 = torch.from_numpy(W.vec(W.basis_state(n_tilde, 0))).to("cuda:0")
    out = torch.empty((2, w.n, 2), dtype=torch.float64, device="cuda:0")
    with pytest.raises(C.QswError) as e:
        C.qsw_expmv_series_noalloc(ctx.handle, w.op, rho0, 0.0, 1.0, 1, out, None)
    assert e.value.name == "QSW_ERR_TOO_LARGE"
    assert "bytes of scratch" in e.value.message
    w.close()
    # the next call on the same context still works
    w2 = _walk(ctx, W.cycle_graph(16), 0.5)
    r2 = _rho0(w2, 3)
    _, pops, _ = _run(ctx, w2, "qsw_expmv_series_noalloc", r2, 0.0, 0.5, 4)
    _, ref, _ = _run(ctx, w2, "qsw_expmv_series", r2, 0.0, 0.5, 4)
    assert np.max(np.abs(pops - ref)) <= TOL_C128
    w2.close()


def test_noalloc_needs_norms(ctx):
    """An operator built with deferred norms is refused (its norms need
    workspace) until the allocating entry point has computed them."""
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g = W.cycle_graph(12)
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.4, precision="c128", defer_norms=True)
    rho0 = torch.from_numpy(W.vec(W.basis_state(12, 0))).to("cuda:0")
    pops = torch.empty((4, 12), dtype=torch.float64, device="cuda:0")
    with pytest.raises(C.QswError) as e:
        C.qsw_expmv_series_noalloc(ctx.handle, op, rho0, 0.0, 0.5, 3, None, pops)
    assert e.value.name == "QSW_ERR_INVALID_ARG"
    C.qsw_expmv_series(ctx.handle, op, rho0, 0.0, 0.5, 3, None, pops)
    ref = pops.cpu().numpy()
    pops.fill_(float("nan"))
    C.qsw_expmv_series_noalloc(ctx.handle, op, rho0, 0.0, 0.5, 3, None, pops)
    assert np.max(np.abs(pops.cpu().numpy() - ref)) <= TOL_C128
    C.qsw_op_destroy(op)
