"""qsw_expmv_series_host: host buffers in and out, the copies inside the call.
The series kernel reports each Taylor block's finished outputs through a
host-mapped counter and the call copies them to the host on a second stream
while later blocks run.  Checked: the host result equals the device-buffer
result bit for bit and the oracle within the complex128 tolerance, for
pinned and pageable host arrays, Hermitian and general inputs, both operator
forms, complex64 bulk, global walks, and the edge cases (steps = 0, outputs
only, populations only)."""
import numpy as np
import pytest

from oracle import expmv, gqsw, graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    import torch
    from paper_2003_02450_gb300.walk import Context
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return Context(0)


def _host_arrays(shape_out, shape_pops, pinned):
    import torch
    out = torch.empty(shape_out, dtype=torch.complex128)
    pops = torch.empty(shape_pops, dtype=torch.float64)
    if pinned:
        out, pops = out.pin_memory(), pops.pin_memory()
    return out, pops


def _device_series(C, ctx, op, x0, t0, dt, steps, nt):
    import torch
    out = torch.empty((steps + 1, nt * nt), dtype=torch.complex128, device="cuda:0")
    pops = torch.empty((steps + 1, nt), dtype=torch.float64, device="cuda:0")
    C.qsw_expmv_series(ctx.handle, op, torch.from_numpy(x0).to("cuda:0"), t0, dt, steps, out, pops)
    return out.cpu().numpy(), pops.cpu().numpy()


@pytest.mark.parametrize("operator", ["matfree", "csr"])
@pytest.mark.parametrize("herm", [True, False])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_series_matches_device_and_oracle(ctx, operator, herm, pinned):
    from paper_2003_02450_gb300 import qsw as C
    g = W.random_digraph(30, 0.15, 31)
    src, snk = [(0, 0.6)], [(29, 0.9)]
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.4, src, snk, operator=operator)
    walk = graph.lqsw_walk(graph.adjacency(g), sources=src, sinks=snk)
    nt = walk.n_tilde
    x0 = W.vec(W.random_density_matrix(nt, 5)) if herm else \
        np.random.default_rng(6).standard_normal(nt * nt) + 0j
    t0, dt, steps = 0.3, 0.25, 24
    out, pops = _host_arrays((steps + 1, nt * nt), (steps + 1, nt), pinned)
    C.qsw_expmv_series_host(ctx.handle, op, np.ascontiguousarray(x0), t0, dt, steps, out, pops)
    d_out, d_pops = _device_series(C, ctx, op, x0, t0, dt, steps, nt)
    assert np.array_equal(out.numpy(), d_out)
    assert np.array_equal(pops.numpy(), d_pops)
    ref = expmv.expmv_series(superop.superoperator(walk, 0.4), x0, t0, dt, steps)
    assert np.max(np.abs(out.numpy() - ref)) <= 1e-10
    C.qsw_op_destroy(op)


def test_host_series_edge_cases(ctx):
    from paper_2003_02450_gb300 import qsw as C
    g = W.cycle_graph(12)
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.5)
    x0 = W.vec(W.basis_state(12, 0))
    d_out, d_pops = _device_series(C, ctx, op, x0, 0.0, 0.5, 9, 12)
    # steps = 0: rho(t0) only
    out, pops = _host_arrays((1, 144), (1, 12), True)
    C.qsw_expmv_series_host(ctx.handle, op, x0, 1.7, 0.0, 0, out, pops)
    e_out, _ = _device_series(C, ctx, op, x0, 1.7, 0.0, 0, 12)
    assert np.array_equal(out.numpy(), e_out)
    # outputs only, then populations only
    out, pops = _host_arrays((10, 144), (10, 12), True)
    C.qsw_expmv_series_host(ctx.handle, op, x0, 0.0, 0.5, 9, out, None)
    assert np.array_equal(out.numpy(), d_out)
    C.qsw_expmv_series_host(ctx.handle, op, x0, 0.0, 0.5, 9, None, pops)
    assert np.array_equal(pops.numpy(), d_pops)
    C.qsw_op_destroy(op)


def test_host_series_complex64_and_global(ctx):
    from paper_2003_02450_gb300 import qsw as C
    g = W.random_digraph(16, 0.2, 16)
    x0 = W.vec(W.random_density_matrix(16, 2))
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.6, precision="c64")
    out, pops = _host_arrays((13, 256), (13, 16), True)
    C.qsw_expmv_series_host(ctx.handle, op, x0, 0.0, 0.4, 12, out, pops)
    d_out, d_pops = _device_series(C, ctx, op, x0, 0.0, 0.4, 12, 16)
    assert np.array_equal(out.numpy(), d_out) and np.array_equal(pops.numpy(), d_pops)
    walk = graph.lqsw_walk(graph.adjacency(g))
    ref = expmv.expmv_series(superop.superoperator(walk, 0.6), x0, 0.0, 0.4, 12)
    assert np.max(np.abs(pops.numpy() - superop.populations(ref, 16))) <= 1e-4
    C.qsw_op_destroy(op)
    op = C.qsw_build_gqsw(ctx.handle, g, None, 0.6)
    C.qsw_expmv_series_host(ctx.handle, op, x0, 0.0, 0.4, 12, out, pops)
    L = gqsw.superoperator(gqsw.global_walk(g.dense()), 0.6)
    ref = expmv.expmv_series(L, x0, 0.0, 0.4, 12)
    assert np.max(np.abs(out.numpy() - ref)) <= 1e-10
    C.qsw_op_destroy(op)
