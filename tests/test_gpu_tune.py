"""The autotuned CSR schedule (lanes per row and unroll depth of the series
kernel's CSR sweep).

The first CSR series of a (precision, row-length, size) bucket measures every
candidate and caches the fastest; later operators of the bucket reuse it.  The
choice may only change the summation order within a row, so the tuned result
matches the oracle at the parity bound and the fixed-schedule result to
rounding."""
import numpy as np
import pytest

from oracle import expmv, graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    import torch
    from paper_2003_02450_gb300.walk import Context
    assert torch.cuda.is_available()
    return Context(0)


def _series(ctx, op, g, rho0, steps, dt):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    n = g.n * g.n
    out = torch.empty((steps + 1, n), dtype=torch.complex128, device="cuda")
    C.qsw_expmv_series(ctx.handle, op, torch.from_numpy(W.vec(rho0)).cuda(), 0.0, dt, steps, out, None)
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_tuned_csr_schedule_is_cached_and_exact(ctx, precision):
    from paper_2003_02450_gb300 import qsw as C
    g = W.erdos_renyi_digraph(60, 0.1, 4242)
    rho0 = W.random_density_matrix(60, 17)
    C.qsw_tune_reset()
    m0 = C.qsw_tune_measurements()
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.35, precision=precision, operator="csr")
    heuristic = C.qsw_op_schedule(op)
    assert heuristic in (1, 2, 4, 8, 16, 32)
    assert C.qsw_op_schedule(op, with_unroll=True) == (heuristic, 2)
    got = _series(ctx, op, g, rho0, 12, 0.25)
    tuned = C.qsw_op_schedule(op)
    assert tuned in (1, 2, 4, 8, 16, 32)
    assert C.qsw_op_schedule(op, with_unroll=True)[1] in (2, 4)
    assert C.qsw_tune_measurements() == m0 + 1           # one measurement for the bucket
    # a second operator of the same bucket reuses the choice without measuring
    op2 = C.qsw_build_superoperator(ctx.handle, g, None, 0.6, precision=precision, operator="csr")
    _series(ctx, op2, g, rho0, 3, 0.25)
    assert C.qsw_op_schedule(op2, with_unroll=True) == C.qsw_op_schedule(op, with_unroll=True)
    assert C.qsw_tune_measurements() == m0 + 1
    # set_omega keeps the tuned schedule (same structure)
    C.qsw_set_omega(ctx.handle, op2, 0.2)
    assert C.qsw_op_schedule(op2) == tuned
    # a fixed-schedule operator keeps the heuristic and gives the same result to rounding
    opf = C.qsw_build_superoperator(ctx.handle, g, None, 0.35, precision=precision, operator="csr",
                                    fixed_schedule=True)
    ref_fixed = _series(ctx, opf, g, rho0, 12, 0.25)
    assert C.qsw_op_schedule(opf, with_unroll=True) == (heuristic, 2)
    assert C.qsw_tune_measurements() == m0 + 1
    walk = graph.lqsw_walk(graph.adjacency(g))
    L = superop.superoperator(walk, 0.35)
    X = expmv.expmv_series(L, W.vec(rho0), 0.0, 0.25, 12)
    if precision == "c128":
        assert np.max(np.abs(got - X)) <= 1e-10
        assert np.max(np.abs(got - ref_fixed)) <= 1e-13
    else:
        pops = superop.populations(got, 60)
        assert np.max(np.abs(pops - superop.populations(X, 60))) <= 1e-4
        assert np.max(np.abs(pops - superop.populations(ref_fixed, 60))) <= 1e-5
    for o in (op, op2, opf):
        C.qsw_op_destroy(o)


def test_matrix_free_operator_has_no_csr_schedule(ctx):
    from paper_2003_02450_gb300 import qsw as C
    op = C.qsw_build_superoperator(ctx.handle, W.cycle_graph(8), None, 0.5)
    assert C.qsw_op_schedule(op) == 0
    assert C.qsw_op_schedule(op, with_unroll=True) == (0, 0)
    C.qsw_op_destroy(op)
