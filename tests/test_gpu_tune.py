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
    assert tuned in (-1, 1, 2, 4, 8, 16, 32)   # -1: the sliced form
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


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_every_fixed_csr_schedule_matches_the_oracle(ctx, precision):
    """Each CSR schedule, the sliced form (-1) included, at both unroll depths:
    the series matches the oracle at the parity bound.  The graph's degrees
    vary, so the sliced form's rows are sorted and padded; 41^2 rows leave a
    partial last slice."""
    from paper_2003_02450_gb300 import qsw as C
    g = W.erdos_renyi_digraph(41, 0.12, 99)
    rho0 = W.random_density_matrix(41, 5)
    walk = graph.lqsw_walk(graph.adjacency(g))
    X = expmv.expmv_series(superop.superoperator(walk, 0.45), W.vec(rho0), 0.0, 0.3, 8)
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.45, precision=precision, operator="csr")
    m0 = C.qsw_tune_measurements()
    results = {}
    for lanes in (-1, 1, 2, 4, 8, 16, 32):
        for unroll in (2, 4):
            C.qsw_op_set_csr_schedule(op, lanes, unroll)
            got = _series(ctx, op, g, rho0, 8, 0.3)
            assert C.qsw_op_schedule(op, with_unroll=True) == (lanes, unroll)
            if precision == "c128":
                assert np.max(np.abs(got - X)) <= 1e-10, (lanes, unroll)
            else:
                err = np.max(np.abs(superop.populations(got, 41) - superop.populations(X, 41)))
                assert err <= 1e-4, (lanes, unroll)
            results[(lanes, unroll)] = got
    assert C.qsw_tune_measurements() == m0   # fixed schedules never tune
    # the sliced form survives set_omega (rebuilt from the new values)
    C.qsw_op_set_csr_schedule(op, -1, 2)
    C.qsw_set_omega(ctx.handle, op, 0.8)
    X8 = expmv.expmv_series(superop.superoperator(walk, 0.8), W.vec(rho0), 0.0, 0.3, 8)
    got8 = _series(ctx, op, g, rho0, 8, 0.3)
    if precision == "c128":
        assert np.max(np.abs(got8 - X8)) <= 1e-10
    assert C.qsw_op_schedule(op) == -1
    for lanes, unroll in ((0, 2), (3, 2), (64, 2), (2, 3)):
        with pytest.raises(C.QswError):
            C.qsw_op_set_csr_schedule(op, lanes, unroll)
    C.qsw_op_destroy(op)
    mf = C.qsw_build_superoperator(ctx.handle, W.cycle_graph(8), None, 0.5)
    with pytest.raises(C.QswError):
        C.qsw_op_set_csr_schedule(mf, 2, 2)
    C.qsw_op_destroy(mf)
