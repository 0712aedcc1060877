"""The 1-norm series on the GPU: every estimate is one the Higham & Tisseur
block estimator (Algorithm 2.4) can return, checked against the exact powers.

The library shares work between the estimates: one chain for the common
starting block, cached chains A^k e_c for the unit vectors of later
iterations, products restricted to the growing support of those chains, and
the adjoint step split as (A^H)^p 1 + (A^H)^p (sign(Y) - 1) where that support
is small.  L~ maps X^dag to (L~ X)^dag, so the columns (a, b) and (b, a) of
L~^p have equal norms and the row ranking has exact ties that rounding breaks;
the GPU and the oracle's estimator (different summation orders) may therefore
follow different valid branches.  What must hold on every branch:

* the estimate is the 1-norm of A^p x for a column x the algorithm tries:
  a unit vector e_c or a column of the starting block [1, s] / n;
* hence it is at most ||A^p||_1, and it is close to it (here >= 1/10).

The walks are small enough for the exact powers (dense, n <= 4356) and shaped
so that the supports stay small for several powers (a cycle, a lattice) or
fill after a few (a random digraph)."""
import functools

import numpy as np
import pytest

from oracle import graph, normest, superop
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


def _weighted(g, seed):
    rng = np.random.default_rng(seed)
    dst = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    return W.from_arcs(g.n, dst, g.col, rng.uniform(0.5, 1.5, g.nnz))


def _graph(kind):
    if kind == "cycle60":
        return _weighted(W.cycle_graph(60), 60)
    if kind == "grid8":
        return _weighted(W.grid_graph(8, 8), 8)
    return W.random_digraph(40, 0.1, 40)


CASES = [
    ("cycle60", 0.3, [(0, 0.7)], [(30, 1.1)]),
    ("cycle60", 0.0, [(5, 0.4)], []),
    ("cycle60", 1.0, [], [(10, 0.9)]),
    ("grid8", 0.6, [(0, 0.5)], [(63, 0.8)]),
    ("er40", 0.45, [(3, 0.5)], [(17, 0.8)]),
]


def _achievable(L, pmax=9):
    """Per p: ||L^p||_1 and the sorted 1-norms of every column of L^p and of
    L^p [1, s] / n (the values the estimator can return)."""
    n = L.shape[0]
    X0 = np.ones((n, 2), complex)
    X0[:, 1] = normest.start_signs(n)
    X0 /= n
    P = np.eye(n, dtype=complex)
    out = {}
    for p in range(1, pmax + 1):
        P = L @ P
        X0 = L @ X0
        cols = np.abs(P).sum(axis=0)
        out[p] = (cols.max(), np.sort(np.concatenate([cols, np.abs(X0).sum(axis=0)])))
    return out


@functools.lru_cache(maxsize=None)
def _exact(kind, omega, sources, sinks):
    walk = graph.lqsw_walk(graph.adjacency(_graph(kind)), sources=sources, sinks=sinks)
    return _achievable(superop.superoperator(walk, omega))


@pytest.mark.parametrize("kind,omega,sources,sinks", CASES)
@pytest.mark.parametrize("operator", ["matfree", "csr"])
def test_norm_series_is_an_estimator_outcome(ctx, kind, omega, sources, sinks, operator):
    from paper_2003_02450_gb300.walk import LQSW
    g = _graph(kind)
    vals = _exact(kind, omega, tuple(sources), tuple(sinks))
    w = LQSW(g, omega, sources=sources, sinks=sinks, ctx=ctx, operator=operator)
    got = np.asarray(w.norms)
    assert got[0] == pytest.approx(vals[1][0], rel=1e-14)
    for p in range(2, 10):
        exact, v = vals[p]
        est = got[p - 1]
        assert est <= exact * (1 + 1e-12)
        assert est >= exact / 10
        k = np.searchsorted(v, est)
        near = min(abs(v[max(k - 1, 0)] - est), abs(v[min(k, v.size - 1)] - est))
        assert near <= 1e-10 * exact, (p, est, exact)
    again = LQSW(g, omega, sources=sources, sinks=sinks, ctx=ctx, operator=operator)
    assert np.array_equal(np.asarray(again.norms), got)


GLOBAL_CASES = [
    # (kind, omega, sources, sinks)
    ("gqsw", 0.5, [(0, 0.6)], [(19, 0.9)]),
    ("gqsw", 0.0, [], []),
    ("nm", 0.3, [], []),
    ("nm", 1.0, [], []),
]


@functools.lru_cache(maxsize=None)
def _global_exact(kind, omega, sources, sinks):
    from oracle import gqsw, nm
    g = W.random_digraph(20, 0.15, 20) if kind == "gqsw" else W.random_digraph(9, 0.3, 9)
    if kind == "gqsw":
        walk = gqsw.global_walk(g.dense(), sources=sources, sinks=sinks)
    else:
        walk, _ = nm.nm_walk(g.dense())
    return g, _achievable(gqsw.superoperator(walk, omega))


@pytest.mark.parametrize("kind,omega,sources,sinks", GLOBAL_CASES)
def test_global_walk_norm_series_is_an_estimator_outcome(ctx, kind, omega, sources, sinks):
    """Global walks take the Hermitian column through the two-pass Hermitian
    apply (W_k and R = x Q^dag, then the upper triangle, mirrored)."""
    from paper_2003_02450_gb300 import qsw as C
    g, vals = _global_exact(kind, omega, tuple(sources), tuple(sinks))
    build = (lambda: C.qsw_build_gqsw(ctx.handle, g, None, omega, sources, sinks)) \
        if kind == "gqsw" else (lambda: C.qsw_build_nm_gqsw(ctx.handle, g, omega))
    op = build()
    got = np.asarray(C.qsw_op_info(ctx.handle, op)["norms"])
    C.qsw_op_destroy(op)
    assert got[0] <= vals[1][0] * (1 + 1e-12) and got[0] >= vals[1][0] / 10
    for p in range(2, 10):
        exact, v = vals[p]
        est = got[p - 1]
        assert est <= exact * (1 + 1e-12)
        assert est >= exact / 10
        k = np.searchsorted(v, est)
        near = min(abs(v[max(k - 1, 0)] - est), abs(v[min(k, v.size - 1)] - est))
        assert near <= 1e-10 * exact, (p, est, exact)
    op = build()
    again = np.asarray(C.qsw_op_info(ctx.handle, op)["norms"])
    C.qsw_op_destroy(op)
    assert np.array_equal(again, got)


@pytest.mark.parametrize("kind,omega,sources,sinks", CASES[:1] + CASES[3:])
def test_fp64_ranking_flag_gives_estimator_outcomes(ctx, kind, omega, sources, sinks):
    """QSW_BUILD_FP64_RANKING keeps the adjoint step of every estimate in
    complex128; the default ranks rows in complex64.  Both return values the
    estimator can return (FP64 norms of tried columns), both repeatably."""
    from paper_2003_02450_gb300 import qsw as C
    g = _graph(kind)
    vals = _exact(kind, omega, tuple(sources), tuple(sinks))
    got = {}
    for rank64 in (False, True):
        runs = []
        for _ in range(2):
            op = C.qsw_build_superoperator(ctx.handle, g, None, omega, sources, sinks,
                                           fp64_ranking=rank64)
            runs.append(np.asarray(C.qsw_op_info(ctx.handle, op)["norms"]))
            C.qsw_op_destroy(op)
        assert np.array_equal(runs[0], runs[1])
        got[rank64] = runs[0]
        for p in range(2, 10):
            exact, v = vals[p]
            est = runs[0][p - 1]
            assert exact / 10 <= est <= exact * (1 + 1e-12)
            k = np.searchsorted(v, est)
            near = min(abs(v[max(k - 1, 0)] - est), abs(v[min(k, v.size - 1)] - est))
            assert near <= 1e-10 * exact, (rank64, p, est, exact)
    assert got[False][0] == got[True][0]
