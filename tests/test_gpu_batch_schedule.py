"""The batched series phase's schedule: clusters of 2..16 CTAs, and the limit
below which a walk runs on one CTA with its Taylor terms in shared memory.

A walk's populations must not depend on the schedule: every element gets the
same arithmetic in the same order on every path, and the phase's cluster
reductions are maxima (order-free).  The autotuner times every candidate on
the first batch of a kind, then reuses its choice.
"""
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
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300.walk import Context
    assert torch.cuda.is_available()
    c = Context(0)
    yield c
    C.qsw_batch_set_schedule(c.handle, 0, -1)


def _batch(ctx, walks, n0, precision, q=10, dt=0.2):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    ops, rhos, pops = [], [], []
    for g, omega, states in walks:
        ops.append(C.qsw_build_superoperator(ctx.handle, g, None, omega, precision=precision,
                                             defer_norms=True))
        rhos.append(torch.from_numpy(np.concatenate([W.vec(s) for s in states[:n0]])).cuda())
        pops.append(torch.empty((q + 1) * n0 * g.n, dtype=torch.float64, device="cuda"))
    k = len(walks)
    st = C.qsw_batch_series(ctx.handle, ops, rhos, n0, [0.0] * k, [dt] * k, [q] * k, pops)
    for o in ops:
        C.qsw_op_destroy(o)
    return [p.cpu().numpy().reshape(q + 1, n0, g.n) for p, (g, _, _) in zip(pops, walks)], st


def _walks():
    # N = 8 .. 80: two Taylor-term blocks of 4 complex64 columns take
    # 64 N^2 bytes, so the set straddles the 32 KB and 64 KB limits
    return W.batch_regular(count=20, seed=31, nmin=8, nmax=80, rhs=4)


@pytest.mark.parametrize("precision,n0", [("c64", 4), ("c128", 2)])
def test_populations_do_not_depend_on_the_schedule(ctx, precision, n0):
    from paper_2003_02450_gb300 import qsw as C
    walks = _walks()
    ref = None
    seen = set()
    for cs in (2, 4, 8, 16):
        for limit in (0, 32768, 65536):
            C.qsw_batch_set_schedule(ctx.handle, cs, limit)
            got, st = _batch(ctx, walks, n0, precision)
            assert (st["cluster_size"], st["small_limit"], st["tuned"]) == (cs, limit, 0)
            seen.add(st["small_walks"])
            if ref is None:
                ref = got
            else:
                for a, b in zip(ref, got):
                    assert np.array_equal(a, b), (cs, limit)
    assert len(seen) == 3   # the limits moved walks between the two paths
    C.qsw_batch_set_schedule(ctx.handle, 0, -1)
    # and the results are the oracle's
    tol = 1e-10 if precision == "c128" else 1e-4
    for (g, omega, states), p in list(zip(walks, ref))[::7]:
        walk = graph.lqsw_walk(graph.adjacency(g))
        L = superop.superoperator(walk, omega)
        B = np.stack([W.vec(s) for s in states[:n0]], axis=1)
        X = expmv.expmv_series(L, B, 0.0, 0.2, 10, n0=n0)
        nt = walk.n_tilde
        o = np.real(X[:, np.arange(nt) * (nt + 1), :]).transpose(0, 2, 1)
        assert np.max(np.abs(p - o)) <= tol


def test_tuner_measures_once_per_kind_and_keeps_results(ctx):
    from paper_2003_02450_gb300 import qsw as C
    C.qsw_batch_set_schedule(ctx.handle, 0, -1)
    C.qsw_tune_reset()
    walks = _walks()
    m0 = C.qsw_tune_measurements()
    got1, st1 = _batch(ctx, walks, 4, "c64")
    assert st1["tuned"] == 1 and C.qsw_tune_measurements() == m0 + 1
    assert st1["cluster_size"] in (4, 8, 16) and st1["small_limit"] in (0, 32768, 65536)
    got2, st2 = _batch(ctx, walks, 4, "c64")
    assert st2["tuned"] == 0 and C.qsw_tune_measurements() == m0 + 1
    assert (st2["cluster_size"], st2["small_limit"]) == (st1["cluster_size"], st1["small_limit"])
    for a, b in zip(got1, got2):
        assert np.array_equal(a, b)
    # below the tuning size: the default schedule, no measurement
    few, st3 = _batch(ctx, walks[:5], 4, "c64")
    assert st3["tuned"] == 0 and (st3["cluster_size"], st3["small_limit"]) == (8, 65536)
    assert C.qsw_tune_measurements() == m0 + 1
    for a, b in zip(few, got1[:5]):
        assert np.array_equal(a, b)
    # one half fixed, the other from the tuned pair
    C.qsw_batch_set_schedule(ctx.handle, 2, -1)
    _, st4 = _batch(ctx, walks, 4, "c64")
    assert st4["cluster_size"] == 2 and st4["tuned"] == 0
    assert st4["small_limit"] == st1["small_limit"]
    C.qsw_batch_set_schedule(ctx.handle, 0, -1)


def test_schedule_arguments_are_checked(ctx):
    from paper_2003_02450_gb300 import qsw as C
    for cs, limit in ((3, -1), (32, -1), (-1, -1), (0, -2), (0, 65537)):
        with pytest.raises(C.QswError) as e:
            C.qsw_batch_set_schedule(ctx.handle, cs, limit)
        assert e.value.name == "QSW_ERR_INVALID_ARG"
