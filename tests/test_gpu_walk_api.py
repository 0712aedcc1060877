"""The Section 4.1.2 example session through the object API (walk.py): the
three-vertex digraph as a G-QSW, as an NM-G-QSW and as an L-QSW, at omega = 1
and after set_omega(0), with the printed populations at t = 100."""
import numpy as np
import pytest

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


def _example():
    G = np.zeros((3, 3))
    G[2, 0] = G[2, 1] = 1.0
    GU = np.maximum(G, G.T)
    return W.from_dense(G), W.from_dense(GU)


def test_example_session(ctx):
    from paper_2003_02450_gb300.walk import GQSW, LQSW, NMGQSW
    G, GU = _example()
    rho_0 = [1.0, 0.0, 0.0]

    gqsw = GQSW(G, 1.0, ctx=ctx)
    gqsw.initial_state(populations=rho_0)
    p = gqsw.populations(gqsw.step(100.0)).cpu().numpy()[0]
    assert np.allclose(p, [0.25, 0.25, 0.5], atol=1e-10)

    nm = NMGQSW(G, 1.0, ctx=ctx)
    nm.initial_state(populations=rho_0)
    p = nm.series_vertices(100.0, 0.0, 0).cpu().numpy()[0]
    assert p[0] == pytest.approx(3.72007598e-44, rel=1e-6)
    assert abs(p[1]) <= 1e-14 and p[2] == pytest.approx(1.0, abs=1e-12)

    lqsw = LQSW(G, 1.0, H=GU, ctx=ctx)
    lqsw.initial_state(populations=rho_0)
    p = lqsw.populations(lqsw.step(100.0)).cpu().numpy()[0]
    assert abs(p[0]) <= 1e-15 and abs(p[1]) <= 1e-15 and p[2] == pytest.approx(1.0, abs=1e-12)

    # coherent limit: set_omega(0) on both, printed [3.80773381e-07 9.98766244e-01 1.23337485e-03]
    nm.set_omega(0.0)
    lqsw.set_omega(0.0)
    p_nm = nm.series_vertices(100.0, 0.0, 0).cpu().numpy()[0]
    p_l = lqsw.populations(lqsw.step(100.0)).cpu().numpy()[0]
    for p in (p_nm, p_l):
        assert p[0] == pytest.approx(3.8077338e-07, abs=1e-12)
        assert p[1] == pytest.approx(9.98766244e-01, abs=5e-9)
        assert p[2] == pytest.approx(1.23337485e-03, abs=5e-11)

    # the omega = 0.9 series of both walks (the figure's comparison): the
    # NM-G-QSW moves more probability into the sink vertex v3
    nm.set_omega(0.9)
    lqsw.set_omega(0.9)
    nm.initial_state(populations=rho_0)
    lqsw.initial_state(populations=rho_0)
    s_nm = nm.series_vertices(0.0, 25.0 / 500, 500).cpu().numpy()
    _, s_l = lqsw.series(0.0, 25.0 / 500, 500, states=False)
    s_l = s_l.cpu().numpy()
    assert np.allclose(s_nm.sum(axis=1), 1.0, atol=1e-10) and np.allclose(s_l.sum(axis=1), 1.0, atol=1e-10)
    assert s_nm[-1, 2] > s_l[-1, 2]
    for w in (gqsw, nm, lqsw):
        w.close()


def test_walk_survival_time_method(ctx):
    from paper_2003_02450_gb300.walk import LQSW
    g, h = W.dipole_network(4, 3)
    w = LQSW(g, 0.7, H=h, sources=[(0, 0.5)], sinks=[(3, 0.5)], ctx=ctx)
    w.initial_state(rho0=W.basis_state(6, 4))
    eta = w.survival_time(20.0, 40, 5)
    from oracle import est, graph, superop
    walk = graph.lqsw_walk(graph.adjacency(g), H=h, sources=[(0, 0.5)], sinks=[(3, 0.5)])
    ref, _ = est.survival_time(superop.superoperator(walk, 0.7), 6, W.vec(W.basis_state(6, 4)),
                               20.0, 40, 5)
    assert abs(eta - ref) <= 20.0 * 1e-10
    w.close()
