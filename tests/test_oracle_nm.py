"""Pins of the NM-G-QSW demoralisation (oracle/nm.py)."""
import numpy as np
import pytest

from oracle import expmv, gqsw, nm, superop
from paper_2003_02450_gb300 import workloads as W


def _three():
    G = np.zeros((3, 3))
    G[2, 0] = G[2, 1] = 1.0     # arcs v1 -> v3, v2 -> v3
    return G


def _evolve(G, omega, pops0, t):
    walk, vs = nm.nm_walk(G)
    L = gqsw.superoperator(walk, omega)
    rho = expmv.expmv_step(L, W.vec(nm.initial_state(pops0, vs)), t)
    return nm.populations(superop.populations(rho, walk.n_tilde), vs)


def test_paper_example_omega_one():
    """Section 4.1.2: the NM-G-QSW at omega = 1 moves the walker to the sink,
    printed [3.72007598e-44, 0, 1] at t = 100 (v1 decays at unit rate)."""
    p = _evolve(_three(), 1.0, [1, 0, 0], 100.0)
    assert p[0] == pytest.approx(3.72007598e-44, rel=1e-6)
    assert abs(p[1]) <= 1e-14
    assert p[2] == pytest.approx(1.0, abs=1e-12)


def test_paper_example_omega_zero():
    """Printed at omega = 0, t = 100: [3.80773381e-07, 9.98766244e-01, 1.23337485e-03]."""
    p = _evolve(_three(), 0.0, [1, 0, 0], 100.0)
    assert p[0] == pytest.approx(3.80773381e-07, abs=1e-12)
    assert p[1] == pytest.approx(9.98766244e-01, abs=5e-9)
    assert p[2] == pytest.approx(1.23337485e-03, abs=5e-11)


def test_no_spontaneous_moralisation():
    """At omega = 1 population only moves along arcs: a vertex unreachable from
    the start keeps probability 0 (the G-QSW moralises: v2 gets 1/4)."""
    rng = np.random.default_rng(3)
    for trial in range(4):
        n = 7
        G = np.triu((rng.random((n, n)) < 0.4) * rng.uniform(0.5, 1.5, (n, n)), 1).T  # DAG: j -> i, i > j
        start = 2
        reach = {start}
        for _ in range(n):
            reach |= {i for i in range(n) for j in reach if G[i, j] > 0}
        p = _evolve(G, 1.0, np.eye(n)[start], 3.0)
        for v in range(n):
            if v not in reach:
                assert abs(p[v]) <= 1e-13
        assert p.sum() == pytest.approx(1.0, abs=1e-12)
    g = _three()
    walk = gqsw.global_walk(g)
    rho = expmv.expmv_step(gqsw.superoperator(walk, 1.0), W.vec(W.basis_state(3, 0)), 100.0)
    assert superop.populations(rho, 3)[1] == pytest.approx(0.25, abs=1e-10)


def test_structure():
    G = W.random_digraph(6, 0.4, 11).dense()
    walk, vs = nm.nm_walk(G)
    nd = walk.n_tilde
    deg = (np.maximum(G, G.T) > 0).sum(axis=0)
    assert [len(s) for s in vs] == [max(1, d) for d in deg]
    Hd = walk.H.toarray()
    R = walk.H_rot.toarray()
    assert np.allclose(Hd, Hd.conj().T) and np.allclose(R, R.conj().T)
    assert np.allclose(Hd.sum(axis=0), 0.0)                    # trans(): zero column sums
    # copies of different vertices are coupled only along G^u edges
    Gu = np.maximum(G, G.T)
    for v in range(6):
        for u in range(6):
            if v != u and Gu[v, u] == 0:
                assert np.all(Hd[np.ix_(vs[v], vs[u])] == 0)
                assert np.all(walk.Ls[0].toarray()[np.ix_(vs[v], vs[u])] == 0)
    # the rows of L^D coming from different in-neighbours of v are orthogonal
    L = walk.Ls[0].toarray()
    for v in range(6):
        cols = [L[np.ix_(vs[v], vs[u])][:, 0] for u in range(6) if G[v, u] > 0]
        for a in range(len(cols)):
            for b in range(a + 1, len(cols)):
                assert abs(np.vdot(cols[a], cols[b])) <= 1e-12
    pops = np.arange(1, 7) / 21.0
    rho = nm.initial_state(pops, vs)
    assert np.allclose(nm.populations(np.real(np.diag(rho)), vs), pops)
