"""Host logic of the seeded input generators (paper_2003_02450_gb300/workloads.py),
which feed both the oracle and the CUDA path: structure, seeds, and the
shapes the benchmarks rely on."""
import numpy as np
import pytest

from paper_2003_02450_gb300 import workloads as W


def _check_csr(g):
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.nnz
    assert np.all(np.diff(g.rowptr) >= 0)
    for i in range(g.n):
        cols = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)            # sorted, no duplicates
        assert np.all(cols != i)                    # simple: no self-loops
    assert np.all(g.w > 0)


def test_from_arcs_sorts_and_rejects_duplicates():
    g = W.from_arcs(4, [2, 0, 2], [1, 3, 0], [1.0, 2.0, 3.0])
    _check_csr(g)
    assert g.dense()[2, 0] == 3.0 and g.dense()[0, 3] == 2.0
    with pytest.raises(ValueError):
        W.from_arcs(3, [1, 1], [0, 0], [1.0, 1.0])


@pytest.mark.parametrize("make", [lambda: W.cycle_graph(16), lambda: W.grid_graph(5, 7),
                                  lambda: W.random_regular_graph(30, 4, 3),
                                  lambda: W.erdos_renyi_digraph(50, 0.1, 4),
                                  lambda: W.erdos_renyi_mean_degree(40, 8.0, 5),
                                  lambda: W.random_digraph(20, 0.3, 6)])
def test_generators_give_simple_csr(make):
    _check_csr(make())


def test_undirected_families_are_symmetric_with_the_stated_degrees():
    for g, deg in ((W.cycle_graph(16), 2), (W.random_regular_graph(40, 4, 9), 4)):
        A = g.dense()
        assert np.array_equal(A, A.T)
        assert np.all((A > 0).sum(axis=0) == deg)
    G = W.grid_graph(45, 45).dense()
    assert np.array_equal(G, G.T) and G.shape == (2025, 2025)
    assert sorted(set((G > 0).sum(axis=0))) == [2, 3, 4]
    assert G[22 * 45 + 22, 22 * 45 + 23] == 1.0            # vertex r*45 + c


def test_generators_are_seeded():
    a = W.erdos_renyi_digraph(60, 0.1, 17)
    b = W.erdos_renyi_digraph(60, 0.1, 17)
    c = W.erdos_renyi_digraph(60, 0.1, 18)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w)
    assert not (np.array_equal(a.col, c.col) and np.array_equal(a.w, c.w))


def test_states_are_density_matrices():
    for rho in (W.basis_state(5, 2), W.uniform_superposition(6), W.maximally_mixed(4),
                W.random_density_matrix(7, 3), W.random_pure_states(5, 1, 2)[0]):
        assert np.allclose(rho, rho.conj().T)
        assert np.trace(rho).real == pytest.approx(1.0, abs=1e-12)
        assert np.min(np.linalg.eigvalsh(rho)) >= -1e-12
    r = W.random_density_matrix(6, 1)
    assert np.array_equal(W.unvec(W.vec(r), 6), r)
    v = W.vec(W.basis_state(3, 1))
    assert v[1 + 3 * 1] == 1.0                              # column-major k = i + N j


def test_dipole_network():
    x = W.unit_ball_points(200, 5)
    assert np.all(np.linalg.norm(x, axis=1) <= 1.0)
    g, H = W.dipole_network(8, 3)
    _check_csr(g)
    A = g.dense()
    assert np.allclose(A, A.T) and np.allclose(H, H.T)
    off = ~np.eye(8, dtype=bool)
    assert np.allclose(A[off], -H[off]) and np.all(H[off] < 0) and np.all(np.diag(H) == 0)
    pts = W.unit_ball_points(8, 3)
    d = np.linalg.norm(pts[0] - pts[1])
    assert H[0, 1] == pytest.approx(-d ** -3)


def test_benchmark_configs():
    cfg = W.er1000()
    assert cfg.graph.n == 1000 and cfg.steps == 50 and cfg.dt == 0.1 and cfg.omega == 0.3
    assert cfg.rho0.shape == (1000, 1000)
    c16 = W.cycle16()
    assert c16.graph.n == 16 and c16.graph.nnz == 32
    walks = W.batch_regular(count=12)
    assert len(walks) == 12
    for g, omega, states in walks:
        assert 16 <= g.n <= 512 and 0.0 <= omega <= 1.0 and len(states) == 4
    est = W.est_dipole()
    assert len(est) == 256 and est[0]["t_end"] == 300.0 and est[0]["q"] == 600
    assert sorted({w["omega"] for w in est})[0] == pytest.approx(1 / 64)
    assert est[0]["sink"] == 11 and est[0]["rho0"][10, 10] == 1.0
    reqs = W.serve_requests(count=200)
    ns = np.array([r["n"] for r in reqs])
    assert ns.min() >= 32 and ns.max() <= 1024
    assert 0.3 < np.mean([r["precision"] == "c64" for r in reqs]) < 0.7
