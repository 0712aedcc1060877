"""Pins for oracle/graph.py and oracle/superop.py.

The oracle forms L~ from explicit Kronecker products; here it is checked
against (a) a brute-force construction that applies the master equation to
every basis matrix |m><l| with dense products (tests/pins.py), (b) the nnz
closed form of the L-QSW structure and (c) trace preservation.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests import pins


CASES = [
    # (N, arc probability, seed, omega, sources, sinks, explicit H?)
    (2, 1.0, 1, 0.5, [], [], False),
    (3, 0.5, 2, 0.0, [], [], False),
    (4, 0.4, 3, 1.0, [], [], False),
    (5, 0.5, 4, 0.37, [], [], True),
    (4, 0.6, 5, 0.8, [(0, 2.0)], [(1, 3.0)], False),
    (6, 0.3, 6, 0.25, [(2, 0.5)], [(5, 0.5), (0, 1.5)], True),
]


def _case(N, p, seed, explicit_h):
    g = W.random_digraph(N, p, seed)
    G = g.dense()
    H = None
    if explicit_h:
        rng = np.random.default_rng(seed + 1000)
        a = rng.standard_normal((N, N))
        H = (a + a.T) * (rng.random((N, N)) < 0.6)
        H = (H + H.T) / 2
    return g, G, H


@pytest.mark.parametrize("N,p,seed,omega,sources,sinks,explicit_h", CASES)
def test_superoperator_matches_brute_force(N, p, seed, omega, sources, sinks, explicit_h):
    g, G, H = _case(N, p, seed, explicit_h)
    walk = graph.lqsw_walk(graph.adjacency(g), H=None if H is None else sp.csr_matrix(H),
                           sources=sources, sinks=sinks)
    L = superop.superoperator(walk, omega).toarray()
    nt = walk.n_tilde
    Hd = pins.laplacian_of_undirected(G) if H is None else H
    Hx = np.zeros((nt, nt))
    Hx[:N, :N] = Hd
    ref = pins.brute_force_superoperator(Hx, pins.dense_jumps(G, sources, sinks), omega)
    assert np.max(np.abs(L - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


def test_default_hamiltonian_is_laplacian_of_undirected_companion():
    g = W.random_digraph(7, 0.35, 11)
    G = g.dense()
    walk = graph.lqsw_walk(graph.adjacency(g))
    assert np.array_equal(walk.H.toarray(), pins.laplacian_of_undirected(G))


def test_out_degree_is_column_sum():
    g = W.random_digraph(9, 0.3, 12)
    G = g.dense()
    assert np.allclose(graph.out_degree(graph.adjacency(g)), G.sum(axis=0), rtol=0, atol=1e-15)


def test_rejects_self_loops():
    G = sp.csr_matrix(np.array([[1.0, 0], [1, 0]]))
    with pytest.raises(ValueError):
        graph.lqsw_walk(G)


def _nnz_closed_form(walk, G):
    # n + 2 N~ nnz_off(H) + (number of jump operators): diagonal rows/cols of
    # the structure (Section 3.2: block diagonal I(x)H, stripes H^T(x)I, and one
    # entry (i,i),(j,j) per jump operator).
    H = walk.H.tocoo()
    off = int(np.sum(H.row != H.col))
    return walk.n_tilde ** 2 + 2 * walk.n_tilde * off + len(walk.jumps)


def test_nnz_closed_form_cycle16():
    cfg = W.cycle16()
    walk = graph.lqsw_walk(graph.adjacency(cfg.graph))
    L = superop.superoperator(walk, cfg.omega)
    assert L.nnz == 1312 == _nnz_closed_form(walk, cfg.graph.dense())


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_nnz_closed_form_random(seed):
    g = W.erdos_renyi_digraph(25, 0.15, seed)
    walk = graph.lqsw_walk(graph.adjacency(g), sources=[(0, 1.0)], sinks=[(3, 2.0)])
    L = superop.superoperator(walk, 0.4)
    # the oracle drops exact zeros; a vertex with no outgoing jump (the sink)
    # has a zero diagonal entry in row (i, i)
    zero_diag = int(np.sum(L.diagonal() == 0))
    assert L.nnz + zero_diag == _nnz_closed_form(walk, g.dense())


@pytest.mark.parametrize("omega", [0.0, 0.3, 1.0])
def test_trace_preserving_columns(omega):
    # d/dt Tr rho = 0 for every rho  <=>  sum_i L~[(i,i), c] = 0 for every column c.
    g = W.erdos_renyi_digraph(12, 0.3, 5)
    walk = graph.lqsw_walk(graph.adjacency(g), sources=[(1, 0.7)], sinks=[(2, 0.9)])
    L = superop.superoperator(walk, omega)
    nt = walk.n_tilde
    diag_rows = np.arange(nt) * (nt + 1)
    colsum = np.asarray(L[diag_rows, :].sum(axis=0)).ravel()
    assert np.max(np.abs(colsum)) <= 1e-14


def test_populations_reads_diagonal():
    rho = W.random_density_matrix(5, 3)
    assert np.allclose(superop.populations(W.vec(rho), 5), np.real(np.diag(rho)), atol=0)
