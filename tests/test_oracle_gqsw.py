"""Pins of the G-QSW oracle (oracle/gqsw.py)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import expmv, gqsw, superop
from paper_2003_02450_gb300 import workloads as W
from tests import pins


def _random_case(n, seed, ports=True):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < 0.5) * rng.uniform(0.5, 1.5, (n, n))
    np.fill_diagonal(A, 0.0)
    Hc = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Hc = Hc + Hc.conj().T
    Ls = [A, rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))]
    src = [(0, 0.7)] if ports else []
    snk = [(n - 1, 1.3)] if ports else []
    return A, Hc, Ls, src, snk


def _dense_list(walk):
    nt = walk.n_tilde
    out = [(L.toarray(), 1.0, True) for L in walk.Ls]
    for j in walk.ports:
        M = np.zeros((nt, nt), complex)
        M[j.i, j.j] = j.amp
        out.append((M, j.tau, False))
    return out


@pytest.mark.parametrize("n,seed,omega,ports", [(3, 1, 0.0, False), (3, 2, 1.0, True),
                                                (4, 3, 0.35, True), (5, 4, 0.8, False)])
def test_superoperator_matches_master_equation(n, seed, omega, ports):
    A, Hc, Ls, src, snk = _random_case(n, seed, ports)
    walk = gqsw.global_walk(A, H=Hc, Ls=Ls, sources=src, sinks=snk)
    rot = np.zeros((walk.n_tilde, walk.n_tilde), complex)
    rot[:n, :n] = np.triu(np.ones((n, n)), 1) * 1j
    rot = rot + rot.conj().T
    walk.H_rot = sp.csr_matrix(rot)
    got = gqsw.superoperator(walk, omega).toarray()
    ref = pins.brute_force_superoperator(walk.H.toarray(), _dense_list(walk), omega, h_rot=rot)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_default_operators_are_laplacian_and_adjacency():
    G = W.random_digraph(6, 0.4, 9).dense()
    walk = gqsw.global_walk(G)
    assert np.allclose(walk.Ls[0].toarray(), G)
    assert np.allclose(walk.H.toarray(), pins.laplacian_of_undirected(G))


def test_trace_preserving():
    A, Hc, Ls, src, snk = _random_case(4, 7)
    walk = gqsw.global_walk(A, H=Hc, Ls=Ls, sources=src, sinks=snk)
    L = gqsw.superoperator(walk, 0.6).toarray()
    nt = walk.n_tilde
    diag_rows = np.arange(nt) * (nt + 1)
    assert np.max(np.abs(L[diag_rows].sum(axis=0))) <= 1e-12


def test_omega_zero_is_ctqw():
    G = W.cycle_graph(7).dense()
    walk = gqsw.global_walk(G)
    rho0 = W.basis_state(7, 2)
    L = gqsw.superoperator(walk, 0.0)
    got = expmv.expmv_step(L, W.vec(rho0), 3.0)
    ref = pins.ctqw_density(walk.H.toarray(), rho0, 3.0)
    assert np.max(np.abs(got - W.vec(ref))) <= 1e-12


def test_paper_three_vertex_example():
    """Section 4.1.2: two vertices feeding a common sink (arcs v1 -> v3 and
    v2 -> v3), H = trans(1, GU), L = [G], omega = 1, rho(0) = |v1><v1|: at
    t = 100 the printed populations are [0.25, 0.25, 0.5] (spontaneous
    moralisation: half of |v1> is the dark state (|v1> - |v2>)/sqrt 2)."""
    G = np.zeros((3, 3))
    G[2, 0] = G[2, 1] = 1.0
    walk = gqsw.global_walk(G)
    L = gqsw.superoperator(walk, 1.0)
    rho = expmv.expmv_step(L, W.vec(W.basis_state(3, 0)), 100.0)
    pops = superop.populations(rho, 3)
    assert np.allclose(pops, [0.25, 0.25, 0.5], atol=1e-10)
