"""The identities the GPU 1-norm estimator relies on to share work, checked on
the oracle's superoperators (CPU, no GPU):

* L~ and L~^H map X^dag to (L~ X)^dag (every term of the master equation does),
  so column (a, b) of L~^p is column (b, a) conjugate-transposed: equal norms,
  which is what lets a unit-vector pair e_(a,b), e_(b,a) cost one column;
* the box rule: a vector supported on rows I x columns J maps to one supported
  on I' x J' with I' = I + {i : row i of H meets I} + T, J' likewise, T the
  targets of jumps whose source q lies in I and J (for L~^H: jumps reversed);
* for L-QSW and global walks alike, the all-ones matrix is Hermitian, so the
  starting block's first column stays Hermitian under every power."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gqsw, graph, superop
from paper_2003_02450_gb300 import workloads as W


def _lqsw(kind, omega, sources=(), sinks=()):
    g = {"grid": W.grid_graph(4, 5), "er": W.random_digraph(11, 0.3, 5),
         "cycle": W.cycle_graph(9)}[kind]
    walk = graph.lqsw_walk(graph.adjacency(g), sources=sources, sinks=sinks)
    return walk, superop.superoperator(walk, omega).tocsr()


def _dag(v, nt):
    return v.reshape(nt, nt, order="F").conj().T.reshape(-1, order="F")


CASES = [("grid", 0.3, [(0, 0.7)], [(19, 1.1)]), ("er", 0.0, [(2, 0.5)], []),
         ("er", 1.0, [], [(4, 0.9)]), ("cycle", 0.55, [], [])]


@pytest.mark.parametrize("kind,omega,src,snk", CASES)
def test_hermiticity_preservation_and_transposed_columns(kind, omega, src, snk):
    walk, L = _lqsw(kind, omega, src, snk)
    nt = walk.n_tilde
    LH = L.conj().T.tocsr()
    rng = np.random.default_rng(3)
    for M in (L, LH):
        x = rng.standard_normal(nt * nt) + 1j * rng.standard_normal(nt * nt)
        assert np.allclose(M @ _dag(x, nt), _dag(M @ x, nt), rtol=0, atol=1e-12)
    P = sp.identity(nt * nt, format="csr", dtype=complex)
    for _ in range(3):
        P = (L @ P).tocsr()
    cols = np.asarray(abs(P).sum(axis=0)).ravel()
    a, b = np.divmod(np.arange(nt * nt), nt)       # index k = b + nt a -> (row b, column a)
    swapped = a + nt * b
    assert np.allclose(cols, cols[swapped], rtol=1e-13, atol=0)


def _grow(I, J, Hs, into):
    I2 = I | ((Hs @ I.astype(int)) > 0)
    J2 = J | ((Hs @ J.astype(int)) > 0)
    both = I & J
    T = np.array([any(both[q] for q in into[v]) for v in range(len(I))])
    return I2 | T, J2 | T


@pytest.mark.parametrize("kind,omega,src,snk", CASES)
def test_box_rule_contains_the_support(kind, omega, src, snk):
    walk, L = _lqsw(kind, omega, src, snk)
    nt = walk.n_tilde
    LH = L.conj().T.tocsr()
    Hoff = sp.csr_matrix(walk.H)
    Hoff.setdiag(0)
    Hoff.eliminate_zeros()
    Hs = (abs(Hoff) > 0).astype(int) if omega < 1.0 else sp.csr_matrix((nt, nt), dtype=int)
    fwd = [[] for _ in range(nt)]
    adj = [[] for _ in range(nt)]
    for jp in walk.jumps:
        if jp.tau * (omega if jp.omega_scaled else 1.0) == 0.0:
            continue
        fwd[jp.i].append(jp.j)   # jump j -> i feeds (i, i) from (j, j)
        adj[jp.j].append(jp.i)
    rng = np.random.default_rng(7)
    for M, into in ((L, fwd), (LH, adj)):
        for c in rng.integers(0, nt * nt, 12):
            x = np.zeros(nt * nt, complex)
            x[c] = 1.0
            I = np.zeros(nt, bool)
            J = np.zeros(nt, bool)
            I[c % nt] = True
            J[c // nt] = True
            for _ in range(5):
                x = M @ x
                I, J = _grow(I, J, Hs, into)
                inside = np.zeros((nt, nt), bool)
                inside[np.ix_(I, J)] = True
                assert not np.any(x.reshape(nt, nt, order="F")[~inside])


def test_global_walk_preserves_hermiticity():
    g = W.random_digraph(8, 0.3, 8)
    walk = gqsw.global_walk(g.dense(), sources=[(0, 0.4)], sinks=[(7, 0.6)])
    L = gqsw.superoperator(walk, 0.45).tocsr()
    nt = walk.n_tilde
    x = np.random.default_rng(2).standard_normal(nt * nt) + 0j
    x = x + _dag(x, nt)                             # Hermitian
    y = L @ x
    assert np.allclose(y, _dag(y, nt), rtol=0, atol=1e-12)
    ones = np.ones(nt * nt, complex)
    for M in (L, L.conj().T.tocsr()):
        z = ones
        for _ in range(3):
            z = M @ z
            assert np.allclose(z, _dag(z, nt), rtol=0, atol=1e-10 * np.abs(z).max())
