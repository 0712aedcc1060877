"""Property-based checks of the oracle on random small walks (CPU; skipped
where hypothesis is not installed).  For any digraph, omega in [0, 1], ports
and density matrix rho0, the L-QSW evolution is a quantum channel:

* trace preserved, Hermiticity preserved, eigenvalues >= 0 (to rounding);
* Algorithm 5.2's series equals dense expm of t L~ (the A-H backward error);
* the row (a, b) <-> (b, a) symmetry of L~ (Hermiticity preservation) and the
  vanishing column sums of L~ over the diagonal rows (trace preservation)."""
import numpy as np
import pytest
import scipy.linalg as sl

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import expmv, graph, superop  # noqa: E402
from paper_2003_02450_gb300 import workloads as W  # noqa: E402


@st.composite
def walks(draw):
    n = draw(st.integers(2, 6))
    p = draw(st.floats(0.2, 1.0))
    seed = draw(st.integers(0, 10_000))
    omega = draw(st.sampled_from([0.0, 1.0]) | st.floats(0.0, 1.0))
    g = W.random_digraph(n, p, seed)
    src = [(draw(st.integers(0, n - 1)), draw(st.floats(0.1, 2.0)))] if draw(st.booleans()) else []
    snk = [(draw(st.integers(0, n - 1)), draw(st.floats(0.1, 2.0)))] if draw(st.booleans()) else []
    walk = graph.lqsw_walk(graph.adjacency(g), sources=src, sinks=snk)
    rho0 = W.random_density_matrix(walk.n_tilde, seed + 1, rank=draw(st.integers(1, 3)))
    return walk, omega, rho0


@settings(max_examples=40, deadline=None)
@given(walks(), st.floats(0.05, 3.0))
def test_evolution_is_a_channel(w, t):
    walk, omega, rho0 = w
    nt = walk.n_tilde
    L = superop.superoperator(walk, omega)
    X = expmv.expmv_series(L, W.vec(rho0), 0.0, t / 4, 4)
    E = sl.expm(t * L.toarray()) @ W.vec(rho0)
    assert np.max(np.abs(X[-1] - E)) <= 1e-12
    for x in X:
        R = x.reshape(nt, nt, order="F")
        assert abs(np.trace(R) - 1.0) <= 1e-12
        assert np.max(np.abs(R - R.conj().T)) <= 1e-12
        assert np.min(np.linalg.eigvalsh((R + R.conj().T) / 2)) >= -1e-12


@settings(max_examples=40, deadline=None)
@given(walks())
def test_superoperator_structure(w):
    walk, omega, _ = w
    nt = walk.n_tilde
    L = superop.superoperator(walk, omega).toarray()
    diag_rows = [i + nt * i for i in range(nt)]
    assert np.max(np.abs(L[diag_rows, :].sum(axis=0)), initial=0.0) <= 1e-12
    k = np.arange(nt * nt)
    sw = (k // nt) + nt * (k % nt)                 # (i, j) -> (j, i)
    assert np.allclose(L[np.ix_(sw, sw)], L.conj(), rtol=0, atol=1e-14)
