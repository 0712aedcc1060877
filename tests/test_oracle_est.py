"""Pins of the oracle's expected-survival-time procedure (oracle/est.py)."""
import numpy as np
import pytest
import scipy.integrate
import scipy.sparse as sp

from oracle import est, graph, superop
from paper_2003_02450_gb300 import workloads as W


def test_simpson_exact_on_cubics():
    # Simpson's rule integrates polynomials of degree <= 3 exactly
    f = lambda x: 2.0 * x ** 3 - 3.0 * x ** 2 + 0.5 * x + 1.25
    F = lambda x: 0.5 * x ** 4 - x ** 3 + 0.25 * x ** 2 + 1.25 * x
    for q, a, b in ((2, 0.0, 1.0), (4, -1.0, 2.0), (10, 0.3, 7.1)):
        x = np.linspace(a, b, q + 1)
        assert est.simpson(f(x), (b - a) / q) == pytest.approx(F(b) - F(a), rel=1e-13, abs=1e-13)


def test_simpson_matches_scipy():
    rng = np.random.default_rng(5)
    for q in (2, 6, 100, 1000):
        y = rng.standard_normal(q + 1)
        h = 0.37
        ref = scipy.integrate.simpson(y, dx=h)
        assert est.simpson(y, h) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_simpson_rejects_odd_q():
    with pytest.raises(ValueError):
        est.simpson(np.ones(4), 0.1)


def _dipole_walk(n, seed, scale=1.0):
    g, h = W.dipole_network(n, seed)
    g = W.Digraph(g.n, g.rowptr, g.col, g.w * scale)
    return graph.lqsw_walk(graph.adjacency(g), H=h * scale, sources=[(0, 0.5)],
                           sinks=[(n - 1, 0.5)])


def test_limit_equals_classical_absorption_time_at_omega_one():
    """At omega = 1 the populations follow the classical master equation
    dp/dt = Q p (rates G_ij plus the port rates); the expected time to
    absorption in the sink is 1^T (-Q_TT)^-1 p0_T over the transient states."""
    for n, seed in ((4, 1), (6, 2), (10, W.SEED_EST * 31)):
        walk = _dipole_walk(n, seed)
        nt = walk.n_tilde
        Q = np.zeros((nt, nt))
        for jmp in walk.jumps:
            Q[jmp.i, jmp.j] += jmp.tau * jmp.amp ** 2
        Q -= np.diag(Q.sum(axis=0))
        sink = nt - 1
        T = [v for v in range(nt) if v != sink]
        p0 = np.zeros(nt)
        p0[n] = 1.0                                       # the source vertex
        tau = np.ones(len(T)) @ np.linalg.solve(-Q[np.ix_(T, T)], p0[T])
        L = superop.superoperator(walk, 1.0)
        rho0 = W.vec(W.basis_state(nt, n))
        assert est.survival_time_limit(L, nt, rho0, sink) == pytest.approx(tau, rel=1e-10)


@pytest.mark.parametrize("omega", [0.4, 1.0])
def test_procedure_converges_to_limit(omega):
    """Simpson on the series populations approaches the integral to infinity
    with the rule's h^4 order when t_end covers the decay (couplings scaled by
    0.5 so that the slowest decay rate is ~0.06 and h = 0.25 resolves the
    coherent oscillations)."""
    walk = _dipole_walk(5, 11, scale=0.5)
    nt = walk.n_tilde
    L = superop.superoperator(walk, omega)
    rho0 = W.vec(W.basis_state(nt, 5))
    limit = est.survival_time_limit(L, nt, rho0, nt - 1)
    eta_h, _ = est.survival_time(L, nt, rho0, 600.0, 1200, nt - 1)
    eta_h2, pops = est.survival_time(L, nt, rho0, 600.0, 2400, nt - 1)
    assert abs(1.0 - pops[-1, nt - 1]) < 1e-12
    assert eta_h2 == pytest.approx(limit, rel=1e-7)
    ratio = abs(eta_h - limit) / abs(eta_h2 - limit)
    assert 12.0 < ratio < 20.0          # halving h divides the error by ~2^4
