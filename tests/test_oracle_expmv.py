"""Pins for oracle/expmv.py (Algorithms 3.2 and 5.2, Code Fragment 3.1).

Independent references: scipy.linalg.expm on the dense superoperator, the
values printed in the paper's Section 4 example (tests/golden), the omega = 0
CTQW and omega = 1 CTRW limits solved in the N x N vertex space
(tests/pins.py), density-matrix invariants (Section 2.4) and SciPy's own
implementation of the same Al-Mohy--Higham algorithm.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

from oracle import expmv, graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_example_lqsw.txt")


def _walk(g, omega, **kw):
    walk = graph.lqsw_walk(graph.adjacency(g), **kw)
    return walk, superop.superoperator(walk, omega)


def test_paper_example_printed_populations():
    G = sp.csr_matrix(([1.0, 1.0], ([2, 2], [0, 1])), shape=(3, 3))
    GU = sp.csr_matrix(([1.0, 1, 1, 1], ([0, 1, 2, 2], [2, 2, 0, 1])), shape=(3, 3))
    rows = np.loadtxt(GOLDEN)
    for omega, t, *printed in rows:
        walk = graph.lqsw_walk(G, H=GU)
        L = superop.superoperator(walk, omega)
        x = expmv.expmv_step(L, W.vec(W.basis_state(3, 0)), t)
        p = superop.populations(x, 3)
        # printed to 9 significant digits (half a unit: 5e-9 relative) plus the
        # paper's accuracy bound of 1e-10
        printed = np.array(printed)
        assert np.all(np.abs(p - printed) <= 5e-9 * np.abs(printed) + 1e-10), (omega, p, printed)


@pytest.mark.parametrize("seed,omega,t", [(1, 0.5, 0.3), (2, 0.1, 2.0), (3, 0.9, 7.5),
                                          (4, 0.0, 12.0), (5, 1.0, 40.0)])
def test_step_matches_dense_expm(seed, omega, t):
    g = W.random_digraph(5, 0.5, seed)
    walk, L = _walk(g, omega, sources=[(0, 0.5)], sinks=[(4, 0.7)])
    rho0 = W.vec(W.random_density_matrix(walk.n_tilde, seed))
    ref = sl.expm(t * L.toarray()) @ rho0
    got = expmv.expmv_step(L, rho0, t)
    assert np.max(np.abs(got - ref)) <= 1e-12


@pytest.mark.parametrize("q,dt", [(3, 4.0), (10, 0.25), (37, 0.2), (60, 0.05)])
def test_series_matches_dense_expm(q, dt):
    # covers q <= s (stepwise branch) and q > s with and without remainder block
    g = W.random_digraph(4, 0.6, 9)
    walk, L = _walk(g, 0.6)
    rho0 = W.vec(W.random_density_matrix(4, 1))
    st = {}
    X = expmv.expmv_series(L, rho0, 0.5, dt, q, stats=st)
    Ld = L.toarray()
    for k in range(q + 1):
        ref = sl.expm((0.5 + k * dt) * Ld) @ rho0
        assert np.max(np.abs(X[k] - ref)) <= 1e-12, (k, st)


def test_series_branches_exercised():
    g = W.random_digraph(4, 0.6, 9)
    _, L = _walk(g, 0.6)
    info = expmv.NormInfo(L)
    # q <= s, q > s with r = 0, q > s with r != 0
    seen = set()
    for q, dt in [(3, 4.0), (10, 0.25), (37, 0.2)]:
        m, s = expmv.select_params(info, q * dt)
        d = q // s if q > s else 0
        seen.add("step" if q <= s else ("exact" if q % d == 0 else "remainder"))
    assert seen == {"step", "exact", "remainder"}


def test_step_and_series_agree():
    # Section 5: `step` and `series` agree to ~1e-14
    cfg = W.cycle16()
    walk, L = _walk(cfg.graph, cfg.omega)
    rho0 = W.vec(cfg.rho0)
    X = expmv.expmv_series(L, rho0, 0.0, 0.5, 20)
    for k in (1, 7, 20):
        assert np.max(np.abs(X[k] - expmv.expmv_step(L, rho0, 0.5 * k))) <= 1e-13


def test_ctqw_limit_omega0():
    g = W.erdos_renyi_digraph(30, 0.12, 77)
    walk, L = _walk(g, 0.0)
    rho0 = W.uniform_superposition(30)
    for t in (0.7, 5.0):
        got = W.unvec(expmv.expmv_step(L, W.vec(rho0), t), 30)
        ref = pins.ctqw_density(pins.laplacian_of_undirected(g.dense()), rho0, t)
        assert np.max(np.abs(got - ref)) <= 1e-12
        assert abs(np.trace(got @ got).real - 1.0) <= 1e-12   # stays pure


def test_ctrw_limit_omega1():
    g = W.erdos_renyi_digraph(20, 0.15, 78)
    G = g.dense()
    walk, L = _walk(g, 1.0)
    rho0 = W.random_density_matrix(20, 5, rank=4)
    t = 1.3
    got = W.unvec(expmv.expmv_step(L, W.vec(rho0), t), 20)
    p_ref = pins.ctrw_populations(G, np.real(np.diag(rho0)), t)
    assert np.max(np.abs(np.real(np.diag(got)) - p_ref)) <= 1e-12
    d = G.sum(axis=0)
    decay = np.exp(-0.5 * (d[:, None] + d[None, :]) * t)
    off = ~np.eye(20, dtype=bool)
    assert np.max(np.abs(got[off] - (decay * rho0)[off])) <= 1e-12


@pytest.mark.parametrize("omega", [0.2, 0.5, 0.85])
def test_density_matrix_invariants(omega):
    g = W.erdos_renyi_digraph(15, 0.2, 31)
    walk, L = _walk(g, omega)
    rho0 = W.random_pure_states(15, 1, 4)[0]
    X = expmv.expmv_series(L, W.vec(rho0), 0.0, 0.4, 12)
    purity_prev = 1.0 + 1e-12
    for k in range(13):
        r = W.unvec(X[k], 15)
        assert abs(np.trace(r) - 1.0) <= 1e-12
        assert np.max(np.abs(r - r.conj().T)) <= 1e-13
        assert np.min(np.linalg.eigvalsh((r + r.conj().T) / 2)) >= -1e-12
        pur = np.trace(r @ r).real
        assert pur <= 1.0 + 1e-12


def test_regular_graph_steady_state_has_no_coherence():
    # Section 4 example 2: the cycle (a regular graph) relaxes to I/N.
    cfg = W.cycle16()
    _, L = _walk(cfg.graph, 0.5)
    x = expmv.expmv_step(L, W.vec(cfg.rho0), 200.0)
    assert np.max(np.abs(W.unvec(x, 16) - np.eye(16) / 16)) <= 1e-9


def test_matches_scipy_expm_multiply():
    spl = pytest.importorskip("scipy.sparse.linalg")
    cfg = W.cycle16()
    _, L = _walk(cfg.graph, cfg.omega)
    rho0 = W.vec(cfg.rho0)
    X = expmv.expmv_series(L, rho0, cfg.t0, cfg.dt, cfg.steps)
    ref = spl.expm_multiply(L, rho0, start=cfg.t0, stop=cfg.t0 + cfg.steps * cfg.dt,
                            num=cfg.steps + 1, endpoint=True)
    assert np.max(np.abs(X - ref)) <= 1e-13


def test_params_match_scipy_choice_small_norm_branch():
    # With SciPy's theta subset, Code Fragment 3.1 on the 16-cycle over
    # [0, 10] (||tL||_1 = 40: condition (3.13) holds) must give SciPy's (m, s).
    mod = pytest.importorskip("scipy.sparse.linalg._expm_multiply")
    cfg = W.cycle16()
    _, L = _walk(cfg.graph, cfg.omega)
    info = expmv.NormInfo(L)
    t = cfg.steps * cfg.dt
    ref_norm = mod.LazyOperatorNormInfo(t * L, A_1_norm=t * info.one, ell=2)
    ref = mod._fragment_3_1(ref_norm, 1, 2.0 ** -53, ell=2)
    assert expmv.select_params(info, t, 1, theta=mod._theta) == tuple(ref) == (50, 5)


def test_params_zero_norm():
    info = expmv.NormInfo(sp.csr_matrix((4, 4), dtype=complex))
    assert expmv.select_params(info, 3.0) == (0, 1)
    x = np.arange(4, dtype=complex)
    assert np.array_equal(expmv.expmv_step(sp.csr_matrix((4, 4), dtype=complex), x, 3.0), x)
