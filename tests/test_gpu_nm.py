"""NM-G-QSW on the GPU (qsw_build_nm_gqsw) against the oracle's independent
demoralisation (oracle/nm.py): the operator (applications to random vectors),
the vertex subspaces, the printed Section 4.1.2 example and series with the
population map of Eq. nm_rho_map."""
import numpy as np
import pytest

from oracle import expmv, gqsw, nm, superop
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


def _dev(v, dtype=None):
    import torch
    a = np.ascontiguousarray(v)
    return torch.from_numpy(a).to("cuda:0")


def _three():
    G = np.zeros((3, 3))
    G[2, 0] = G[2, 1] = 1.0
    return G


GRAPHS = [("three", None), ("rand6", 21), ("rand9", 5), ("cycle5", None)]


def _graph(name, seed):
    if name == "three":
        return _three()
    if name == "cycle5":
        return W.cycle_graph(5).dense()
    n = int(name[4:])
    return W.random_digraph(n, 0.35, seed).dense()


@pytest.mark.parametrize("name,seed", GRAPHS)
@pytest.mark.parametrize("omega", [0.0, 0.45, 1.0])
def test_operator_matches_oracle(ctx, name, seed, omega):
    from paper_2003_02450_gb300 import qsw as C
    G = _graph(name, seed)
    op = C.qsw_build_nm_gqsw(ctx.handle, W.from_dense(G), omega)
    walk, vs = nm.nm_walk(G)
    off = C.qsw_nm_vsets(ctx.handle, op, G.shape[0])
    assert list(off) == [int(s[0]) for s in vs] + [walk.n_tilde]
    L = gqsw.superoperator(walk, omega)
    nd = walk.n_tilde
    rng = np.random.default_rng(7)
    for trial in range(2):
        x = rng.standard_normal(nd * nd) + 1j * rng.standard_normal(nd * nd)
        y = _dev(np.zeros(nd * nd, complex))
        C.qsw_apply(ctx.handle, op, _dev(x), y)
        ref = L @ x
        assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    info = C.qsw_op_info(ctx.handle, op)
    assert info["n_tilde"] == nd
    assert info["norms"][0] == pytest.approx(abs(L).sum(axis=0).max(), rel=1e-12)
    C.qsw_op_destroy(op)


def _run(ctx, G, omega, pops0, t0, dt, steps):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    op = C.qsw_build_nm_gqsw(ctx.handle, W.from_dense(G), omega)
    nd = C.qsw_op_info(ctx.handle, op)["n_tilde"]
    state = torch.empty(nd * nd, dtype=torch.complex128, device="cuda:0")
    C.qsw_nm_initial_state(ctx.handle, op, pops0, state)
    pe = torch.empty((steps + 1, nd), dtype=torch.float64, device="cuda:0")
    C.qsw_expmv_series(ctx.handle, op, state, t0, dt, steps, None, pe)
    p = torch.empty((steps + 1, G.shape[0]), dtype=torch.float64, device="cuda:0")
    C.qsw_nm_populations(ctx.handle, op, pe, steps + 1, p)
    C.qsw_op_destroy(op)
    return state.cpu().numpy(), p.cpu().numpy()


def test_paper_example_gpu(ctx):
    """Section 4.1.2: [3.72007598e-44, 0, 1] at omega = 1 and
    [3.80773381e-07, 9.98766244e-01, 1.23337485e-03] at omega = 0 (t = 100)."""
    _, p1 = _run(ctx, _three(), 1.0, [1.0, 0.0, 0.0], 100.0, 0.0, 0)
    assert p1[0, 0] == pytest.approx(3.72007598e-44, rel=1e-6)
    assert abs(p1[0, 1]) <= 1e-14 and p1[0, 2] == pytest.approx(1.0, abs=1e-12)
    _, p0 = _run(ctx, _three(), 0.0, [1.0, 0.0, 0.0], 100.0, 0.0, 0)
    assert p0[0, 0] == pytest.approx(3.80773381e-07, abs=1e-12)
    assert p0[0, 1] == pytest.approx(9.98766244e-01, abs=5e-9)
    assert p0[0, 2] == pytest.approx(1.23337485e-03, abs=5e-11)


@pytest.mark.parametrize("name,seed", GRAPHS[1:])
def test_series_matches_oracle(ctx, name, seed):
    G = _graph(name, seed)
    n = G.shape[0]
    pops0 = np.random.default_rng(3).random(n)
    pops0 /= pops0.sum()
    state, p = _run(ctx, G, 0.6, pops0, 0.5, 0.25, 12)
    walk, vs = nm.nm_walk(G)
    rho0 = nm.initial_state(pops0, vs)
    assert np.max(np.abs(state - W.vec(rho0))) == 0.0
    L = gqsw.superoperator(walk, 0.6)
    ref = expmv.expmv_series(L, W.vec(rho0), 0.5, 0.25, 12)
    pref = nm.populations(superop.populations(ref, walk.n_tilde), vs)
    assert np.max(np.abs(p - pref)) <= 1e-10
    assert np.allclose(p.sum(axis=1), 1.0, atol=1e-12)


def test_bench_config_first_output_full_size(ctx):
    """The NM-G-QSW bench walk (ER N = 60, p = 0.06, 424 copies, omega = 0.3,
    uniform vertex populations): the populations at t = 0.1 against the oracle."""
    g = W.erdos_renyi_digraph(60, 0.06, W.SEED_ER1000 + 2)
    G = g.dense()
    pops0 = np.full(60, 1.0 / 60)
    _, p = _run(ctx, G, 0.3, pops0, 0.0, 0.1, 1)
    walk, vs = nm.nm_walk(G)
    assert walk.n_tilde == 424
    L = gqsw.superoperator(walk, 0.3)
    ref = expmv.expmv_series(L, W.vec(nm.initial_state(pops0, vs)), 0.0, 0.1, 1)
    pref = nm.populations(superop.populations(ref, walk.n_tilde), vs)
    assert np.max(np.abs(p - pref)) <= 1e-10
