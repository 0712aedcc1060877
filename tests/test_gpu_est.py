"""Expected survival time on the GPU (qsw_survival_time, qsw_batch_survival_time)
against the oracle's procedure (oracle/est.py) on the same grid.

Tolerances: complex128 populations agree to <= 1e-10 (the series bound), so
eta = h/3 sum c_k (1 - p_k) agrees to <= t_end * 1e-10; complex64 bulk
populations to <= 1e-4, so eta to <= t_end * 1e-4."""
import numpy as np
import pytest

from oracle import est, graph, superop
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


def _case(n, seed, omega, scale=1.0):
    g, h = W.dipole_network(n, seed)
    g = W.Digraph(g.n, g.rowptr, g.col, g.w * scale)
    return g, h * scale, omega


def _oracle(g, h, omega, t_end, q, precision="double"):
    n = g.n
    walk = graph.lqsw_walk(graph.adjacency(g), H=h, sources=[(0, 0.5)], sinks=[(n - 1, 0.5)])
    L = superop.superoperator(walk, omega)
    rho0 = W.vec(W.basis_state(n + 2, n))
    return est.survival_time(L, n + 2, rho0, t_end, q, n + 1, precision=precision)


def _op(ctx, g, h, omega, precision="c128"):
    from paper_2003_02450_gb300 import qsw as C
    n = g.n
    return C.qsw_build_superoperator(ctx.handle, g, h, omega, sources=[(0, 0.5)],
                                     sinks=[(n - 1, 0.5)], precision=precision)


def _rho0(n):
    import torch
    return torch.from_numpy(W.vec(W.basis_state(n + 2, n))).to("cuda:0")


@pytest.mark.parametrize("n,seed,omega,scale,t_end,q", [
    (4, 3, 0.7, 1.0, 20.0, 40),
    (5, 11, 0.4, 0.5, 60.0, 120),
    (6, 21, 0.0, 0.2, 30.0, 60),
    (10, W.SEED_EST * 31, 0.5, 1.0, 8.0, 32),
])
def test_survival_time_matches_oracle(ctx, n, seed, omega, scale, t_end, q):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g, h, omega = _case(n, seed, omega, scale)
    eta_ref, pops_ref = _oracle(g, h, omega, t_end, q)
    op = _op(ctx, g, h, omega)
    pops = torch.full((q + 1, n + 2), float("nan"), dtype=torch.float64, device="cuda:0")
    eta, stats = C.qsw_survival_time(ctx.handle, op, _rho0(n), t_end, q, n + 1, pops)
    assert np.max(np.abs(pops.cpu().numpy() - pops_ref)) <= 1e-10
    assert abs(eta - eta_ref) <= t_end * 1e-10
    # without a populations buffer: the same value
    eta2, _ = C.qsw_survival_time(ctx.handle, op, _rho0(n), t_end, q, n + 1)
    assert eta2 == eta
    C.qsw_op_destroy(op)


def test_batch_survival_time_sweep(ctx):
    """A sweep over omega on two networks in one batched launch, against the
    single-walk entry point and the oracle."""
    from paper_2003_02450_gb300 import qsw as C
    nets = [_case(5, 11, 0.0, 0.5)[:2], _case(4, 3, 0.0, 1.0)[:2]]
    omegas = [0.1, 0.45, 0.9]
    t_end, q = 16.0, 40
    ops, rhos, meta = [], [], []
    for g, h in nets:
        for om in omegas:
            ops.append(_op(ctx, g, h, om))
            rhos.append(_rho0(g.n))
            meta.append((g, h, om))
    etas, stats = C.qsw_batch_survival_time(ctx.handle, ops, rhos, [t_end] * len(ops),
                                            [q] * len(ops), [g.n + 1 for g, _, _ in meta])
    assert stats["walks"] == len(ops)
    for k, (g, h, om) in enumerate(meta):
        single, _ = C.qsw_survival_time(ctx.handle, ops[k], rhos[k], t_end, q, g.n + 1)
        assert abs(etas[k] - single) <= t_end * 1e-12
        if k % 2 == 0:
            ref, _ = _oracle(g, h, om, t_end, q)
            assert abs(etas[k] - ref) <= t_end * 1e-10
    for op in ops:
        C.qsw_op_destroy(op)


def test_batch_survival_time_c64(ctx):
    from paper_2003_02450_gb300 import qsw as C
    g, h, om = _case(5, 11, 0.6, 0.5)
    t_end, q = 20.0, 40
    ops = [_op(ctx, g, h, om, "c64"), _op(ctx, g, h, om, "c128")]
    etas, _ = C.qsw_batch_survival_time(ctx.handle, ops, [_rho0(5)] * 2, [t_end] * 2, [q] * 2, [6] * 2)
    ref, _ = _oracle(g, h, om, t_end, q)
    assert abs(etas[1] - ref) <= t_end * 1e-10
    assert abs(etas[0] - ref) <= t_end * 1e-4
    for op in ops:
        C.qsw_op_destroy(op)


def test_survival_time_rejects_bad_grids(ctx):
    from paper_2003_02450_gb300 import qsw as C
    g, h, om = _case(4, 3, 0.5)
    op = _op(ctx, g, h, om)
    for t_end, q, sink in ((10.0, 3, 5), (10.0, 0, 5), (0.0, 4, 5), (10.0, 4, 6), (10.0, 4, -1)):
        with pytest.raises(C.QswError) as e:
            C.qsw_survival_time(ctx.handle, op, _rho0(4), t_end, q, sink)
        assert e.value.name == "QSW_ERR_INVALID_ARG"
    eta, _ = C.qsw_survival_time(ctx.handle, op, _rho0(4), 10.0, 4, 5)   # still usable
    assert np.isfinite(eta)
    C.qsw_op_destroy(op)


def test_full_sweep_sampled_walks(ctx):
    """The bench's sweep (4 networks x 64 omega, t_end 300, q 600) in one
    batched call; two of its walks recomputed by the oracle."""
    from paper_2003_02450_gb300 import qsw as C
    walks = W.est_dipole()
    ops = [C.qsw_build_superoperator(ctx.handle, w["graph"], w["H"], w["omega"], w["sources"],
                                     w["sinks"], defer_norms=True) for w in walks]
    rhos = [_rho0(w["graph"].n) for w in walks]
    etas, stats = C.qsw_batch_survival_time(ctx.handle, ops, rhos, [w["t_end"] for w in walks],
                                            [w["q"] for w in walks], [w["sink"] for w in walks])
    assert stats["walks"] == 256 and len(etas) == 256
    for k in (5, 64 * 3 + 40):
        w = walks[k]
        walk = graph.lqsw_walk(graph.adjacency(w["graph"]), H=w["H"], sources=w["sources"],
                               sinks=w["sinks"])
        L = superop.superoperator(walk, w["omega"])
        ref, pops = est.survival_time(L, walk.n_tilde, W.vec(w["rho0"]), w["t_end"], w["q"],
                                      w["sink"])
        assert 1.0 - pops[-1, w["sink"]] < 1e-5          # t_end covers the decay
        assert abs(etas[k] - ref) <= w["t_end"] * 1e-10
    for op in ops:
        C.qsw_op_destroy(op)
