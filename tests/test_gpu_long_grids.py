"""Time grids with more outputs per Algorithm 5.2 block than a kernel keeps state for.

Algorithm 5.2 (used by the paper's `series`, Section 3.1) groups q output
times into blocks of d = floor(q / s) outputs that share the Taylor powers of
one input Z.  The series kernel keeps per-output state for 128 outputs at a
time and the batched kernel for 64: a longer block is run as several jobs that
start from the same Z, so every output gets exactly the arithmetic of the
whole block.  These grids put 200 (series) and 150 (batched) outputs in one
block and compare every output with the oracle: complex128 <= 1e-10,
complex64 bulk populations <= 1e-4.
"""
import numpy as np
import pytest

from oracle import expmv, graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    import torch
    from paper_2003_02450_gb300.walk import Context
    assert torch.cuda.is_available()
    return Context(0)


def _oracle(g, omega, rho0, t0, dt, steps, n0=None):
    walk = graph.lqsw_walk(graph.adjacency(g))
    L = superop.superoperator(walk, omega)
    stats = {}
    X = expmv.expmv_series(L, rho0, t0, dt, steps, n0=n0, stats=stats)
    return X, walk.n_tilde, stats


@pytest.mark.parametrize("operator", ["matfree", "csr"])
def test_cycle16_thousand_outputs(ctx, operator):
    # the 16-cycle on [0, 10] with 1000 output times: (m*, s) = (50, 5), so
    # Algorithm 5.2 runs 5 blocks of d = 200 outputs each
    from paper_2003_02450_gb300.walk import LQSW
    cfg = W.cycle16()
    steps, dt = 1000, 0.01
    X, nt, ost = _oracle(cfg.graph, cfg.omega, W.vec(cfg.rho0), 0.0, dt, steps)
    w = LQSW(cfg.graph, cfg.omega, ctx=ctx, operator=operator)
    w.initial_state(rho0=cfg.rho0)
    states, pops = w.series(0.0, dt, steps)
    st = w.last_stats
    assert st["outputs_per_block"] == steps // st["s"] > 128
    assert np.max(np.abs(states.cpu().numpy() - X)) <= 1e-10
    assert np.max(np.abs(pops.cpu().numpy() - superop.populations(X, nt))) <= 1e-10
    # populations only: the outputs live in a ring of d + 1 slots
    _, pops2 = w.series(0.0, dt, steps, states=False)
    assert np.array_equal(pops2.cpu().numpy(), pops.cpu().numpy())
    w.close()


def test_cycle16_thousand_outputs_c64(ctx):
    from paper_2003_02450_gb300.walk import LQSW
    cfg = W.cycle16()
    X, nt, _ = _oracle(cfg.graph, cfg.omega, W.vec(cfg.rho0), 0.0, 0.01, 1000)
    w = LQSW(cfg.graph, cfg.omega, ctx=ctx, precision="c64")
    w.initial_state(rho0=cfg.rho0)
    _, pops = w.series(0.0, 0.01, 1000, states=False)
    assert np.max(np.abs(pops.cpu().numpy() - superop.populations(X, nt))) <= 1e-4
    w.close()


@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64", 1e-4)])
def test_batched_block_of_150_outputs(ctx, precision, tol):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    walks = W.batch_regular(count=3, seed=91, nmin=8, nmax=20, rhs=2)
    n0 = 2
    ops, rhos, pops, steps, refs = [], [], [], [], []
    for g, omega, states in walks:
        B = np.stack([W.vec(s) for s in states[:n0]], axis=1)
        # a grid long enough for d = 150 outputs per block at this walk's s
        op = C.qsw_build_superoperator(ctx.handle, g, None, omega, precision=precision)
        s = C.qsw_select_params(C.qsw_op_info(ctx.handle, op)["norms"], 1.5, n0,
                                precision)[1]
        C.qsw_op_destroy(op)
        q = 150 * s
        dt = 1.5 / q
        X, nt, _ = _oracle(g, omega, B, 0.0, dt, q, n0=n0)
        refs.append(np.real(X[:, np.arange(nt) * (nt + 1), :]).transpose(0, 2, 1))
        ops.append(C.qsw_build_superoperator(ctx.handle, g, None, omega, precision=precision,
                                             defer_norms=True))
        rhos.append(torch.from_numpy(np.concatenate([W.vec(s_) for s_ in states[:n0]])).cuda())
        pops.append(torch.empty((q + 1) * n0 * g.n, dtype=torch.float64, device="cuda"))
        steps.append((q, dt))
    st = C.qsw_batch_series(ctx.handle, ops, rhos, n0, [0.0] * 3, [d for _, d in steps],
                            [q for q, _ in steps], pops)
    for o in ops:
        C.qsw_op_destroy(o)
    for (g, _, _), p, (q, _), ref in zip(walks, pops, steps, refs):
        got = p.cpu().numpy().reshape(q + 1, n0, g.n)
        assert np.max(np.abs(got - ref)) <= tol
