"""Batched walks (one cluster per walk, many walks per launch) vs the oracle.

The oracle evolves each walk's n0 right-hand sides as one n x n0 block
(Algorithms 3.2/5.2 on a block, ||.||_inf = largest row sum of moduli).
Tolerances: complex128 1e-10 (states/populations), complex64 bulk 1e-4
(populations).  "Alone and in the mix": a walk's populations from a batch equal
those from a single-walk call within the tolerance.
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


def _oracle_pops(g, omega, states, t0, dt, steps):
    walk = graph.lqsw_walk(graph.adjacency(g))
    L = superop.superoperator(walk, omega)
    B = np.stack([W.vec(s) for s in states], axis=1)          # n x n0
    X = expmv.expmv_series(L, B, t0, dt, steps, n0=B.shape[1])  # (q+1) x n x n0
    nt = walk.n_tilde
    idx = np.arange(nt) * (nt + 1)
    return np.real(X[:, idx, :]).transpose(0, 2, 1)            # (q+1) x n0 x nt


def _run_batch(ctx, walks, n0, t0s, dts, steps, precision):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    ops, rhos, pops = [], [], []
    for (g, omega, states), q in zip(walks, steps):
        ops.append(C.qsw_build_superoperator(ctx.handle, g, None, omega, precision=precision,
                                             defer_norms=True))
        B = np.concatenate([W.vec(s) for s in states[:n0]])
        rhos.append(torch.from_numpy(B).cuda())
        pops.append(torch.empty((q + 1) * n0 * g.n, dtype=torch.float64, device="cuda"))
    st = C.qsw_batch_series(ctx.handle, ops, rhos, n0, t0s, dts, steps, pops)
    out = [p.cpu().numpy().reshape(q + 1, n0, g.n) for p, q, (g, _, _) in zip(pops, steps, walks)]
    for o in ops:
        C.qsw_op_destroy(o)
    return out, st


@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64", 1e-4)])
@pytest.mark.parametrize("n0", [1, 4])
def test_small_regular_batch_matches_oracle(ctx, precision, tol, n0):
    walks = W.batch_regular(count=10, seed=77, nmin=6, nmax=24, rhs=4)
    steps = [10] * len(walks)
    got, st = _run_batch(ctx, walks, n0, [0.0] * len(walks), [0.2] * len(walks), steps, precision)
    assert st["walks"] == len(walks)
    for (g, omega, states), p in zip(walks, got):
        ref = _oracle_pops(g, omega, states[:n0], 0.0, 0.2, 10)
        assert np.max(np.abs(p - ref)) <= tol


def test_mixed_grids_and_sizes_match_single_walk(ctx):
    # different t0 / dt / steps per walk (serving-like), n0 = 1, complex128;
    # each walk's result must equal the single-walk call on the same input
    import torch
    from paper_2003_02450_gb300.walk import LQSW
    rng = np.random.default_rng(5)
    walks, t0s, dts, steps = [], [], [], []
    for k in range(9):
        n = int(rng.integers(5, 40))
        g = W.erdos_renyi_mean_degree(n, 3.0, 100 + k)
        omega = float(rng.uniform(0, 1))
        walks.append((g, omega, [W.random_pure_states(n, 1, 200 + k)[0]]))
        t0s.append(float(rng.choice([0.0, 0.7])))
        dts.append(float(rng.uniform(0.05, 0.5)))
        steps.append(int(rng.integers(1, 30)))
    got, _ = _run_batch(ctx, walks, 1, t0s, dts, steps, "c128")
    for (g, omega, states), p, t0, dt, q in zip(walks, got, t0s, dts, steps):
        w = LQSW(g, omega, ctx=ctx)
        w.initial_state(rho0=states[0])
        _, alone = w.series(t0, dt, q, states=False)
        assert np.max(np.abs(p[:, 0, :] - alone.cpu().numpy())) <= 1e-10
        ref = _oracle_pops(g, omega, states, t0, dt, q)
        assert np.max(np.abs(p - ref)) <= 1e-10


def test_full_regular_batch_invariants_and_samples(ctx):
    # the 256-walk batch (N ~ U{16..512}, four pure states each, complex64):
    # populations of every output sum to 1 and the smallest walks match the oracle
    walks = W.batch_regular()
    steps = [10] * len(walks)
    got, st = _run_batch(ctx, walks, 4, [0.0] * len(walks), [0.2] * len(walks), steps, "c64")
    for p in got:
        assert np.max(np.abs(p.sum(axis=2) - 1.0)) <= 1e-4
        assert np.min(p) >= -1e-4
    order = np.argsort([g.n for g, _, _ in walks])[:3]
    for w_i in order:
        g, omega, states = walks[w_i]
        ref = _oracle_pops(g, omega, states, 0.0, 0.2, 10)
        assert np.max(np.abs(got[w_i] - ref)) <= 1e-4
