"""The grid barrier of the series kernel waits a bounded time: with one block
absent (a participant that never arrives) every other block gives up, the
timeout is reported, and the context stays usable for the next series."""
import numpy as np
import pytest

from oracle import expmv, graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu


def test_barrier_wait_gives_up_and_context_survives():
    ensure_built()
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300.walk import Context
    ctx = Context(0)
    sec = C.qsw_probe_wait_limit(ctx.handle)
    assert 0.0 < sec < 30.0
    g = W.cycle_graph(6)
    op = C.qsw_build_superoperator(ctx.handle, g, None, 0.5)
    rho0 = torch.from_numpy(W.vec(W.basis_state(6, 0))).to("cuda:0")
    pops = torch.empty((4, 6), dtype=torch.float64, device="cuda:0")
    C.qsw_expmv_series(ctx.handle, op, rho0, 0.0, 0.5, 3, None, pops)
    walk = graph.lqsw_walk(graph.adjacency(g))
    ref = superop.populations(expmv.expmv_series(superop.superoperator(walk, 0.5),
                                                 W.vec(W.basis_state(6, 0)), 0.0, 0.5, 3), 6)
    assert np.max(np.abs(pops.cpu().numpy() - ref)) <= 1e-10
    C.qsw_op_destroy(op)
    ctx.close()
