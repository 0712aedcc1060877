"""Global-interaction walks on the GPU (qsw_build_gqsw / qsw_build_global)
against the oracle (oracle/gqsw.py), element by element, through the C ABI.

Tolerances as for the L-QSW: one application of L~ to <= 1e-12 of its scale
(different summation order); complex128 series <= 1e-10 max-abs; complex64
bulk populations <= 1e-4."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import expmv, gqsw, superop
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


def _dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.complex128)).to("cuda:0")


def _host(t):
    return t.cpu().numpy()


def _general_case(n, seed, n_l=2, ports=True, rot=True):
    rng = np.random.default_rng(seed)
    Hc = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Hc = (Hc + Hc.conj().T) * (rng.random((n, n)) < 0.6)
    Hc = np.triu(Hc) + np.triu(Hc, 1).conj().T
    Ls = []
    for k in range(n_l):
        L = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * (rng.random((n, n)) < 0.4)
        if n_l == 1:   # no diagonal: the closed-form 1-norm applies
            np.fill_diagonal(L, 0.0)
        Ls.append(L)
    R = None
    if rot:
        R = np.zeros((n, n), complex)
        for i in range(n - 1):
            R[i, i + 1] = 1j
        R = R + R.conj().T
    src = [(0, 0.7)] if ports else []
    snk = [(n - 1, 1.3)] if ports else []
    return Hc, Ls, R, src, snk


def _oracle_general(n, Hc, Ls, R, src, snk):
    G = np.zeros((n, n))
    walk = gqsw.global_walk(G, H=Hc, Ls=Ls, sources=src, sinks=snk)
    if R is not None:
        Rt = np.zeros((walk.n_tilde, walk.n_tilde), complex)
        Rt[:n, :n] = R
        walk.H_rot = sp.csr_matrix(Rt)
    return walk


@pytest.mark.parametrize("n,seed,omega,n_l,ports,rot", [
    (3, 1, 0.0, 1, False, False), (4, 2, 1.0, 2, True, True), (6, 3, 0.35, 2, True, True),
    (7, 4, 0.8, 1, False, True), (9, 5, 0.5, 3, True, False)])
def test_apply_and_adjoint_norm_match_oracle(ctx, n, seed, omega, n_l, ports, rot):
    from paper_2003_02450_gb300 import qsw as C
    Hc, Ls, R, src, snk = _general_case(n, seed, n_l, ports, rot)
    op = C.qsw_build_global(ctx.handle, n, Hc, Ls, R, omega, src, snk)
    walk = _oracle_general(n, Hc, Ls, R, src, snk)
    L = gqsw.superoperator(walk, omega)
    nt = walk.n_tilde
    rng = np.random.default_rng(seed + 100)
    for trial in range(3):
        x = rng.standard_normal(nt * nt) + 1j * rng.standard_normal(nt * nt)
        y = _dev(np.zeros(nt * nt))
        C.qsw_apply(ctx.handle, op, _dev(x), y)
        ref = L @ x
        assert np.max(np.abs(_host(y) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    info = C.qsw_op_info(ctx.handle, op)
    exact = abs(L).sum(axis=0).max()
    if n_l == 1 or omega == 0.0:   # closed form (single operator without diagonal)
        assert info["norms"][0] == pytest.approx(exact, rel=1e-12)
    else:                          # estimated: a lower bound
        assert info["norms"][0] <= exact * (1 + 1e-12)
    C.qsw_op_destroy(op)


def _gqsw_case(kind):
    if kind == "three":
        G = np.zeros((3, 3))
        G[2, 0] = G[2, 1] = 1.0
        return W.from_dense(G)
    if kind == "cycle":
        return W.cycle_graph(8)
    return W.random_digraph(12, 0.25, 17)


@pytest.mark.parametrize("kind,omega,ports,herm", [
    ("three", 1.0, False, True), ("cycle", 0.0, False, True), ("cycle", 0.6, True, True),
    ("er", 0.3, True, True), ("er", 0.9, False, False), ("er", 1.0, True, False)])
def test_gqsw_series_matches_oracle(ctx, kind, omega, ports, herm):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g = _gqsw_case(kind)
    n = g.n
    src = [(0, 0.5)] if ports else []
    snk = [(n - 1, 0.8)] if ports else []
    op = C.qsw_build_gqsw(ctx.handle, g, None, omega, src, snk)
    walk = gqsw.global_walk(g.dense(), sources=src, sinks=snk)
    L = gqsw.superoperator(walk, omega)
    nt = walk.n_tilde
    rho0 = W.random_density_matrix(nt, 3) if herm else \
        np.random.default_rng(4).standard_normal((nt, nt)) + 0j
    x0 = W.vec(rho0)
    steps, dt = 6, 0.4
    ref = expmv.expmv_series(L, x0, 0.2, dt, steps)
    out = torch.empty((steps + 1, nt * nt), dtype=torch.complex128, device="cuda:0")
    pops = torch.empty((steps + 1, nt), dtype=torch.float64, device="cuda:0")
    st = C.qsw_expmv_series(ctx.handle, op, _dev(x0), 0.2, dt, steps, out, pops)
    assert st["hermitian"] == (1 if herm else 0)
    assert np.max(np.abs(_host(out) - ref)) <= 1e-10
    assert np.max(np.abs(_host(pops) - superop.populations(ref, nt))) <= 1e-10
    C.qsw_op_destroy(op)


def test_paper_three_vertex_example_gpu(ctx):
    """Section 4.1.2 G-QSW example: [0.25, 0.25, 0.5] at t = 100, omega = 1."""
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g = _gqsw_case("three")
    op = C.qsw_build_gqsw(ctx.handle, g, None, 1.0)
    pops = torch.empty((1, 3), dtype=torch.float64, device="cuda:0")
    C.qsw_expmv_series(ctx.handle, op, _dev(W.vec(W.basis_state(3, 0))), 100.0, 0.0, 0, None, pops)
    assert np.allclose(_host(pops)[0], [0.25, 0.25, 0.5], atol=1e-10)
    C.qsw_op_destroy(op)


def test_gqsw_complex64_bulk(ctx):
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g = _gqsw_case("er")
    op = C.qsw_build_gqsw(ctx.handle, g, None, 0.5, precision="c64")
    walk = gqsw.global_walk(g.dense())
    L = gqsw.superoperator(walk, 0.5)
    x0 = W.vec(W.random_density_matrix(12, 8))
    ref = superop.populations(expmv.expmv_series(L, x0, 0.0, 0.5, 8), 12)
    pops = torch.empty((9, 12), dtype=torch.float64, device="cuda:0")
    C.qsw_expmv_series(ctx.handle, op, _dev(x0), 0.0, 0.5, 8, None, pops)
    assert np.max(np.abs(_host(pops) - ref)) <= 1e-4
    C.qsw_op_destroy(op)


def test_gqsw_set_omega_and_limits(ctx):
    """set_omega rebuilds Q and L'; the CSR export, the batched and the
    no-allocation entry points refuse global walks."""
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g = _gqsw_case("cycle")
    op = C.qsw_build_gqsw(ctx.handle, g, None, 0.2)
    C.qsw_set_omega(ctx.handle, op, 0.7)
    walk = gqsw.global_walk(g.dense())
    L = gqsw.superoperator(walk, 0.7)
    x = W.vec(W.random_density_matrix(8, 2))
    y = _dev(np.zeros(64))
    C.qsw_apply(ctx.handle, op, _dev(x), y)
    assert np.max(np.abs(_host(y) - L @ x)) <= 1e-12 * max(1.0, np.max(np.abs(L @ x)))
    assert C.qsw_op_info(ctx.handle, op)["nnz"] == 0
    with pytest.raises(C.QswError):
        C.qsw_op_export_csr(ctx.handle, op, None, None, None)
    pops = torch.empty((3, 8), dtype=torch.float64, device="cuda:0")
    with pytest.raises(C.QswError):
        C.qsw_batch_series(ctx.handle, [op], [_dev(x)], 1, [0.0], [0.5], [2], [pops])
    with pytest.raises(C.QswError):
        C.qsw_expmv_series_noalloc(ctx.handle, op, _dev(x), 0.0, 0.5, 2, None, pops)
    C.qsw_op_destroy(op)


def test_bench_config_first_outputs_full_size(ctx):
    """The G-QSW bench walk (ER N = 400, p = 0.025, omega = 0.3, uniform
    superposition): the first two outputs of dt = 0.1 against the oracle."""
    import torch
    from paper_2003_02450_gb300 import qsw as C
    g = W.erdos_renyi_digraph(400, 0.025, W.SEED_ER1000 + 1)
    op = C.qsw_build_gqsw(ctx.handle, g, None, 0.3)
    walk = gqsw.global_walk(g.dense())
    L = gqsw.superoperator(walk, 0.3)
    x0 = W.vec(W.uniform_superposition(400))
    ref = expmv.expmv_series(L, x0, 0.0, 0.1, 2)
    out = torch.empty((3, 400 * 400), dtype=torch.complex128, device="cuda:0")
    C.qsw_expmv_series(ctx.handle, op, _dev(x0), 0.0, 0.1, 2, out, None)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-10
    C.qsw_op_destroy(op)


@pytest.mark.parametrize("kind", ["gqsw", "nm"])
def test_hermitian_form_long_horizon(ctx, kind):
    """The Hermitian form takes the Q terms from R = x Q^dag, which assumes an
    exactly Hermitian term; a rounding-level imaginary diagonal would grow like
    exp(t ||L'^dag L'|| / 2) (seen as 1e-10 at t = 4.8 on this walk before the
    diagonal was kept real).  Twenty steps of 0.4 against the oracle."""
    import torch
    from oracle import nm
    from paper_2003_02450_gb300 import qsw as C
    g = W.random_digraph(16, 0.2, 16) if kind == "gqsw" else W.random_digraph(9, 0.3, 9)
    if kind == "gqsw":
        op = C.qsw_build_gqsw(ctx.handle, g, None, 0.6)
        walk = gqsw.global_walk(g.dense())
    else:
        op = C.qsw_build_nm_gqsw(ctx.handle, g, 0.6)
        walk, _ = nm.nm_walk(g.dense())
    nt = walk.n_tilde
    L = gqsw.superoperator(walk, 0.6)
    x0 = W.vec(W.random_density_matrix(nt, 2))
    ref = expmv.expmv_series(L, x0, 0.0, 0.4, 20)
    out = torch.empty((21, nt * nt), dtype=torch.complex128, device="cuda:0")
    st = C.qsw_expmv_series(ctx.handle, op, _dev(x0), 0.0, 0.4, 20, out, None)
    assert st["hermitian"] == 1
    got = _host(out)
    assert np.max(np.abs(got - ref)) <= 1e-10
    # every output exactly Hermitian
    for k in (5, 20):
        R = got[k].reshape(nt, nt, order="F")
        assert np.array_equal(R, R.conj().T)
    C.qsw_op_destroy(op)
