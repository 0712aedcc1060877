"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances:
* assembly: identical structure after dropping exact zeros; values within
  4 ulp of the largest |entry| (the condensed rule and the Kronecker sums round
  differently);
* complex128 series: max |rho_gpu - rho_oracle| <= 1e-10 (the target stated for
  the method; both sides meet the 2^-53 backward-error tolerance, so the
  observed gap is ~1e-14);
* complex64-bulk series: population error <= 1e-4.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import expmv, graph, normest, superop
from paper_2003_02450_gb300 import workloads as W
from tests import pins
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu

TOL_C128 = 1e-10
TOL_C64_POP = 1e-4


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    import torch
    from paper_2003_02450_gb300.walk import Context
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return Context(0)


def _oracle(g, omega, H=None, sources=(), sinks=()):
    walk = graph.lqsw_walk(graph.adjacency(g), H=H, sources=sources, sinks=sinks)
    return walk, superop.superoperator(walk, omega)


def _gpu(ctx, g, omega, H=None, sources=(), sinks=(), precision="c128", operator="matfree"):
    from paper_2003_02450_gb300.walk import LQSW
    return LQSW(g, omega, H=H, sources=sources, sinks=sinks, precision=precision, ctx=ctx,
                operator=operator)


OPERATORS = ["matfree", "csr"]


def _csr_from_gpu(w):
    rowptr, col, val = w.export_csr()
    m = sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy().astype(np.int64),
                       rowptr.cpu().numpy().astype(np.int64)), shape=(w.n, w.n))
    return m


def _compare_csr(Lg, Lo):
    Lg = Lg.copy()
    Lg.eliminate_zeros()
    Lg.sort_indices()
    Lo = Lo.copy()
    Lo.eliminate_zeros()
    Lo.sort_indices()
    assert np.array_equal(Lg.indptr, Lo.indptr)
    assert np.array_equal(Lg.indices, Lo.indices)
    scale = np.max(np.abs(Lo.data)) if Lo.nnz else 1.0
    assert np.max(np.abs(Lg.data - Lo.data), initial=0.0) <= 4 * np.finfo(float).eps * scale


SMALL = [
    # (N, p, seed, omega, sources, sinks, explicit_h)
    (1, 0.0, 1, 0.5, [], [], False),
    (2, 1.0, 1, 0.5, [], [], False),
    (3, 0.5, 2, 0.0, [], [], False),
    (5, 0.4, 3, 1.0, [], [], False),
    (6, 0.5, 4, 0.37, [], [], True),
    (7, 0.4, 5, 0.8, [(0, 2.0)], [(1, 3.0)], False),
    (9, 0.3, 6, 0.25, [(2, 0.5), (2, 1.5)], [(5, 0.5), (0, 1.5)], True),
    (40, 0.1, 7, 0.6, [(0, 0.5)], [(39, 0.5)], False),
]


def _small_case(N, p, seed, explicit_h):
    g = W.random_digraph(N, p, seed)
    H = None
    if explicit_h:
        rng = np.random.default_rng(seed + 1000)
        a = rng.standard_normal((N, N)) * (rng.random((N, N)) < 0.5)
        H = sp.csr_matrix((a + a.T) / 2)
    return g, H


@pytest.mark.parametrize("operator", OPERATORS)
@pytest.mark.parametrize("N,p,seed,omega,sources,sinks,explicit_h", SMALL)
def test_assembly_matches_oracle(ctx, N, p, seed, omega, sources, sinks, explicit_h, operator):
    g, H = _small_case(N, p, seed, explicit_h)
    _, Lo = _oracle(g, omega, H, sources, sinks)
    w = _gpu(ctx, g, omega, H, sources, sinks, operator=operator)
    assert w.nnz == _csr_from_gpu(w).nnz
    _compare_csr(_csr_from_gpu(w), Lo)


@pytest.mark.parametrize("operator", OPERATORS)
@pytest.mark.parametrize("N,p,seed,omega,sources,sinks,explicit_h", SMALL)
def test_norms_and_params_match_oracle(ctx, N, p, seed, omega, sources, sinks, explicit_h, operator):
    g, H = _small_case(N, p, seed, explicit_h)
    _, Lo = _oracle(g, omega, H, sources, sinks)
    w = _gpu(ctx, g, omega, H, sources, sinks, operator=operator)
    info = expmv.NormInfo(Lo, precompute=True)
    assert w.norms[0] == pytest.approx(info.one, rel=1e-14, abs=0)
    # The block estimator returns a lower bound that is usually the exact norm.
    # Where the row ranking has exact ties (symmetric graphs), rounding picks
    # the branch, so the GPU and the oracle may stop at different valid bounds.
    same = True
    for p_ in range(2, 10):
        exact = normest.onenorm_power_exact(Lo, p_) if Lo.shape[0] <= 400 else None
        est = w.norms[p_ - 1]
        if exact is not None:
            assert est <= exact * (1 + 1e-12)
            assert est >= exact / 10
        same &= abs(est ** (1.0 / p_) - info.d(p_)) <= 1e-10 * max(info.d(p_), 1e-300)
    if same:
        ginfo = expmv.NormInfo(Lo, norms=w.norms)
        for t in (0.1, 1.0, 10.0, 100.0):
            assert expmv.select_params(ginfo, t) == expmv.select_params(info, t)


@pytest.mark.parametrize("operator", OPERATORS)
@pytest.mark.parametrize("N,p,seed,omega,sources,sinks,explicit_h", SMALL)
def test_apply_matches_oracle(ctx, N, p, seed, omega, sources, sinks, explicit_h, operator):
    import torch
    g, H = _small_case(N, p, seed, explicit_h)
    walk, Lo = _oracle(g, omega, H, sources, sinks)
    w = _gpu(ctx, g, omega, H, sources, sinks, operator=operator)
    x = W.vec(W.random_density_matrix(walk.n_tilde, seed))
    y = w.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = Lo @ x
    assert np.max(np.abs(y - ref)) <= 1e-14 * max(1.0, np.max(np.abs(Lo.data), initial=0))


@pytest.mark.parametrize("operator", OPERATORS)
@pytest.mark.parametrize("N,p,seed,omega,sources,sinks,explicit_h", SMALL)
@pytest.mark.parametrize("t0,dt,steps", [(0.0, 0.1, 100), (0.5, 2.0, 3), (1.0, 0.25, 37),
                                         (2.5, 0.0, 0), (0.0, 0.7, 1)])
def test_series_matches_oracle(ctx, N, p, seed, omega, sources, sinks, explicit_h, t0, dt, steps,
                               operator):
    import torch
    g, H = _small_case(N, p, seed, explicit_h)
    walk, Lo = _oracle(g, omega, H, sources, sinks)
    rho0 = W.vec(W.random_density_matrix(walk.n_tilde, seed + 7))
    ref = expmv.expmv_series(Lo, rho0, t0, dt, steps)
    w = _gpu(ctx, g, omega, H, sources, sinks, operator=operator)
    states, pops = w.series(t0, dt, steps, rho0=torch.from_numpy(rho0).cuda())
    got = states.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL_C128
    assert np.max(np.abs(pops.cpu().numpy() - superop.populations(ref, walk.n_tilde))) <= TOL_C128


@pytest.mark.parametrize("operator", OPERATORS)
@pytest.mark.parametrize("N,p,seed,omega,sources,sinks,explicit_h", SMALL[3:])
def test_series_non_hermitian_input(ctx, N, p, seed, omega, sources, sinks, explicit_h, operator):
    # a general complex vector (not a density matrix): the Hermitian shortcut
    # must not be taken and the result must still match
    import torch
    g, H = _small_case(N, p, seed, explicit_h)
    walk, Lo = _oracle(g, omega, H, sources, sinks)
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal(walk.n_tilde ** 2) + 1j * rng.standard_normal(walk.n_tilde ** 2)
    ref = expmv.expmv_series(Lo, x0, 0.2, 0.3, 12)
    w = _gpu(ctx, g, omega, H, sources, sinks, operator=operator)
    states, _ = w.series(0.2, 0.3, 12, rho0=torch.from_numpy(x0).cuda())
    assert w.last_stats["hermitian"] == 0
    assert np.max(np.abs(states.cpu().numpy() - ref)) <= TOL_C128 * max(1.0, np.max(np.abs(ref)))


def test_hermitian_shortcut_taken_for_density_matrices(ctx):
    import torch
    cfg = W.cycle16()
    w = _gpu(ctx, cfg.graph, cfg.omega)
    w.initial_state(rho0=cfg.rho0)
    states, _ = w.series(0.0, 0.5, 4)
    assert w.last_stats["hermitian"] == 1
    S = states.reshape(5, 16, 16)
    assert torch.equal(S, S.conj().transpose(1, 2))   # lower triangles mirrored exactly


def test_cycle16_config_series(ctx):
    import torch
    cfg = W.cycle16()
    walk, Lo = _oracle(cfg.graph, cfg.omega)
    rho0 = W.vec(cfg.rho0)
    st = {}
    ref = expmv.expmv_series(Lo, rho0, cfg.t0, cfg.dt, cfg.steps, stats=st)
    w = _gpu(ctx, cfg.graph, cfg.omega)
    w.initial_state(rho0=cfg.rho0)
    states, pops = w.series(cfg.t0, cfg.dt, cfg.steps)
    err = np.max(np.abs(states.cpu().numpy() - ref))
    assert err <= TOL_C128, err
    assert (w.last_stats["m_star"], w.last_stats["s"]) == (st["series_m"], st["series_s"])
    assert w.last_stats["matvecs"] == st["matvecs"]


def test_pops_only_uses_ring_and_matches(ctx):
    import torch
    cfg = W.cycle16()
    walk, Lo = _oracle(cfg.graph, cfg.omega)
    rho0 = W.vec(cfg.rho0)
    ref = superop.populations(expmv.expmv_series(Lo, rho0, 0.3, 0.1, 64), 16)
    w = _gpu(ctx, cfg.graph, cfg.omega)
    _, pops = w.series(0.3, 0.1, 64, rho0=torch.from_numpy(rho0).cuda(), states=False)
    assert np.max(np.abs(pops.cpu().numpy() - ref)) <= TOL_C128


def test_populations_entry_point(ctx):
    import torch
    cfg = W.cycle16()
    w = _gpu(ctx, cfg.graph, cfg.omega)
    w.initial_state(populations=np.eye(16)[3])
    states, pops = w.series(0.0, 0.5, 8)
    again = w.populations(states)
    assert torch.equal(again, pops)
    assert np.allclose(states[0].cpu().numpy(), W.vec(W.basis_state(16, 3)), atol=0)


def test_set_omega_rebuilds(ctx):
    import torch
    g, _ = _small_case(8, 0.4, 11, False)
    w = _gpu(ctx, g, 0.2)
    w.set_omega(0.9)
    walk, Lo = _oracle(g, 0.9)
    _compare_csr(_csr_from_gpu(w), Lo)
    rho0 = W.vec(W.random_density_matrix(8, 2))
    ref = expmv.expmv_series(Lo, rho0, 0.0, 0.3, 10)
    states, _ = w.series(0.0, 0.3, 10, rho0=torch.from_numpy(rho0).cuda())
    assert np.max(np.abs(states.cpu().numpy() - ref)) <= TOL_C128


def test_paper_example_on_gpu(ctx):
    # the Section 4 example, H = GU passed explicitly
    G = sp.csr_matrix(([1.0, 1.0], ([2, 2], [0, 1])), shape=(3, 3))
    GU = sp.csr_matrix(([1.0, 1, 1, 1], ([0, 1, 2, 2], [2, 2, 0, 1])), shape=(3, 3))
    printed = np.loadtxt(__file__.replace("test_gpu_parity.py", "golden/paper_example_lqsw.txt"))
    g = W.from_dense(G.toarray())
    for omega, t, *p in printed:
        w = _gpu(ctx, g, omega, H=GU)
        w.initial_state(populations=[1.0, 0.0, 0.0])
        _, pops = w.series(t, 0.0, 0)
        p = np.array(p)
        assert np.all(np.abs(pops.cpu().numpy()[0] - p) <= 5e-9 * np.abs(p) + 1e-10)


# ------------------------------------------------------------ full sizes --

@pytest.fixture(scope="module")
def er1000(ctx):
    cfg = W.er1000()
    walk, Lo = _oracle(cfg.graph, cfg.omega)
    return cfg, walk, Lo


def test_er1000_assembly_full_size(ctx, er1000):
    cfg, walk, Lo = er1000
    w = _gpu(ctx, cfg.graph, cfg.omega)
    assert w.nnz == Lo.nnz
    _compare_csr(_csr_from_gpu(w), Lo)
    assert w.norms[0] == pytest.approx(expmv.NormInfo(Lo).one, rel=1e-14)


@pytest.mark.parametrize("operator", OPERATORS)
def test_er1000_series_first_steps_full_size(ctx, er1000, operator):
    # the bench's launch (same call, same operator size); the oracle finishes the
    # first two output times of the 50-step grid in seconds
    cfg, walk, Lo = er1000
    rho0 = W.vec(cfg.rho0)
    ref = expmv.expmv_series(Lo, rho0, cfg.t0, cfg.dt, 2)
    w = _gpu(ctx, cfg.graph, cfg.omega, operator=operator)
    w.initial_state(rho0=cfg.rho0)
    states, _ = w.series(cfg.t0, cfg.dt, 2)
    assert np.max(np.abs(states.cpu().numpy() - ref)) <= TOL_C128


def test_er1000_full_series_invariants(ctx, er1000):
    import torch
    cfg, walk, Lo = er1000
    w = _gpu(ctx, cfg.graph, cfg.omega)
    w.initial_state(rho0=cfg.rho0)
    states, pops = w.series(cfg.t0, cfg.dt, cfg.steps)
    N = 1000
    S = states.reshape(cfg.steps + 1, N, N).transpose(1, 2)   # rho[k][i][j]
    tr = torch.diagonal(S, dim1=1, dim2=2).sum(-1)
    assert torch.max(torch.abs(tr - 1)).item() <= 1e-12
    herm = torch.max(torch.abs(S - S.conj().transpose(1, 2))).item()
    assert herm <= 1e-13
    assert torch.allclose(pops.sum(-1), torch.ones_like(pops[:, 0]), atol=1e-12, rtol=0)
    ev = torch.linalg.eigvalsh(S[-1]).min().item()
    assert ev >= -1e-12
    # the plan matches the oracle's parameter choice for the same norms
    info = expmv.NormInfo(Lo, norms=w.norms)
    assert (w.last_stats["m_star"], w.last_stats["s"]) == expmv.select_params(info, cfg.steps * cfg.dt)


def test_er1000_omega0_closed_form(ctx, er1000):
    cfg, walk, Lo = er1000
    w = _gpu(ctx, cfg.graph, 0.0)
    w.initial_state(rho0=cfg.rho0)
    states, _ = w.series(0.0, 0.1, 5)
    H = walk.H.toarray()
    for k in (1, 5):
        ref = pins.ctqw_density(H, cfg.rho0, 0.1 * k)
        got = W.unvec(states[k].cpu().numpy(), 1000)
        assert np.max(np.abs(got - ref)) <= TOL_C128
        assert abs(np.trace(got @ got).real - 1.0) <= 1e-10


def test_er1000_omega1_closed_form(ctx, er1000):
    cfg, walk, Lo = er1000
    G = cfg.graph.dense()
    rho0 = W.random_density_matrix(1000, 3, rank=2)
    w = _gpu(ctx, cfg.graph, 1.0)
    w.initial_state(rho0=rho0)
    states, pops = w.series(0.0, 0.1, 4)
    p_ref = pins.ctrw_populations(G, np.real(np.diag(rho0)), 0.4)
    assert np.max(np.abs(pops[4].cpu().numpy() - p_ref)) <= TOL_C128
    d = G.sum(axis=0)
    got = W.unvec(states[4].cpu().numpy(), 1000)
    decay = np.exp(-0.5 * (d[:, None] + d[None, :]) * 0.4) * rho0
    off = ~np.eye(1000, dtype=bool)
    assert np.max(np.abs(got[off] - decay[off])) <= TOL_C128


@pytest.fixture(scope="module")
def grid45(ctx):
    cfg = W.grid45("c128")
    walk, Lo = _oracle(cfg.graph, cfg.omega)
    rho0 = W.vec(cfg.rho0)
    ref = expmv.expmv_series(Lo, rho0, cfg.t0, cfg.dt, 2)
    return cfg, walk, Lo, ref


def test_grid45_assembly_and_first_steps_c128(ctx, grid45):
    cfg, walk, Lo, ref = grid45
    w = _gpu(ctx, cfg.graph, cfg.omega)
    _compare_csr(_csr_from_gpu(w), Lo)
    w.initial_state(rho0=cfg.rho0)
    states, _ = w.series(cfg.t0, cfg.dt, 2)
    assert np.max(np.abs(states.cpu().numpy() - ref)) <= TOL_C128


@pytest.mark.parametrize("operator", OPERATORS)
def test_grid45_c64_bulk_populations(ctx, grid45, operator):
    cfg, walk, Lo, ref = grid45
    w = _gpu(ctx, cfg.graph, cfg.omega, precision="c64", operator=operator)
    w.initial_state(rho0=cfg.rho0)
    _, pops = w.series(cfg.t0, cfg.dt, 2)
    err = np.max(np.abs(pops.cpu().numpy() - superop.populations(ref, 2025)))
    assert err <= TOL_C64_POP, err


@pytest.mark.parametrize("operator", OPERATORS)
def test_cycle16_c64_bulk(ctx, operator):
    cfg = W.cycle16()
    walk, Lo = _oracle(cfg.graph, cfg.omega)
    ref = expmv.expmv_series(Lo, W.vec(cfg.rho0), cfg.t0, cfg.dt, cfg.steps)
    w = _gpu(ctx, cfg.graph, cfg.omega, precision="c64", operator=operator)
    w.initial_state(rho0=cfg.rho0)
    _, pops = w.series(cfg.t0, cfg.dt, cfg.steps)
    assert np.max(np.abs(pops.cpu().numpy() - superop.populations(ref, 16))) <= TOL_C64_POP


# ------------------------------------------------------------ edge cases --

def test_rejects_bad_arguments(ctx):
    from paper_2003_02450_gb300 import qsw
    g = W.cycle_graph(4)
    with pytest.raises(qsw.QswError) as e:
        _gpu(ctx, g, 1.5)
    assert e.value.name == "QSW_ERR_OMEGA_RANGE"
    loop = W.Digraph(2, np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.array([1.0]))
    with pytest.raises(qsw.QswError) as e:
        _gpu(ctx, loop, 0.5)
    assert e.value.name == "QSW_ERR_NOT_SIMPLE"
    H = sp.csr_matrix(np.array([[0, 1.0, 0, 0], [2.0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]]))
    with pytest.raises(qsw.QswError) as e:
        _gpu(ctx, g, 0.5, H=H)
    assert e.value.name == "QSW_ERR_NOT_HERMITIAN"
    w = _gpu(ctx, g, 0.5)
    w.initial_state(populations=[1, 0, 0, 0])
    with pytest.raises(qsw.QswError):
        w.series(-1.0, 0.1, 3)
    with pytest.raises(qsw.QswError):
        w.series(0.0, 0.1, -1)
    with pytest.raises(qsw.QswError):
        w.initial_state(populations=[0.5, 0, 0, 0])


def test_empty_graph_is_static(ctx):
    import torch
    g = W.from_arcs(5, [], [], [])
    for omega in (0.0, 0.4, 1.0):
        w = _gpu(ctx, g, omega)
        rho0 = W.random_density_matrix(5, 1)
        w.initial_state(rho0=rho0)
        states, _ = w.series(0.0, 1.0, 4)
        # L~ = 0; the Hermitian form returns the Hermitian part of rho0 (numpy's
        # rho0 is Hermitian only to ~1e-17)
        assert np.max(np.abs(states.cpu().numpy() - W.vec(rho0)[None, :])) <= 1e-15


def test_rejects_operator_beyond_32bit_indices(ctx):
    # N~^2 must fit the 32-bit element indices: 46341^2 = 2,147,488,281 >= 2^31 - 1.
    # The check runs on the host before any device work; the context stays usable.
    from paper_2003_02450_gb300 import qsw as C
    n = 46341
    g = W.Digraph(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with pytest.raises(C.QswError) as e:
        C.qsw_build_superoperator(ctx.handle, g, None, 0.5)
    assert e.value.name == "QSW_ERR_TOO_LARGE"
    # one source port pushes a graph just below the limit over it (N~ = N + ports)
    g2 = W.Digraph(n - 1, np.zeros(n, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with pytest.raises(C.QswError) as e:
        C.qsw_build_superoperator(ctx.handle, g2, None, 0.5, sources=[(0, 0.5)])
    assert e.value.name == "QSW_ERR_TOO_LARGE"
    w = _gpu(ctx, W.cycle_graph(6), 0.5)
    w.initial_state(populations=[1, 0, 0, 0, 0, 0])
    _, pops = w.series(0.0, 0.5, 3)
    assert abs(float(pops[-1].sum().item()) - 1.0) <= 1e-12
