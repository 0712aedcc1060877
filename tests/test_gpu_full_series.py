"""The benchmark's own series calls, compared with the oracle over the WHOLE time grid.

The expected values were written by ``tests/golden/make_full_series.py``, which
runs only the FP64 oracle (Algorithm 5.2 over the full grid, Section 3.1): for
every output time, all N~ populations, one full row of the density matrix and
2048 seeded upper-triangle elements.  Here the library runs the same calls as
``bench.py`` (ER-1000: 50 steps of 0.1 from t0 = 0; 45 x 45 lattice: 20 steps
of 0.5) through the C ABI, and every stored element of every output is compared.

Tolerances (the stated accuracy of the method): complex128 max-abs density
matrix error <= 1e-10; complex64 bulk population error <= 1e-4.
"""
import os

import numpy as np
import pytest

from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_C128 = 1e-10
TOL_C64_POP = 1e-4


def _golden(name):
    g = np.load(os.path.join(HERE, "golden", f"{name}_series.npz"))
    return {k: g[k] for k in g.files}


@pytest.fixture(scope="module")
def lib():
    ensure_built()
    import torch
    from paper_2003_02450_gb300 import qsw as C
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(0, stream.cuda_stream)
    yield C, ctx, dev
    C.qsw_destroy(ctx)


def _run(lib, cfg, precision, operator):
    import torch
    C, ctx, dev = lib
    N, n, q = cfg.graph.n, cfg.graph.n ** 2, cfg.steps
    rho0 = torch.from_numpy(W.vec(cfg.rho0)).to(dev)
    out = torch.empty((q + 1, n), dtype=torch.complex128, device=dev)
    pops = torch.empty((q + 1, N), dtype=torch.float64, device=dev)
    op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision=precision,
                                   operator=operator)
    try:
        st = C.qsw_expmv_series(ctx, op, rho0, cfg.t0, cfg.dt, q, out, pops)
    finally:
        C.qsw_op_destroy(op)
    torch.cuda.synchronize(dev)
    return out, pops, st


def _errors(out, pops, g):
    """Max-abs errors against the stored oracle values: (populations, row r,
    column r = conj of row r (the mirrored lower triangle), sampled elements)."""
    import torch
    nt = int(g["n_tilde"])
    r = int(g["row_index"])
    dev = out.device
    row_idx = torch.as_tensor(r + nt * np.arange(nt), device=dev)
    col_idx = torch.as_tensor(np.arange(nt) + nt * r, device=dev)
    smp_idx = torch.as_tensor(g["sample_idx"], device=dev)
    e_pop = np.max(np.abs(pops.cpu().numpy() - g["pops"]))
    e_row = np.max(np.abs(out[:, row_idx].cpu().numpy() - g["row"]))
    e_col = np.max(np.abs(out[:, col_idx].cpu().numpy() - np.conj(g["row"])))
    e_smp = np.max(np.abs(out[:, smp_idx].cpu().numpy() - g["sample"]))
    return e_pop, e_row, e_col, e_smp


@pytest.mark.parametrize("operator", ["matfree", "csr"])
def test_er1000_whole_series_matches_oracle(lib, operator):
    cfg = W.er1000()
    g = _golden("er1000")
    assert (float(g["dt"]), int(g["steps"]), float(g["omega"])) == (cfg.dt, cfg.steps, cfg.omega)
    out, pops, st = _run(lib, cfg, "c128", operator)
    errs = _errors(out, pops, g)
    print(f"er1000 {operator}: max|err| pops {errs[0]:.2e} row {errs[1]:.2e} "
          f"col {errs[2]:.2e} sample {errs[3]:.2e}; (m*, s) = ({st['m_star']}, {st['s']}), "
          f"{st['matvecs']} products (oracle ({int(g['oracle_m_star'])}, {int(g['oracle_s'])}), "
          f"{int(g['oracle_matvecs'])})")
    assert max(errs) <= TOL_C128, errs
    assert out.shape[0] == 51


def test_er1000_whole_series_host_buffers(lib):
    # the end-to-end call of the benchmark: host buffers in and out, copies overlapped
    import torch
    C, ctx, dev = lib
    cfg = W.er1000()
    g = _golden("er1000")
    N, n, q = cfg.graph.n, cfg.graph.n ** 2, cfg.steps
    h_rho0 = torch.from_numpy(W.vec(cfg.rho0)).pin_memory()
    h_out = torch.empty((q + 1, n), dtype=torch.complex128).pin_memory()
    h_pops = torch.empty((q + 1, N), dtype=torch.float64).pin_memory()
    op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision="c128")
    try:
        C.qsw_expmv_series_host(ctx, op, h_rho0, cfg.t0, cfg.dt, q, h_out, h_pops)
    finally:
        C.qsw_op_destroy(op)
    errs = _errors(h_out, h_pops, g)
    assert max(errs) <= TOL_C128, errs


@pytest.fixture(scope="module")
def grid45_golden():
    return _golden("grid45")


@pytest.mark.parametrize("operator", ["matfree", "csr"])
def test_grid45_whole_series_c128(lib, grid45_golden, operator):
    cfg = W.grid45("c128")
    g = grid45_golden
    assert (float(g["dt"]), int(g["steps"]), float(g["omega"])) == (cfg.dt, cfg.steps, cfg.omega)
    out, pops, st = _run(lib, cfg, "c128", operator)
    errs = _errors(out, pops, g)
    print(f"grid45 c128 {operator}: max|err| pops {errs[0]:.2e} row {errs[1]:.2e} "
          f"col {errs[2]:.2e} sample {errs[3]:.2e}")
    assert max(errs) <= TOL_C128, errs


@pytest.mark.parametrize("operator", ["matfree", "csr"])
def test_grid45_whole_series_c64_bulk(lib, grid45_golden, operator):
    cfg = W.grid45("c64")
    g = grid45_golden
    out, pops, st = _run(lib, cfg, "c64", operator)
    e_pop = np.max(np.abs(pops.cpu().numpy() - g["pops"]))
    errs = _errors(out, pops, g)
    print(f"grid45 c64 {operator}: population error {e_pop:.2e}, density-matrix "
          f"max|err| row {errs[1]:.2e} sample {errs[3]:.2e}")
    assert e_pop <= TOL_C64_POP, e_pop
    # every output, not only the last, is within the bound
    per_output = np.max(np.abs(pops.cpu().numpy() - g["pops"]), axis=1)
    assert per_output.shape == (21,) and np.all(per_output <= TOL_C64_POP)
