"""Pins for oracle/normest.py."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import normest, graph, superop
from paper_2003_02450_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    # Published reference stream of SplitMix64 started from state 0.
    assert [normest.splitmix64(0, i) for i in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    signs = normest.random_signs(64, 0)
    ref = [-1.0 if normest.splitmix64(0, i) >> 63 else 1.0 for i in range(64)]
    assert signs.tolist() == ref


def _rand_sparse(n, density, seed, complex_=True, nonneg=False):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=rng, format="csr")
    if nonneg:
        return A.astype(np.complex128)
    A.data = rng.standard_normal(A.nnz) + (1j * rng.standard_normal(A.nnz) if complex_ else 0)
    return A


@pytest.mark.parametrize("p", [1, 2, 3, 5, 9])
def test_exact_power_norm_against_numpy(p):
    A = _rand_sparse(30, 0.15, 7 + p)
    ref = np.linalg.norm(np.linalg.matrix_power(A.toarray(), p), 1)
    assert abs(normest.onenorm_power_exact(A, p) - ref) <= 1e-12 * ref


@pytest.mark.parametrize("seed", range(6))
def test_estimate_is_lower_bound_and_close(seed):
    A = _rand_sparse(40, 0.1, seed)
    for p in (2, 4, 9):
        ex = normest.onenorm_power_exact(A, p)
        est = normest.onenorm_power_est(A, p)
        assert est <= ex * (1 + 1e-12)
        assert est >= ex / 10


@pytest.mark.parametrize("seed", range(4))
def test_estimate_exact_for_nonnegative(seed):
    # For entrywise non-negative A, sign(A^p X) is the all-ones block, the
    # adjoint products give the column sums, and the next iterate is the unit
    # vector of the largest column: the estimate equals the exact norm.
    A = _rand_sparse(50, 0.08, 100 + seed, nonneg=True)
    for p in (2, 3, 7):
        ex = normest.onenorm_power_exact(A, p)
        assert abs(normest.onenorm_power_est(A, p) - ex) <= 1e-12 * ex


def test_onenorm_of_cycle_superoperator():
    # 16-cycle Laplacian (degree 2), omega = 0.5: every column of L~ holds
    # |diag| + commutator entries; the largest column sum is 4 (diagonal
    # columns: 0.5*2*... computed by hand below).
    cfg = W.cycle16()
    L = superop.superoperator(graph.lqsw_walk(graph.adjacency(cfg.graph)), 0.5)
    dense = np.abs(L.toarray()).sum(axis=0).max()
    assert normest.onenorm(L) == pytest.approx(dense, rel=1e-15)
    assert normest.onenorm(L) == pytest.approx(4.0, rel=1e-15)
