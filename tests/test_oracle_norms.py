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


# ---------------------------------------------------------------------------
# Hand-derived traces of Higham--Tisseur Algorithm 2.4 (complex form, t = 2).
# n = 3: the starting block is [1, x] / 3 with x = (1, 1, -1) (the first three
# SplitMix64 signs at the estimator's seed, pinned above by the reference
# stream).  Every number below is derived by hand in the comments; the tests
# assert the iteration trace, not only the final estimate, so that a transposed
# adjoint (A^T instead of A^H), a real-valued sign, a missing history check or
# an off-by-one in the iteration cap each fails one of them.

def _trace(A, p, **kw):
    tr = []
    est = normest.onenorm_power_est(sp.csr_matrix(np.array(A, dtype=complex)), p, trace=tr, **kw)
    return est, tr


A_ADJ = [[0, 0, 1], [0, 0, 1j], [1j, 0, 0]]


def test_signs_of_three_element_start():
    assert normest.random_signs(3).tolist() == [1.0, 1.0, -1.0]


def test_adjoint_is_conjugate_transpose_p1():
    # A = [[0,0,1],[0,0,i],[i,0,0]], A^H = [[0,0,-i],[0,0,0],[1,-i,0]],
    # ||A||_1 = 2 (column 2: |1| + |i|).
    # k = 1: Y = A X0 = [[1,-1],[i,-i],[i,i]] / 3, column norms (1, 1): est = 1.
    #   S = sign(Y) = [[1,-1],[i,-i],[i,i]];  Z = A^H S:
    #   row 0 = -i S_2 = (1, 1); row 1 = 0; row 2 = S_0 - i S_1 = (1+1, -1-1) = (2, -2)
    #   h = (1, 0, 2) -> order (2, 0, 1), next = [2, 0].
    #   (With A^T = [[0,0,i],[0,0,0],[1,i,0]]: row 2 = S_0 + i S_1 = (0, 0), h = (1, 0, 0),
    #   next = [0, 1], Y = [A e0, A e1] has norms (1, 0) and the estimate stays 1.)
    # k = 2: Y = [A e2, A e0] = [(1, i, 0), (0, 0, i)], norms (2, 1): est = 2, ind_best = 2.
    #   S = [(1, i, 1), (1, 1, i)] (sign(0) = 1);  Z = A^H S:
    #   column 0 = (-i, 0, 1 - i*i) = (-i, 0, 2); column 1 = (-i*i, 0, 1 - i) = (1, 0, 1-i)
    #   h = (1, 0, 2): max h = h[ind_best] -> stop with est = 2 (the exact norm).
    est, tr = _trace(A_ADJ, 1)
    assert est == 2.0
    assert [r["k"] for r in tr] == [1, 2]
    assert np.allclose(tr[0]["colnorms"], [1.0, 1.0], rtol=0, atol=1e-15)
    assert np.allclose(tr[0]["h"], [1.0, 0.0, 2.0], rtol=0, atol=1e-15)
    assert tr[0]["next"] == [2, 0]
    assert tr[1]["from"] == [2, 0]
    assert np.allclose(tr[1]["colnorms"], [2.0, 1.0], rtol=0, atol=1e-15)
    assert tr[1]["stop"] == "h max at ind_best"


def test_adjoint_is_conjugate_transpose_p2():
    # A^2 = [[i,0,0],[-1,0,0],[0,0,i]] (column norms 2, 0, 1: ||A^2||_1 = 2),
    # (A^2)^H = [[-i,-1,0],[0,0,0],[0,0,-i]].
    # k = 1: Y = A^2 X0 = [[i,i],[-1,-1],[i,-i]] / 3, norms (1, 1): est = 1.
    #   S = [[i,i],[-1,-1],[i,-i]];  Z = (A^2)^H S:
    #   row 0 = -i*i + (-1)(-1) = 2 (both columns); row 1 = 0; row 2 = -i*(+-i) = (1, -1)
    #   h = (2, 0, 1) -> next = [0, 2].
    #   (With (A^2)^T: row 0 = i*i + 1 = 0, row 2 = i*(+-i) -> h = (0, 0, 1), next = [2, 0].)
    # k = 2: Y = [A^2 e0, A^2 e2] = [(i,-1,0), (0,0,i)], norms (2, 1): est = 2, ind_best = 0.
    #   S = [(i,-1,1), (1,1,i)];  Z: column 0 = (2, 0, -i), column 1 = (-i-1, 0, 1)
    #   h = (2, 0, 1): max h = h[0] -> stop, est = 2.
    est, tr = _trace(A_ADJ, 2)
    assert est == 2.0
    assert np.allclose(tr[0]["h"], [2.0, 0.0, 1.0], rtol=0, atol=1e-15)
    assert tr[0]["next"] == [0, 2]
    assert np.allclose(tr[1]["colnorms"], [2.0, 1.0], rtol=0, atol=1e-15)
    assert tr[1]["stop"] == "h max at ind_best"


def test_sign_is_complex_phase():
    # A = [[2,0,1],[0,0,i],[0,1,-i]], A^H = [[2,0,0],[0,0,1],[1,-i,i]], ||A||_1 = 3
    # (column 2: 1 + 1 + 1).
    # k = 1: Y = [[3,1],[i,-i],[1-i,1+i]] / 3, norms ((4+sqrt2)/3, (2+sqrt2)/3): est = (4+sqrt2)/3.
    #   S = [[1,1],[i,-i],[(1-i)/sqrt2,(1+i)/sqrt2]];  Z = A^H S:
    #   row 0 = (2, 2); row 1 = S_2 (modulus 1, 1);
    #   row 2 = S_0 - i S_1 + i S_2 = (2 + (1+i)/sqrt2, (i-1)/sqrt2), moduli (sqrt(5+2 sqrt2), 1)
    #   h = (2, 1, sqrt(5 + 2 sqrt2) = 2.798) -> next = [2, 0].
    # k = 2: Y = [A e2, A e0] = [(1, i, -i), (2, 0, 0)], norms (3, 2): est = 3, ind_best = 2.
    #   S = [(1, i, -i), (1, 1, 1)]; Z column 0 = (2, -i, 1 + 1 + 1) -> h = (2, 1, 3):
    #   max h = h[2] -> stop with est = 3 (exact).  A real-valued sign (sign of Re z)
    #   sends iteration 2 to other columns and returns 2.
    est, tr = _trace([[2, 0, 1], [0, 0, 1j], [0, 1, -1j]], 1)
    r2 = np.sqrt(2.0)
    assert np.allclose(tr[0]["colnorms"], [(4 + r2) / 3, (2 + r2) / 3], rtol=0, atol=1e-15)
    assert np.allclose(tr[0]["h"], [2.0, 1.0, np.sqrt(5 + 2 * r2)], rtol=0, atol=1e-14)
    assert tr[0]["next"] == [2, 0]
    assert np.allclose(tr[1]["colnorms"], [3.0, 2.0], rtol=0, atol=1e-15)
    assert tr[1]["stop"] == "h max at ind_best"
    assert est == 3.0


def test_history_leaves_no_fresh_index():
    # A = [[-1,2,0],[-1,0,0],[1+i,-1,-2]]: column norms (2+sqrt2, 3, 2), ||A||_1 = 2 + sqrt2,
    # A^H = [[-1,-1,1-i],[2,0,-1],[0,0,-2]].
    # k = 1: Y = [[1,1],[-1,-1],[-2+i,2+i]] / 3, norms both (2 + sqrt5)/3: est = (2+sqrt5)/3.
    #   S = [[1,1],[-1,-1],[(-2+i)/sqrt5,(2+i)/sqrt5]];  Z = A^H S:
    #   row 0 = (1-i)S_2 -> (-1+3i)/sqrt5, (3-i)/sqrt5: moduli sqrt2, sqrt2
    #   row 1 = 2 - S_2 -> moduli sqrt((2 + 2/sqrt5)^2 + 1/5) = 2.929, sqrt((2 - 2/sqrt5)^2 + 1/5)
    #   row 2 = -2 S_2 -> modulus 2
    #   h = (sqrt2, 2.929, 2) -> next = [1, 2]; history {1, 2}.
    # k = 2: Y = [A e1, A e2] = [(2,0,-1), (0,0,-2)], norms (3, 2): est = 3, ind_best = 1.
    #   S = [(1,1,-1), (1,1,-1)]; Z = A^H S = (-3+i, 3, 2) for both columns,
    #   h = (sqrt10, 3, 2): the maximum is not at ind_best, the top two (0, 1) are not
    #   both in the history, and only index 0 is unused: fewer than t = 2 fresh unit
    #   vectors remain, so the algorithm stops with est = 3 < ||A||_1.  (Reusing a
    #   history index, or ignoring the history, would go on to column 0 and return
    #   2 + sqrt2.)
    est, tr = _trace([[-1, 2, 0], [-1, 0, 0], [1 + 1j, -1, -2]], 1)
    r5 = np.sqrt(5.0)
    assert np.allclose(tr[0]["colnorms"], [(2 + r5) / 3] * 2, rtol=0, atol=1e-15)
    assert np.allclose(tr[0]["h"], [np.sqrt(2.0), np.sqrt((2 + 2 / r5) ** 2 + 0.2), 2.0],
                       rtol=0, atol=1e-14)
    assert tr[0]["next"] == [1, 2]
    assert np.allclose(tr[1]["colnorms"], [3.0, 2.0], rtol=0, atol=1e-15)
    assert np.allclose(tr[1]["h"], [np.sqrt(10.0), 3.0, 2.0], rtol=0, atol=1e-14)
    assert tr[1]["stop"] == "no fresh index"
    assert est == 3.0
    assert normest.onenorm_power_exact(sp.csr_matrix(np.array(
        [[-1, 2, 0], [-1, 0, 0], [1 + 1j, -1, -2]])), 1) == pytest.approx(2 + np.sqrt(2.0))


def test_iteration_cap():
    # itmax = 1 on A_ADJ (trace derived above): iteration 2 still runs (the cap is
    # tested after est_old is updated, k > itmax), finds est = 2 > 1 and stops there.
    est, tr = _trace(A_ADJ, 1, itmax=1)
    assert est == 2.0
    assert [r["k"] for r in tr] == [1, 2] and tr[1]["stop"] == "itmax"
    est, tr = _trace(A_ADJ, 1, itmax=0)   # stops after the starting block
    assert est == 1.0 and tr[0]["stop"] == "itmax"


def test_start_signs_symmetric_under_transpose():
    # n = m^2: the column read as an m x m matrix (column-major) is symmetric,
    # its entries are the SplitMix64 signs of the canonical index, and it is
    # not constant (both signs occur); other n keep the plain stream.
    for m in (2, 5, 16):
        x = normest.start_signs(m * m)
        X = x.reshape((m, m), order="F")
        assert np.array_equal(X, X.T)
        raw = normest.random_signs(m * m)
        for a in range(m):
            for b in range(m):
                assert X[a, b] == raw[min(a + m * b, b + m * a)]
    assert set(normest.start_signs(256).tolist()) == {-1.0, 1.0}
    assert np.array_equal(normest.start_signs(40), normest.random_signs(40))


def test_estimate_unchanged_in_exact_arithmetic_terms_for_superoperator():
    # the estimator with the Hermitian starting column still returns a
    # reachable lower bound of ||L~^p||_1 on a walk's superoperator
    g = W.random_digraph(6, 0.4, 3)
    L = superop.superoperator(graph.lqsw_walk(graph.adjacency(g)), 0.4)
    for p in (2, 3, 5):
        ex = normest.onenorm_power_exact(L, p)
        est = normest.onenorm_power_est(L, p)
        assert ex / 10 <= est <= ex * (1 + 1e-12)
