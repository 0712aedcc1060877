"""1-norms of matrix powers (oracle; test infrastructure only).

The paper precomputes the series {||L~^p||_1, p = 1..9} when a walk is built
(Section 4, footnote on A_norms) for the Al-Mohy--Higham parameter choice.  Here:

* ``onenorm``        -- exact ||A||_1 = max_j sum_i |A_ij|.
* ``onenorm_power_exact`` -- exact ||A^p||_1 by forming A^p e_j for every j
  (small n only).
* ``onenorm_power_est`` -- the Higham--Tisseur block 1-norm estimator
  (Higham & Tisseur 2000, Algorithm 2.4) applied to A^p with t = 2 columns and
  itmax = 5, in its complex form: sign(z) = z/|z| (sign(0) = 1), products with
  (A^p)^H, and no parallel-column tests.  Its starting block is
  [ones/n, x/n] with x_i = +-1 drawn from the counter-based SplitMix64
  generator (Steele, Lea & Flood 2014): output i is mix(seed + (i+1)*phi) with
  phi = 0x9E3779B97F4A7C15 and x_i = -1 iff the top bit of that output is set;
  for n = m^2 entry a + m b uses output min(a + m b, b + m a) (`start_signs`:
  the column is a Hermitian m x m matrix).
  Ties in the row-norm sort are broken by ascending index.

Pinned by tests/test_oracle_norms.py: exact powers against dense numpy powers,
est <= exact always, est == exact on matrices where the estimator provably
hits the maximising column, SplitMix64 against its published reference
outputs, and iteration traces derived by hand for 3 x 3 complex matrices (the
column norms, row maxima, chosen unit vectors and stop reason of every
iteration): cases where A^T in place of A^H, or a real-valued sign, changes the
chosen columns and the estimate, a history that leaves no fresh unit vector
(estimate 3 where ||A||_1 = 2 + sqrt 2), and the iteration cap.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
NORMEST_SEED = 0x51535700


def splitmix64(seed: int, i: int) -> int:
    """Output number i (0-based) of SplitMix64 started at state `seed`."""
    z = (seed + (i + 1) * GOLDEN) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def random_signs(n: int, seed: int = NORMEST_SEED) -> np.ndarray:
    """x_i = -1 if the top bit of SplitMix64 output i is set, else +1 (vectorised
    uint64 arithmetic, which wraps modulo 2^64 exactly like `splitmix64`)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(n, dtype=np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) != 0, -1.0, 1.0)


def start_signs(n: int, seed: int = NORMEST_SEED) -> np.ndarray:
    """Second column of the starting block: +-1 signs from `random_signs`, drawn
    symmetric under the transpose of a vectorised m x m matrix when n = m^2.
    Entry r = a + m b takes the sign of index min(r, b + m a), so the column,
    read as an m x m matrix, is real symmetric (Hermitian).  Higham & Tisseur
    ask only for a random +-1 column; superoperators of the walks map
    Hermitian matrices to Hermitian matrices, so this choice keeps every
    iterate of the column Hermitian.  Other n: `random_signs` itself."""
    x = random_signs(n, seed)
    m = int(round(np.sqrt(n)))
    if m * m != n:
        return x
    r = np.arange(n)
    return x[np.minimum(r, (r // m) + m * (r % m))]


def onenorm(A) -> float:
    A = sp.csc_matrix(A)
    if A.shape[1] == 0:
        return 0.0
    return float(np.max(np.asarray(abs(A).sum(axis=0)).ravel()))


def onenorm_power_exact(A, p: int) -> float:
    """||A^p||_1 from the columns A^p e_j, j = 0..n-1 (dense; small n)."""
    A = sp.csr_matrix(A)
    X = np.eye(A.shape[0], dtype=np.complex128)
    for _ in range(p):
        X = A @ X
    return float(np.max(np.sum(np.abs(X), axis=0)))


def _apply_power(A, X, p):
    for _ in range(p):
        X = A @ X
    return X


def onenorm_power_est(A, p: int, t: int = 2, itmax: int = 5, seed: int = NORMEST_SEED,
                      trace: list | None = None) -> float:
    """Higham--Tisseur Algorithm 2.4 estimate of ||A^p||_1 (a lower bound).

    ``trace``, when given, receives one dict per iteration k: the column
    1-norms of Y = A^p X, the unit-vector indices X was made of (None at k = 1),
    the row maxima h of Z = (A^H)^p sign(Y) when they were formed, the indices
    chosen for the next iteration, and the reason the loop ended ("est <= est_old",
    "itmax", "h max at ind_best", "ind in history", "no fresh index")."""
    A = sp.csr_matrix(A, dtype=np.complex128)
    AH = sp.csr_matrix(A.conj().T)
    n = A.shape[0]
    if n == 0:
        return 0.0
    t = min(t, n)
    X = np.ones((n, t), dtype=np.complex128)
    if t > 1:
        X[:, 1] = start_signs(n, seed)
        for c in range(2, t):
            X[:, c] = random_signs(n, seed + c)
    X /= n
    ind_hist: list[int] = []
    est_old = 0.0
    ind = np.zeros(t, dtype=np.int64)
    ind_best = 0
    k = 1
    est = 0.0
    while True:
        Y = _apply_power(A, X, p)
        colnorms = np.sum(np.abs(Y), axis=0)
        rec = {"k": k, "colnorms": colnorms.copy(), "from": None if k == 1 else ind.tolist()}
        if trace is not None:
            trace.append(rec)
        jbest = int(np.argmax(colnorms))
        est = float(colnorms[jbest])
        if est > est_old or k == 2:
            ind_best = int(ind[jbest])
        if k >= 2 and est <= est_old:
            est = est_old
            rec["stop"] = "est <= est_old"
            break
        est_old = est
        if k > itmax:
            rec["stop"] = "itmax"
            break
        absY = np.abs(Y)
        S = np.where(absY == 0, 1.0 + 0j, Y / np.where(absY == 0, 1.0, absY))
        Z = _apply_power(AH, S, p)
        h = np.max(np.abs(Z), axis=1)
        rec["h"] = h.copy()
        if k >= 2 and np.max(h) == h[ind_best]:
            rec["stop"] = "h max at ind_best"
            break
        order = np.argsort(-h, kind="stable")   # h descending, ties by index
        if t > 1:
            if set(order[:t].tolist()) <= set(ind_hist):
                rec["stop"] = "ind in history"
                break
            fresh = []
            for i in order:             # first t indices of the sorted order not yet used
                if int(i) not in ind_hist:
                    fresh.append(int(i))
                    if len(fresh) == t:
                        break
            if len(fresh) < t:      # fewer than t unused unit vectors remain
                rec["stop"] = "no fresh index"
                break
            ind = np.array(fresh, dtype=np.int64)
        else:
            ind = order[:t].astype(np.int64)
        rec["next"] = ind.tolist()
        X = np.zeros((n, t), dtype=np.complex128)
        for c, i in enumerate(ind):
            X[i, c] = 1.0
        ind_hist.extend(int(i) for i in ind)
        k += 1
    return est


def norm_series(A, pmax: int = 9) -> np.ndarray:
    """[||A||_1 exact, est ||A^p||_1 for p = 2..pmax] (the paper's A_norms)."""
    out = np.zeros(pmax)
    out[0] = onenorm(A)
    for p in range(2, pmax + 1):
        out[p - 1] = onenorm_power_est(A, p)
    return out
