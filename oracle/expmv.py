"""Al-Mohy--Higham truncated-Taylor expmv (oracle; test infrastructure only).

The paper (Section 3.1) computes rho~(t) = exp(t L~) rho~(0) (Eq. qsw_vec_sol)
with the scaling-and-squaring identity exp(A)u = (T_m(s^-1 A))^s u (Eqs. scale
and ss_tay, the latter read as sum_j (s^-1 A)^j / j!), using Al-Mohy & Higham's
Algorithm 3.2 (`step`) and Algorithm 5.2 (`series`) without balancing and
without the trace shift (so eta = 1).  The parameters (m*, s) come from their
Code Fragment 3.1 using the 1-norm series of A (Section 4 footnote, read as
||(tA)^p||_1 = t^p ||A^p||_1, hence d_p(tA) = t d_p(A)).

Readings of points the paper leaves open:
* p_max = 8, m_max = 55, ell = 2 columns in the norm estimator;
* theta_m for every m = 1..55 (oracle/theta_tables.json);
* m* is the smallest m reaching the minimum cost, s = max(cost / m*, 1);
* ||.||_inf of an n x n0 block is the largest row sum of moduli;
* `series(t0, dt, q)` returns the q+1 states at t_k = t0 + k dt, the first
  computed by Algorithm 3.2 with its own parameters for t0 A.

Pinned by tests/test_oracle_expmv.py (dense expm, the printed Section 4 example,
CTQW / CTRW limits, SciPy's expm_multiply) and tests/test_oracle_theta.py.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import scipy.sparse as sp

from .normest import onenorm, onenorm_power_est

M_MAX = 55
P_MAX = 8
ELL = 2
TOL = {"double": 2.0 ** -53, "single": 2.0 ** -24}

_HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(_HERE, "theta_tables.json")) as _fh:
    _TABLES = json.load(_fh)
THETA = {name: {m: _TABLES[name]["theta"][m - 1] for m in range(1, M_MAX + 1)}
         for name in ("double", "single")}


class NormInfo:
    """||A||_1 (exact) and d_p(A) = ||A^p||_1^(1/p), p >= 2, estimated on demand
    (or all at once with ``precompute``, as the paper does at construction)."""

    def __init__(self, A, precompute: bool = False, norms=None):
        self.A = sp.csr_matrix(A, dtype=np.complex128)
        self._d = {}
        if norms is not None:           # [||A||_1, ||A^2||_1, ..., ||A^9||_1]
            self.one = float(norms[0])
            for p in range(2, len(norms) + 1):
                self._d[p] = float(norms[p - 1]) ** (1.0 / p)
        else:
            self.one = onenorm(self.A)
            if precompute:
                for p in range(2, P_MAX + 2):
                    self.d(p)

    def d(self, p: int) -> float:
        if p not in self._d:
            self._d[p] = onenorm_power_est(self.A, p) ** (1.0 / p)
        return self._d[p]

    def alpha(self, p: int) -> float:
        return max(self.d(p), self.d(p + 1))


def condition_3_13(norm1: float, n0: int, theta: dict) -> bool:
    """A-H eq. (3.13): the cheap choice from ||A||_1 alone is good enough."""
    return norm1 <= 2 * ELL * P_MAX * (P_MAX + 3) * theta[M_MAX] / (n0 * M_MAX)


def select_params(info: NormInfo, t: float, n0: int = 1, precision: str = "double",
                  theta: dict | None = None):
    """Code Fragment 3.1 for the matrix tA; returns (m*, s).

    ``theta`` may replace the table by any {m: theta_m} with m_max = 55 among
    its keys (only those m are then candidates)."""
    theta = THETA[precision] if theta is None else theta
    ms = sorted(theta)
    norm1 = t * info.one
    if norm1 == 0.0:
        return 0, 1
    if condition_3_13(norm1, n0, theta):
        best_m, best_cost = None, None
        for m in ms:
            cost = m * math.ceil(norm1 / theta[m])
            if best_cost is None or cost < best_cost:
                best_m, best_cost = m, cost
        return best_m, best_cost // best_m
    best_m, best_cost = None, None
    for m in ms:
        cm = None               # C_m = min over admissible p of m * ceil(alpha_p / theta_m)
        for p in range(2, P_MAX + 1):
            if p * (p - 1) - 1 > m:
                break
            c = m * math.ceil(t * info.alpha(p) / theta[m])
            if cm is None or c < cm:
                cm = c
        if best_cost is None or cm < best_cost:
            best_m, best_cost = m, cm
    return best_m, max(best_cost // best_m, 1)


def inf_norm(B: np.ndarray) -> float:
    """||B||_inf: largest row sum of moduli (max modulus for a vector)."""
    B = np.asarray(B)
    if B.ndim == 1:
        return float(np.max(np.abs(B))) if B.size else 0.0
    return float(np.max(np.sum(np.abs(B), axis=1))) if B.size else 0.0


def expmv_step(A, b: np.ndarray, t: float, info: NormInfo | None = None, n0: int | None = None,
               precision: str = "double", stats: dict | None = None) -> np.ndarray:
    """Algorithm 3.2: exp(tA) b with truncated Taylor series and s stages."""
    A = sp.csr_matrix(A, dtype=np.complex128)
    b = np.array(b, dtype=np.complex128)
    if n0 is None:
        n0 = 1 if b.ndim == 1 else b.shape[1]
    info = info if info is not None else NormInfo(A)
    tol = TOL[precision]
    if not (t >= 0.0 and math.isfinite(t)):
        raise ValueError("t must be finite and >= 0")
    m_star, s = select_params(info, t, n0, precision)
    F = b.copy()
    B = b.copy()
    n_mv = 0
    for _ in range(s):
        c1 = inf_norm(B)
        for j in range(1, m_star + 1):
            B = (t / (s * j)) * (A @ B)
            n_mv += 1
            c2 = inf_norm(B)
            F = F + B
            if c1 + c2 <= tol * inf_norm(F):
                break
            c1 = c2
        B = F                           # eta = 1 (no shift)
    if stats is not None:
        stats.update(m=m_star, s=s, matvecs=stats.get("matvecs", 0) + n_mv)
    return F


def expmv_series(A, b: np.ndarray, t0: float, dt: float, q: int, info: NormInfo | None = None,
                 n0: int | None = None, precision: str = "double",
                 stats: dict | None = None) -> np.ndarray:
    """Algorithm 5.2: X[k] = exp((t0 + k dt) A) b for k = 0..q (q >= 1)."""
    A = sp.csr_matrix(A, dtype=np.complex128)
    b = np.array(b, dtype=np.complex128)
    if n0 is None:
        n0 = 1 if b.ndim == 1 else b.shape[1]
    info = info if info is not None else NormInfo(A)
    tol = TOL[precision]
    if stats is None:
        stats = {}
    X = np.empty((q + 1,) + b.shape, dtype=np.complex128)
    X[0] = expmv_step(A, b, t0, info, n0, precision, stats)
    if q == 0:
        return X
    h = dt
    m_star, s = select_params(info, q * dt, n0, precision)
    stats.update(series_m=m_star, series_s=s)
    if q <= s:
        for k in range(q):
            X[k + 1] = expmv_step(A, X[k], h, info, n0, precision, stats)
        return X
    d = q // s
    j = q // d
    r = q - d * j
    n_mv = 0
    Z = X[0]
    for i in range(1, j + 2):
        dd = d if i <= j else r
        if dd == 0:
            break
        K = [Z]                         # K[p] = (h A)^p Z / p!, formed once per block
        for k in range(1, dd + 1):
            F = Z.copy()
            c1 = inf_norm(Z)
            for p in range(1, m_star + 1):
                if p == len(K):
                    K.append((h / p) * (A @ K[p - 1]))
                    n_mv += 1
                term = (float(k) ** p) * K[p]
                F = F + term
                c2 = inf_norm(term)
                if c1 + c2 <= tol * inf_norm(F):
                    break
                c1 = c2
            X[k + (i - 1) * d] = F       # eta = 1
        Z = X[i * d] if i <= j else Z
    stats["matvecs"] = stats.get("matvecs", 0) + n_mv
    return X
