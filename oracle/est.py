"""Expected survival time of a walk with a sink (oracle; test infrastructure only).

Section 4.1.4 (transport through a disordered network): the efficiency of
transport is the expected survival time

    eta(omega) = integral over t in [0, inf) of (1 - p_sink(t, omega)),

with p_sink the probability accumulated in the sink vertex.  The paper
evaluates it from the `series` output at q equally spaced times on [0, t_q],
with t_q late enough that p_sink is close to 1, by Simpson's rule.

* `simpson` is the composite Simpson 1/3 rule on an odd number of equally
  spaced samples (q even).
* `survival_time` follows the paper's procedure: Algorithm 5.2 populations on
  the grid t_k = k t_end / q, then Simpson on 1 - p_sink.
* `survival_time_limit` is the integral to infinity in closed form (used to pin
  the procedure): with the sink's basis state |z><z| as the only stationary
  state, rho(t) = |z><z| + r(t), r' = L r, Tr r = 0, and the trace-free part of
  L is invertible, so int_0^inf r dt = -x with L x = r(0), Tr x = 0, and
  eta = x_zz.  Dense solve; small n only.

Pinned by tests/test_oracle_est.py (Simpson against cubic polynomials and
scipy.integrate.simpson; the closed form against the classical absorption time
at omega = 1; the procedure against the closed form).
"""
from __future__ import annotations

import numpy as np

from . import expmv, superop


def simpson(y: np.ndarray, h: float) -> float:
    """h/3 (y_0 + 4 y_1 + 2 y_2 + ... + 4 y_{q-1} + y_q), q = len(y) - 1 even."""
    y = np.asarray(y, dtype=np.float64)
    q = y.shape[0] - 1
    if q < 2 or q % 2:
        raise ValueError("Simpson's rule needs an even number q >= 2 of intervals")
    total = y[0] + y[q]
    for k in range(1, q):
        total += (4.0 if k % 2 else 2.0) * y[k]
    return h / 3.0 * total


def survival_time(L, n_tilde: int, rho0_vec: np.ndarray, t_end: float, q: int, sink: int,
                  precision: str = "double"):
    """eta by the paper's procedure; returns (eta, populations (q+1) x N~)."""
    states = expmv.expmv_series(L, rho0_vec, 0.0, t_end / q, q, precision=precision)
    pops = superop.populations(states, n_tilde)
    return simpson(1.0 - pops[:, sink], t_end / q), pops


def survival_time_limit(L, n_tilde: int, rho0_vec: np.ndarray, sink: int) -> float:
    """Integral to infinity via the bordered system [[L, k], [tau^T, 0]]."""
    n = n_tilde * n_tilde
    A = np.asarray(L.todense()) if hasattr(L, "todense") else np.asarray(L)
    k = np.zeros(n, dtype=np.complex128)
    k[sink * (n_tilde + 1)] = 1.0                      # vec |z><z|
    tau = np.zeros(n, dtype=np.complex128)
    tau[np.arange(n_tilde) * (n_tilde + 1)] = 1.0     # vec(I): Tr x = tau^T x
    B = np.zeros((n + 1, n + 1), dtype=np.complex128)
    B[:n, :n] = A
    B[:n, n] = k
    B[n, :n] = tau
    rhs = np.zeros(n + 1, dtype=np.complex128)
    rhs[:n] = np.asarray(rho0_vec, dtype=np.complex128) - k
    x = np.linalg.solve(B, rhs)
    return float(np.real(x[sink * (n_tilde + 1)]))
