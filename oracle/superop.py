"""The vectorised L-QSW superoperator (oracle; test infrastructure only).

Written from Eq. qsw / Eq. qsw_ss (Section 2.5) and the vectorisation
identities of Eq. vec_mappings (Section 2.5.3), with column-stacking vec
(index k = i + N~ j, Eq. qsw_vec_sol's rho~_k <-> rho_ij):

    [X, Y]     <->  (I (x) X - X^T (x) I) vec(Y)
    {X, Y}     <->  (I (x) X + X^T (x) I) vec(Y)
    X Y X^dag  <->  (X^* (x) X) vec(Y)

so that

    L~ = -i(1-omega)(I (x) H - H^T (x) I)
         + sum_k w_k [ L_k^* (x) L_k - 1/2 (I (x) L_k^dag L_k + (L_k^dag L_k)^T (x) I) ],

with w_k = omega * tau_k for the graph's jump operators and w_k = tau_k for the
source/sink operators.  Every Kronecker product is formed explicitly with
scipy.sparse.kron from the operator matrices; nothing uses the condensed
per-row assembly rule (Eq. condensed_lindblads) that the library implements.

Pinned by tests/test_oracle_superop.py: a brute-force construction that applies
the master equation to each basis matrix E_ml, the nnz closed form and the
trace-preservation identity.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .graph import Walk


def jump_matrix(n_tilde: int, jump) -> sp.csr_matrix:
    return sp.csr_matrix(([jump.amp], ([jump.i], [jump.j])), shape=(n_tilde, n_tilde),
                         dtype=np.complex128)


def superoperator(walk: Walk, omega: float) -> sp.csr_matrix:
    """L~ of Eq. qsw_ss in CSR (complex128, n = N~^2 rows), zeros eliminated."""
    if not (0.0 <= omega <= 1.0):
        raise ValueError("omega must lie in [0, 1]")
    nt = walk.n_tilde
    eye = sp.identity(nt, dtype=np.complex128, format="csr")
    H = sp.csr_matrix(walk.H, dtype=np.complex128)
    coherent = -1j * (1.0 - omega) * (sp.kron(eye, H, format="csr")
                                      - sp.kron(H.T, eye, format="csr"))
    # sum_k w_k L_k^* (x) L_k, one explicit Kronecker product per operator,
    # accumulated as triplets and summed once.
    rows, cols, vals = [], [], []
    anti = sp.csr_matrix((nt, nt), dtype=np.complex128)   # sum_k w_k L_k^dag L_k
    anti_parts = []
    for jump in walk.jumps:
        wk = jump.tau * (omega if jump.omega_scaled else 1.0)
        if wk == 0.0:
            continue
        Lk = jump_matrix(nt, jump)
        sandwich = sp.kron(Lk.conj(), Lk, format="coo")
        rows.append(sandwich.row)
        cols.append(sandwich.col)
        vals.append(wk * sandwich.data)
        anti_parts.append(wk * (Lk.conj().T @ Lk))
    if anti_parts:
        anti = sp.csr_matrix(sum(anti_parts[1:], anti_parts[0]))
    n = nt * nt
    if rows:
        jump_term = sp.csr_matrix((np.concatenate(vals),
                                   (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    else:
        jump_term = sp.csr_matrix((n, n), dtype=np.complex128)
    anticomm = -0.5 * (sp.kron(eye, anti, format="csr") + sp.kron(anti.T, eye, format="csr"))
    L = sp.csr_matrix(coherent + jump_term + anticomm)
    L.eliminate_zeros()
    L.sort_indices()
    return L


def populations(rho_vec: np.ndarray, n_tilde: int) -> np.ndarray:
    """p_i = Re rho_ii = Re rho~[i + N~ i] (Section 2.4: diagonal entries are
    the vertex populations).  Works on one vector or a stack (..., n)."""
    idx = np.arange(n_tilde) * (n_tilde + 1)
    return np.real(np.asarray(rho_vec)[..., idx])
