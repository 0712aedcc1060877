"""Digraph normalisation for the L-QSW (oracle; test infrastructure only).

Follows Section 2 of the paper:
* Eq. adjacency_graph: ``G[i, j] = w(v_i, v_j)``; the worked example of
  Section 4 (omega = 1 result) fixes column = source, row = destination, i.e.
  G[i, j] is the weight of the arc j -> i.
* simple graphs only: Tr G = 0 (Section 2.1).
* undirected companion: G^u_ij = max(G_ij, G_ji) (Section 2.1).
* Eq. out_degree: OutDeg(v_j) = sum_{i != j} G_ij (a column sum).
* Eq. generator_matrix: M_ij = -gamma G_ij (i != j), M_jj = gamma OutDeg(j);
  the default Hamiltonian is this matrix for G^u with gamma = 1 (the graph
  Laplacian; the package's ``operators.trans(gamma, GU)``).
* Eq. lindblad (read as one jump operator per arc, no dephasing term):
  L_k = sqrt(G_ij) |v_i><v_j| for every arc j -> i, weighted by omega in Eq. qsw.
* Sources and sinks (Section 2.5.1, Eq. qsw_ss): extra vertices appended after
  the N graph vertices (sources first, in argument order, then sinks); a source
  s feeding vertex v adds the jump |v><s| at rate Gamma, a sink z draining v adds
  |z><v| at rate Theta; these terms are not scaled by omega and the extra
  vertices have no Hamiltonian coupling.

Pinned by tests/test_oracle_superop.py (brute-force master equation) and
tests/test_oracle_expmv.py (printed example values, CTRW/CTQW limits).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


def adjacency(g) -> sp.csr_matrix:
    """scipy CSR from a ``workloads.Digraph`` (row = destination, column = source)."""
    return sp.csr_matrix((np.asarray(g.w, dtype=np.float64),
                          np.asarray(g.col, dtype=np.int64),
                          np.asarray(g.rowptr, dtype=np.int64)), shape=(g.n, g.n))


def check_simple(G: sp.spmatrix) -> None:
    if G.shape[0] != G.shape[1]:
        raise ValueError("adjacency matrix must be square")
    if np.any(G.diagonal() != 0):
        raise ValueError("self-loop: only simple graphs are allowed (Tr G = 0)")
    if G.nnz and np.any(G.tocoo().data <= 0):
        raise ValueError("arc weights must be positive")


def undirected(G: sp.spmatrix) -> sp.csr_matrix:
    """G^u with w^u(v_i, v_j) = max(w(v_j, v_i), w(v_i, v_j))."""
    G = sp.csr_matrix(G)
    return sp.csr_matrix(G.maximum(G.T))


def out_degree(G: sp.spmatrix) -> np.ndarray:
    """OutDeg(v_j) = sum over i != j of G_ij (column sums)."""
    Gc = sp.csr_matrix(G).tolil()
    Gc.setdiag(0)
    return np.asarray(Gc.tocsr().sum(axis=0)).ravel()


def transition_matrix(gamma: float, G: sp.spmatrix) -> sp.csr_matrix:
    """Eq. generator_matrix: M_ij = -gamma G_ij (i != j), M_jj = gamma OutDeg(j)."""
    off = sp.csr_matrix(G).tolil()
    off.setdiag(0)
    off = off.tocsr()
    return sp.csr_matrix(-gamma * off + sp.diags(gamma * out_degree(G)))


@dataclass
class Jump:
    """One Lindblad operator L = amp |v_i><v_j| with dissipator weight tau."""

    i: int
    j: int
    amp: float
    tau: float
    omega_scaled: bool


@dataclass
class Walk:
    """Everything Eq. qsw_ss needs: dimension, Hamiltonian, jump operators."""

    n_tilde: int
    H: sp.csr_matrix            # n_tilde x n_tilde, real symmetric
    jumps: list                 # list[Jump]


def lqsw_walk(G: sp.spmatrix, H: sp.spmatrix | None = None, sources=(), sinks=(),
              gamma: float = 1.0) -> Walk:
    """Normalise a digraph into the operators of Eq. qsw / Eq. qsw_ss.

    ``H`` is used exactly as passed when given (the Section 4 example passes the
    adjacency matrix GU); otherwise H = trans(gamma, G^u), the Laplacian.
    ``sources`` / ``sinks`` are sequences of (vertex, rate).
    """
    G = sp.csr_matrix(G, dtype=np.float64)
    check_simple(G)
    n = G.shape[0]
    n_tilde = n + len(sources) + len(sinks)
    if H is None:
        H = transition_matrix(gamma, undirected(G))
    H = sp.csr_matrix(H, dtype=np.float64)
    if H.shape != (n, n):
        raise ValueError("H must be N x N")
    if abs(H - H.T).max() if H.nnz else 0.0:
        raise ValueError("H must be symmetric")
    Hx = sp.lil_matrix((n_tilde, n_tilde))
    Hx[:n, :n] = H
    jumps = []
    Gc = G.tocoo()
    for i, j, w in zip(Gc.row, Gc.col, Gc.data):
        jumps.append(Jump(int(i), int(j), float(np.sqrt(w)), 1.0, True))
    for s, (v, rate) in enumerate(sources):
        if not (0 <= v < n) or rate <= 0:
            raise ValueError("bad source")
        jumps.append(Jump(int(v), n + s, 1.0, float(rate), False))
    for z, (v, rate) in enumerate(sinks):
        if not (0 <= v < n) or rate <= 0:
            raise ValueError("bad sink")
        jumps.append(Jump(n + len(sources) + z, int(v), 1.0, float(rate), False))
    return Walk(n_tilde, sp.csr_matrix(Hx), jumps)
