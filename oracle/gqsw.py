"""Global-interaction walks: G-QSW and NM-G-QSW (oracle; test infrastructure only).

G-QSW (Section 2.5.2, Eq. L_global): instead of one jump operator per arc, a
single Lindblad operator built from the whole adjacency matrix,
L_global = sum_ij G_ij |v_i><v_j| (the matrix G itself, row = destination),
enters the master equation of Eq. qsw with weight omega:

    d rho/dt = -i(1-omega)[H, rho] + omega sum_k (L_k rho L_k^dag - 1/2 {L_k^dag L_k, rho})
               + (source / sink terms, as for the L-QSW, not scaled by omega)
               + i omega [H_rot, rho]            (NM-G-QSW only, Eq. nm_gqsw)

The superoperator is formed with explicit Kronecker products per Eq.
vec_mappings (column-major vec), one `scipy.sparse.kron` per operator.

Pinned by tests/test_oracle_gqsw.py: the master equation applied to every
basis matrix with dense products, trace preservation, the omega = 0 closed
form, and the printed three-vertex example of Section 4.1.2 ([0.25, 0.25,
0.5] at t = 100, omega = 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .graph import Jump, check_simple, transition_matrix, undirected
from .superop import jump_matrix


@dataclass
class GlobalWalk:
    n_tilde: int
    H: sp.csr_matrix                  # Hermitian, n_tilde x n_tilde
    Ls: list                          # global Lindblad operators, weighted by omega
    ports: list = field(default_factory=list)   # source / sink Jumps (not omega-scaled)
    H_rot: sp.csr_matrix | None = None          # Eq. H_rot (NM-G-QSW), term +i omega [H_rot, rho]


def _embed(M, n_tilde):
    M = sp.coo_matrix(M, dtype=np.complex128)
    return sp.csr_matrix((M.data, (M.row, M.col)), shape=(n_tilde, n_tilde))


def global_walk(G, H=None, Ls=None, sources=(), sinks=(), gamma: float = 1.0) -> GlobalWalk:
    """G-QSW on digraph G: H defaults to trans(gamma, G^u) (the Laplacian), the
    Lindblad operators to [G] (Eq. L_global).  `sources` / `sinks` are
    (vertex, rate) pairs appended after the N vertices, sources first."""
    G = sp.csr_matrix(G, dtype=np.float64)
    check_simple(G)
    n = G.shape[0]
    n_tilde = n + len(sources) + len(sinks)
    if H is None:
        H = transition_matrix(gamma, undirected(G))
    H = sp.csr_matrix(H, dtype=np.complex128)
    if H.shape != (n, n):
        raise ValueError("H must be N x N")
    if H.nnz and abs(H - H.conj().T).max() > 0:
        raise ValueError("H must be Hermitian")
    if Ls is None:
        Ls = [G]
    ports = []
    for s, (v, rate) in enumerate(sources):
        ports.append(Jump(int(v), n + s, 1.0, float(rate), False))
    for z, (v, rate) in enumerate(sinks):
        ports.append(Jump(n + len(sources) + z, int(v), 1.0, float(rate), False))
    return GlobalWalk(n_tilde, _embed(H, n_tilde), [_embed(L, n_tilde) for L in Ls], ports)


def superoperator(walk: GlobalWalk, omega: float) -> sp.csr_matrix:
    """L~ of the walk in CSR (complex128, n = N~^2 rows), zeros eliminated."""
    if not (0.0 <= omega <= 1.0):
        raise ValueError("omega must lie in [0, 1]")
    nt = walk.n_tilde
    eye = sp.identity(nt, dtype=np.complex128, format="csr")
    H = walk.H
    out = -1j * (1.0 - omega) * (sp.kron(eye, H) - sp.kron(H.T, eye))
    dissipators = [(L, omega) for L in walk.Ls] + \
                  [(jump_matrix(nt, j), j.tau) for j in walk.ports]
    for L, w in dissipators:
        if w == 0.0:
            continue
        LdL = L.conj().T @ L
        out = out + w * (sp.kron(L.conj(), L) - 0.5 * (sp.kron(eye, LdL) + sp.kron(LdL.T, eye)))
    if walk.H_rot is not None and omega != 0.0:
        R = walk.H_rot
        out = out + 1j * omega * (sp.kron(eye, R) - sp.kron(R.T, eye))
    out = sp.csr_matrix(out)
    out.eliminate_zeros()
    out.sort_indices()
    return out
