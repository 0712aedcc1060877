"""Demoralisation of a digraph for the NM-G-QSW (oracle; test infrastructure only).

Section 2.5.2, "Graph Demoralisation", in the readings fixed below (the
printed formulas are partly garbled; the three-vertex example of Section
4.1.2 pins them at unit weights):

* vertex subspaces: vertex v becomes d_v = max(1, deg_{G^u}(v)) copies v^0..v^{d-1}
  (the degree in the undirected companion: with in-degrees of G the example's
  two source vertices would vanish);
* G^{uD}: every copy of v joined to every copy of u when v ~ u in G^u, with
  weight w^u(v, u) / sqrt(d_v d_u) (Eq. nm_weight, SubDeg = d_v d_u);
* H^D = trans(1, G^{uD}) = diag(weighted degree) - G^{uD} (Eq. generator_matrix);
* L^D (Eq. dm_lind): for each arc u -> v of G with weight w, every copy u^l
  maps to sum_j F_{d_v}[j, c_v(u)] |v^j> with amplitude w / sqrt(d_v d_u),
  where c_v(u) is u's position among v's G^u neighbours (sorted) and
  F_d[j, c] = exp(2 pi i j c / d) (the Fourier matrix, not normalised: the
  example's e^-100 decay fixes the unit rate);
* H_rot (Eq. H_rot): within each subspace <v^{k+1}|H_rot|v^k> = i (k mod d)
  and the Hermitian counterpart -i; for d = 2 the single pair <v^1|H|v^0> = i;
* the initial state spreads p_v uniformly over v's subspace (diagonal), and
  Eq. nm_rho_map sums a subspace's diagonal back into p_v.

Pinned by tests/test_oracle_nm.py: the printed example at omega = 1
([e^-100, 0, 1]) and omega = 0 (the printed digits), no spontaneous
moralisation on random digraphs, and the structural properties.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import gqsw
from .graph import check_simple, undirected


def vsets(G) -> list:
    """Index arrays of the copies of each vertex in the expanded space."""
    Gu = undirected(sp.csr_matrix(G, dtype=np.float64))
    deg = np.diff(Gu.indptr)
    out, start = [], 0
    for v in range(Gu.shape[0]):
        d = max(1, int(deg[v]))
        out.append(np.arange(start, start + d))
        start += d
    return out


def _size(vs):
    return int(vs[-1][-1]) + 1


def h_demoralised(G, vs, gamma: float = 1.0) -> sp.csr_matrix:
    Gu = undirected(sp.csr_matrix(G, dtype=np.float64)).tocoo()
    nd = _size(vs)
    A = np.zeros((nd, nd))
    for v, u, w in zip(Gu.row, Gu.col, Gu.data):
        dv, du = len(vs[v]), len(vs[u])
        A[np.ix_(vs[v], vs[u])] = w / np.sqrt(dv * du)
    return sp.csr_matrix(gamma * (np.diag(A.sum(axis=0)) - A))


def l_demoralised(G, vs) -> sp.csr_matrix:
    G = sp.csr_matrix(G, dtype=np.float64)
    check_simple(G)
    Gu = undirected(G)
    nd = _size(vs)
    L = np.zeros((nd, nd), dtype=np.complex128)
    Gc = G.tocoo()
    for v, u, w in zip(Gc.row, Gc.col, Gc.data):      # arc u -> v
        nbrs = np.sort(Gu.indices[Gu.indptr[v]:Gu.indptr[v + 1]])
        c = int(np.searchsorted(nbrs, u))
        dv, du = len(vs[v]), len(vs[u])
        col = np.exp(2j * np.pi * np.arange(dv) * c / dv)
        L[np.ix_(vs[v], vs[u])] += np.outer(col, np.ones(du)) * w / np.sqrt(dv * du)
    return sp.csr_matrix(L)


def h_rot(vs) -> sp.csr_matrix:
    nd = _size(vs)
    R = np.zeros((nd, nd), dtype=np.complex128)
    for s in vs:
        d = len(s)
        if d == 2:
            R[s[1], s[0]] = 1j
            R[s[0], s[1]] = -1j
        elif d >= 3:
            for k in range(d):
                R[s[(k + 1) % d], s[k]] = 1j
                R[s[k], s[(k + 1) % d]] = -1j
    return sp.csr_matrix(R)


def nm_walk(G, gamma: float = 1.0):
    """The NM-G-QSW of G as a GlobalWalk on the expanded space, and its vsets."""
    vs = vsets(G)
    nd = _size(vs)
    walk = gqsw.global_walk(np.zeros((nd, nd)), H=h_demoralised(G, vs, gamma),
                            Ls=[l_demoralised(G, vs)])
    walk.H_rot = h_rot(vs)
    return walk, vs


def initial_state(pops, vs) -> np.ndarray:
    nd = _size(vs)
    rho = np.zeros((nd, nd), dtype=np.complex128)
    for p, s in zip(pops, vs):
        rho[s, s] = p / len(s)
    return rho


def populations(pops_expanded, vs) -> np.ndarray:
    """Eq. nm_rho_map: p(v) = sum of the diagonal over v's copies."""
    P = np.asarray(pops_expanded)
    return np.stack([P[..., s].sum(axis=-1) for s in vs], axis=-1)
