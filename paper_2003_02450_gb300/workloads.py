"""Seeded synthetic inputs for the L-QSW time-series path.

This module only draws graphs and initial states; it holds none of the
method's arithmetic (no degrees, no Laplacian, no superoperator).  Both the
CUDA library's tests/benchmark and the FP64 CPU oracle take their inputs from
here, so the two sides see bit-identical graphs and states.

Graph convention (Eq. adjacency_graph, Section 2.1): a digraph on N vertices is
a CSR matrix G with ``G[i, j] = w(v_i, v_j)``, row = destination vertex i,
column = source vertex j (arc j -> i).  Rows are sorted by column, no
self-loops, weights strictly positive.

The paper's own graph sample sets (Section 5: line digraphs, square
lattices, Erdos-Renyi digraphs, complete digraphs, random weights) are not
available; the generators below stand in for them with the same families.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class Digraph:
    """A weighted digraph in CSR form (row = destination, column = source)."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray     # int32[nnz]
    w: np.ndarray       # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                a[i, self.col[k]] = self.w[k]
        return a


def from_arcs(n: int, dst, src, w) -> Digraph:
    """Build a sorted CSR digraph from arc lists (dst <- src, weight)."""
    dst = np.asarray(dst, dtype=np.int64)
    src = np.asarray(src, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    if dst.size:
        key = dst * n + src
        order = np.argsort(key, kind="stable")
        key = key[order]
        if np.any(key[1:] == key[:-1]):
            raise ValueError("duplicate arc")
        dst, src, w = dst[order], src[order], w[order]
    counts = np.bincount(dst, minlength=n) if dst.size else np.zeros(n, np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Digraph(n, rowptr.astype(np.int32), src.astype(np.int32), w.copy())


def from_dense(a: np.ndarray) -> Digraph:
    a = np.asarray(a, dtype=np.float64)
    dst, src = np.nonzero(a)
    return from_arcs(a.shape[0], dst, src, a[dst, src])


def cycle_graph(n: int) -> Digraph:
    """Undirected n-cycle as a digraph with both arcs of every edge, w = 1."""
    v = np.arange(n)
    dst = np.concatenate([v, v])
    src = np.concatenate([(v + 1) % n, (v - 1) % n])
    if n == 2:  # both neighbours coincide
        dst, src = v, (v + 1) % n
    return from_arcs(n, dst, src, np.ones(dst.size))


def erdos_renyi_digraph(n: int, p: float, seed: int, wlo: float = 0.5, whi: float = 1.5) -> Digraph:
    """Directed G(n, p): every ordered pair (j -> i), i != j, is an arc with
    probability p; weights uniform in [wlo, whi)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < p
    np.fill_diagonal(mask, False)
    dst, src = np.nonzero(mask)
    w = rng.uniform(wlo, whi, size=dst.size)
    return from_arcs(n, dst, src, w)


def grid_graph(rows: int, cols: int) -> Digraph:
    """4-neighbour square lattice, undirected (both arcs), w = 1, vertex r*cols + c."""
    dst, src = [], []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            for dr, dc in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < rows and 0 <= cc < cols:
                    dst.append(v)
                    src.append(rr * cols + cc)
    return from_arcs(rows * cols, dst, src, np.ones(len(dst)))


def random_regular_graph(n: int, degree: int, seed: int) -> Digraph:
    """Uniform-ish random simple `degree`-regular undirected graph (pairing
    model with restarts), returned with both arcs of every edge, w = 1."""
    if (n * degree) % 2 or degree >= n:
        raise ValueError("no simple regular graph with these parameters")
    rng = np.random.default_rng(seed)
    for _ in range(1000):
        stubs = np.repeat(np.arange(n), degree)
        rng.shuffle(stubs)
        a, b = stubs[0::2], stubs[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * n + hi
        if np.unique(key).size != key.size:
            continue
        dst = np.concatenate([a, b])
        src = np.concatenate([b, a])
        return from_arcs(n, dst, src, np.ones(dst.size))
    raise RuntimeError("pairing model did not produce a simple graph")


def erdos_renyi_mean_degree(n: int, mean_degree: float, seed: int,
                            wlo: float = 0.5, whi: float = 1.5) -> Digraph:
    return erdos_renyi_digraph(n, min(1.0, mean_degree / max(n - 1, 1)), seed, wlo, whi)


def random_digraph(n: int, p: float, seed: int, wlo: float = 0.1, whi: float = 2.0) -> Digraph:
    """Small random digraphs for brute-force checks."""
    return erdos_renyi_digraph(n, p, seed, wlo, whi)


# ---------------------------------------------------------------- states ----

def basis_state(n: int, v: int) -> np.ndarray:
    """rho0 = |v><v| as a dense complex n x n matrix."""
    r = np.zeros((n, n), dtype=np.complex128)
    r[v, v] = 1.0
    return r


def uniform_superposition(n: int) -> np.ndarray:
    """rho0 = |psi><psi| with psi = (1/sqrt n) sum_i |i>  (all entries 1/n)."""
    return np.full((n, n), 1.0 / n, dtype=np.complex128)


def maximally_mixed(n: int) -> np.ndarray:
    return np.eye(n, dtype=np.complex128) / n


def random_pure_states(n: int, count: int, seed: int) -> list[np.ndarray]:
    """`count` random pure states |psi><psi|, psi complex Gaussian, normalised."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        psi /= np.linalg.norm(psi)
        out.append(np.outer(psi, psi.conj()))
    return out


def random_density_matrix(n: int, seed: int, rank: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, rank)) + 1j * rng.standard_normal((n, rank))
    r = a @ a.conj().T
    return r / np.trace(r).real


def vec(rho: np.ndarray) -> np.ndarray:
    """Column-major vectorisation: index k = i + N*j holds rho[i, j]."""
    return np.ascontiguousarray(np.asarray(rho).reshape(-1, order="F")).astype(np.complex128)


def unvec(v: np.ndarray, n: int) -> np.ndarray:
    return np.asarray(v).reshape((n, n), order="F")


# --------------------------------------------------------------- configs ----

@dataclass
class WalkConfig:
    """One synthetic L-QSW workload."""

    name: str
    graph: Digraph
    omega: float
    rho0: np.ndarray
    t0: float
    dt: float
    steps: int
    precision: str = "c128"       # "c128" or "c64"
    sources: list = field(default_factory=list)  # [(vertex, rate)]
    sinks: list = field(default_factory=list)    # [(vertex, rate)]
    note: str = ""


def unit_ball_points(n: int, seed: int) -> np.ndarray:
    """n points uniform in the unit ball: isotropic direction, radius U^(1/3)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x * rng.uniform(0.0, 1.0, size=(n, 1)) ** (1.0 / 3.0)


def dipole_network(n: int, seed: int):
    """Disordered network of n dipoles uniform in the unit ball (Section 4.1.4):
    V_ij = -d_ij^-3 (i != j).  Returns (G, H): the complete digraph with arc
    weights |V_ij| = d_ij^-3 (jump rates) and H = V as a dense symmetric matrix."""
    x = unit_ball_points(n, seed)
    d = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    off = ~np.eye(n, dtype=bool)
    V = np.zeros((n, n))
    V[off] = -d[off] ** -3.0
    dst, src = np.nonzero(off)
    return from_arcs(n, dst, src, -V[dst, src]), V


SEED_ER1000 = 20030245
SEED_BATCH = 4096
SEED_SERVE = 5150


def cycle16() -> WalkConfig:
    """16-cycle, w = 1, H = Laplacian, omega = 0.5, rho0 = |0><0|, 100 steps on [0, 10]."""
    return WalkConfig("cycle16", cycle_graph(16), 0.5, basis_state(16, 0), 0.0, 0.1, 100,
                      note="undirected 16-cycle, superoperator 256 x 256")


def er1000() -> WalkConfig:
    """Directed G(1000, 0.01), w ~ U(0.5, 1.5), omega = 0.3, uniform superposition,
    complex128, 50 steps of dt = 0.1."""
    g = erdos_renyi_digraph(1000, 0.01, SEED_ER1000)
    return WalkConfig("er1000", g, 0.3, uniform_superposition(1000), 0.0, 0.1, 50,
                      note="Erdos-Renyi digraph N=1000 p=0.01, ~1e6 rows, ~4e7 nnz")


def grid45(precision: str = "c64") -> WalkConfig:
    """45 x 45 lattice, w = 1, omega = 0.1, rho0 = |centre><centre|, 20 steps of dt = 0.5."""
    g = grid_graph(45, 45)
    centre = 22 * 45 + 22
    return WalkConfig("grid45", g, 0.1, basis_state(2025, centre), 0.0, 0.5, 20,
                      precision=precision, note="2-D square lattice 45x45, N=2025")


SEED_EST = 7440


def est_dipole(count: int = 4, n: int = 10, omegas: int = 64, seed: int = SEED_EST,
               t_end: float = 300.0, q: int = 600):
    """Expected-survival-time sweep (Section 4.1.4): `count` dipole networks of
    n points, each with a source (rate 0.5) feeding vertex 0 and a sink (rate
    0.5) draining vertex n - 1, for omega = k / omegas, k = 1..omegas.  The
    walker starts in the source vertex.  Returns a list of dicts (G, H, omega,
    sources, sinks, rho0 as the source's basis state, sink index, t_end, q)."""
    walks = []
    for b in range(count):
        g, h = dipole_network(n, seed * 31 + b)
        nt = n + 2
        for k in range(1, omegas + 1):
            walks.append(dict(graph=g, H=h, omega=k / omegas, sources=[(0, 0.5)],
                              sinks=[(n - 1, 0.5)], rho0=basis_state(nt, n), sink=n + 1,
                              t_end=t_end, q=q, network=b))
    return walks


def batch_regular(count: int = 256, seed: int = SEED_BATCH, nmin: int = 16, nmax: int = 512,
                  rhs: int = 4):
    """`count` random 4-regular graphs, N ~ U{nmin..nmax}, omega ~ U(0,1), `rhs`
    random pure states each; complex64, 10 steps of dt = 0.2."""
    rng = np.random.default_rng(seed)
    walks = []
    for b in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        omega = float(rng.uniform(0.0, 1.0))
        g = random_regular_graph(n, 4, seed * 7919 + b)
        states = random_pure_states(n, rhs, seed * 104729 + b)
        walks.append((g, omega, states))
    return walks


def serve_requests(count: int = 2000, seed: int = SEED_SERVE, nmin: int = 32, nmax: int = 1024):
    """Request stream: ER digraphs with mean out-degree 8, N log-uniform in
    [nmin, nmax], omega ~ U(0,1), 1..100 output times of dt = 0.1, precision
    50/50 complex64/complex128, rho0 = |0><0|.  Arrival times are drawn by the
    caller (they depend on the offered load)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        omega = float(rng.uniform(0.0, 1.0))
        steps = int(rng.integers(1, 101))
        prec = "c64" if rng.random() < 0.5 else "c128"
        reqs.append(dict(n=n, omega=omega, steps=steps, dt=0.1, precision=prec,
                         graph_seed=seed * 7 + r))
    return reqs
