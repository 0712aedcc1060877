"""Independent reference computations used to pin the oracle.

Nothing here imports the oracle's arithmetic: the master equation is applied
to basis matrices with dense numpy products, and the omega = 0 / omega = 1
limits are solved in the N x N vertex space.
"""
import numpy as np
import scipy.linalg as sl


def dense_jumps(G: np.ndarray, sources=(), sinks=()):
    """Explicit dense Lindblad operators: (matrix, weight, omega_scaled)."""
    n = G.shape[0]
    nt = n + len(sources) + len(sinks)
    out = []
    for i in range(n):
        for j in range(n):
            if G[i, j] != 0:
                L = np.zeros((nt, nt), complex)
                L[i, j] = np.sqrt(G[i, j])
                out.append((L, 1.0, True))
    for s, (v, rate) in enumerate(sources):
        L = np.zeros((nt, nt), complex)
        L[v, n + s] = 1.0
        out.append((L, rate, False))
    for z, (v, rate) in enumerate(sinks):
        L = np.zeros((nt, nt), complex)
        L[n + len(sources) + z, v] = 1.0
        out.append((L, rate, False))
    return out


def master_rhs(rho, H, jumps, omega, h_rot=None):
    """d rho / dt of the master equation, evaluated directly: the L-QSW form, or
    any list of Lindblad operators (G-QSW), plus +i omega [H_rot, rho] when a
    rotating Hamiltonian is given (the NM-G-QSW form)."""
    out = -1j * (1 - omega) * (H @ rho - rho @ H)
    if h_rot is not None:
        out = out + 1j * omega * (h_rot @ rho - rho @ h_rot)
    for L, rate, scaled in jumps:
        w = rate * (omega if scaled else 1.0)
        LdL = L.conj().T @ L
        out = out + w * (L @ rho @ L.conj().T - 0.5 * (LdL @ rho + rho @ LdL))
    return out


def brute_force_superoperator(H, jumps, omega, h_rot=None):
    """Column (m + N l) of L~ is vec(RHS(|m><l|)), column-major vec."""
    nt = H.shape[0]
    L = np.zeros((nt * nt, nt * nt), complex)
    for l in range(nt):
        for m in range(nt):
            E = np.zeros((nt, nt), complex)
            E[m, l] = 1.0
            L[:, m + nt * l] = master_rhs(E, H, jumps, omega, h_rot).reshape(-1, order="F")
    return L


def laplacian_of_undirected(G: np.ndarray) -> np.ndarray:
    Gu = np.maximum(G, G.T)
    return np.diag(Gu.sum(axis=0)) - Gu


def ctqw_density(H: np.ndarray, rho0: np.ndarray, t: float) -> np.ndarray:
    """omega = 0: rho(t) = U rho0 U^dag with U = exp(-i t H), by eigh of H."""
    ev, V = np.linalg.eigh(H)
    U = (V * np.exp(-1j * t * ev)) @ V.conj().T
    return U @ rho0 @ U.conj().T


def ctrw_populations(G: np.ndarray, p0: np.ndarray, t: float) -> np.ndarray:
    """omega = 1: dp/dt = -M p with M_ij = -G_ij, M_jj = sum_i G_ij."""
    M = np.diag(G.sum(axis=0)) - G
    return sl.expm(-t * M) @ p0
