"""Write the full-length expected series of the ER-1000 and 45 x 45 lattice walks.

Calls only the FP64 oracle (``oracle/``) and the seeded generators
(``paper_2003_02450_gb300/workloads.py``): every stored value is the oracle's
Algorithm 5.2 series (Section 3.1) for the walk's whole time grid.

For each walk the file holds, for every output time t_k = t0 + k dt:
* ``pops[k, v]``   -- all N~ populations Re rho_vv(t_k) (Section 2.4);
* ``row[k, j]``    -- one full row rho_{r, j}(t_k) of the density matrix (r in
                      ``row_index``: vertex 0 for ER-1000, the centre for the
                      lattice, where the walk starts);
* ``sample[k, s]`` -- rho~_{idx[s]}(t_k) at ``sample_idx`` (column-major vec
                      indices i + N~ j), drawn uniformly from the upper
                      triangle i <= j with a fixed seed.

Run from the repository root:  python tests/golden/make_full_series.py [er1000|grid45]
(about 10 minutes for both on one core).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

from oracle import expmv, graph, superop          # noqa: E402
from paper_2003_02450_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
N_SAMPLE = 2048
SAMPLE_SEED = 777


def sample_upper(nt: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct vec indices i + nt j with i <= j (sorted)."""
    rng = np.random.default_rng(seed)
    chosen: set[int] = set()
    while len(chosen) < count:
        i, j = rng.integers(0, nt, size=2)
        i, j = min(i, j), max(i, j)
        chosen.add(int(i + nt * j))
    return np.array(sorted(chosen), dtype=np.int64)


def write(cfg: W.WalkConfig, row_index: int, path: str) -> None:
    t_start = time.time()
    nt = cfg.graph.n
    walk = graph.lqsw_walk(graph.adjacency(cfg.graph))
    L = superop.superoperator(walk, cfg.omega)
    info = expmv.NormInfo(L)
    stats: dict = {}
    X = expmv.expmv_series(L, W.vec(cfg.rho0), cfg.t0, cfg.dt, cfg.steps, info=info,
                           stats=stats)
    idx = sample_upper(nt, N_SAMPLE, SAMPLE_SEED)
    row = X[:, row_index + nt * np.arange(nt)]
    np.savez_compressed(
        path,
        t0=cfg.t0, dt=cfg.dt, steps=cfg.steps, omega=cfg.omega, n_tilde=nt,
        pops=superop.populations(X, nt),
        row_index=row_index, row=row,
        sample_idx=idx, sample=X[:, idx],
        oracle_m_star=stats["series_m"], oracle_s=stats["series_s"],
        oracle_matvecs=stats["matvecs"],
    )
    print(f"{cfg.name}: wrote {path} in {time.time() - t_start:.0f} s "
          f"(m*, s) = ({stats['series_m']}, {stats['series_s']}), matvecs {stats['matvecs']}")


def main(which: list[str]) -> None:
    if "er1000" in which:
        write(W.er1000(), 0, os.path.join(HERE, "er1000_series.npz"))
    if "grid45" in which:
        cfg = W.grid45("c128")
        write(cfg, 22 * 45 + 22, os.path.join(HERE, "grid45_series.npz"))


if __name__ == "__main__":
    main(sys.argv[1:] or ["er1000", "grid45"])
