"""FP64 CPU oracle for the L-QSW time series (test infrastructure only).

This package is a plain, slow, obviously-correct statement of what the GPU
library computes, written from the paper (QSW_MPI, arXiv:2003.02450) and the
Al-Mohy--Higham expmv algorithms it names (Section 3.1).  It exists so that the
CUDA path can be checked against something independent of it:

* ``graph``    -- digraph normalisation (Section 2.1-2.5, Eqs. adjacency_graph,
                  out_degree, generator_matrix, lindblad, qsw_ss).
* ``superop``  -- the vectorised superoperator built from explicit Kronecker
                  products (Section 2.5.3, Eq. vec_mappings, Eq. qsw).
* ``theta``    -- theta_m(tol) from its backward-error definition (table made
                  by ``make_theta.py`` with mpmath, stored in theta_tables.json).
* ``normest``  -- exact ||A^p||_1 and the Higham--Tisseur block estimator.
* ``expmv``    -- parameter choice (Code Fragment 3.1), Algorithm 3.2 (`step`)
                  and Algorithm 5.2 (`series`), populations.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_2003_02450_gb300``)
never imports, links or calls it, and shares no code with it.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a value or identity fixed independently of it (see the test files
named in each module's docstring).
"""
