"""Oracle: plain, slow, obviously-correct CPU reference of the ADER-DG element kernels.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product library (``paper_1903_11521_gb300``) never imports, links or executes anything
here, and nothing here imports the product library.

Modules
-------
basis    exact (rational) Dubiner basis on the reference tetrahedron and triangle and the
         global matrices of the scheme: M, K^d, Khat^d, Ktilde^d, the unfactorised face
         matrices F^-_sigma and F^+_{sigma,j,h}, and the factorised R^sigma, Rhat^sigma,
         f^h (Sec. 5.1.1, Eqs. seissol:derivative .. seissol:correction_neigh).
scheme   element geometry, elastic Jacobians, star matrices, Riemann flux solvers and the
         direct FP64 evaluation of one ADER-DG step (Sec. 5.1.1).
einsum   the generic tensor operation of Eq. gentensorop by brute force over the global
         index space, equivalent sparsity patterns by Eq. compeqspp, and exhaustive
         strength reduction with the sparse cost of Sec. 4.3.
mesh     a periodic structured tetrahedral mesh and the elastic plane wave used to check
         convergence (Sec. 5, plane-wave validation).

Parity status: every function is pinned by a ``-m "not gpu"`` test in ``tests/``
(closed forms, exact rational identities, brute force, plane-wave convergence).
"""
