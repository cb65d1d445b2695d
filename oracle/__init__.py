"""CPU oracle for the preconditioned CG solve of the GDML force-kernel system.

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 NumPy/SciPy code that states
what the GPU path must compute, step by step in the paper's notation.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import it; the product path (the CUDA library and its Python binding)
never does, and shares no code with it.

Modules
-------
kernel    descriptor, Jacobian, Matern-5/2 force kernel (dense and matrix-free),
          force prediction for query geometries from alpha
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11)
precond   column selection (uniform, ridge leverage, pivoted Cholesky / Alg. 1),
          Nystrom factor (Eq. 5), Woodbury core and apply (Eqs. 3-4)
solver    exact dense solve (Eq. 1) and PCG (Sec. 2.1, Eq. 2)
spectrum  SVD preconditioner (Sec. 2.2, App. A.1), spectrum and condition number of
          P^-1 K_lam (Sec. 4.1, Fig. 3), Lanczos matrix and Ritz values of a PCG run
rule_of_thumb  preconditioner size minimising the runtime model (Sec. 4.3, Eqs. 7-8, Table 1)

Pinned against: finite differences, scikit-learn's Matern kernel, symmetry /
PSD-ness / the rigid-motion null space of K, LAPACK's pivoted Cholesky
(dpstrf), SciPy's CG, the published Philox known-answer vectors, exact
dense linear algebra on tiny inputs, Eckart-Young and the bound every Nystrom
preconditioner obeys against the SVD one, explicit Krylov projections, and Table 1 with the closed-form
stationary point of Eq. 8 (see ``tests/test_oracle_*.py``).
Parity unpinned: none of the functions exported here; the learned column
scorer is not part of the oracle.
"""
