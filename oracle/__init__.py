"""CPU oracle for the shifted-Laplace-preconditioned Helmholtz solver.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package. The product
path (the CUDA library and its Python binding) never calls it. The two share
no code: the only common inputs come from ``workloads``, which holds no
solver arithmetic.

Everything here is plain, slow and written for reading against the paper
(Kazemi, "Application of shifted-Laplace preconditioners for heterogenous
Helmholtz equation, part 1: Data modelling"):

* ``operator``    -- assembly of H (Eq. 2-3) and of the shifted Laplacian
                     (Eq. 6) as sparse matrices, in complex128.
* ``direct``      -- the exact solve u = H^-1 f by sparse LU (Eq. 4).
* ``gmres``       -- restarted, right-preconditioned GMRES (Eq. 7), with the
                     flexible variant that stores the preconditioned vectors,
                     optionally from an initial guess; GMRES on the
                     split-preconditioned system of Eq. 5; block flexible
                     GMRES (many sources sharing one block Krylov space);
                     GCRO-DR (restarted GMRES with a recycled, deflating
                     subspace kept across restarts and across the systems of
                     a frequency sweep).
* ``multigrid``   -- the geometric V-cycle used on the GPU to apply the
                     inverse of the shifted Laplacian, written out step by
                     step (Jacobi, residual, full weighting, bilinear
                     interpolation, dense coarse solve).
* ``closed_form`` -- closed forms that pin the above: the exact 1D discrete
                     solution, the continuous Green's function and a
                     manufactured 2D/3D solution.
* ``density``     -- the variable-density operator of Eq. 1, node by node.

Parity status: ``operator``, ``direct``, ``gmres``, ``multigrid`` and
``density`` are pinned by tests that do not reuse their formulas (closed
forms, brute force, invariants). The paper's figures (spectra, convergence curves, wavefields)
carry no numbers, so any comparison with them is "parity unpinned".
"""
