"""FP64 CPU oracle of the SLAR + adaptive-weight implicit LoMaC method (arxiv 2606.29027).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement
of the paper's method in numpy float64.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import it.  The CUDA library never calls it and shares
no code with it; the only shared module is the seeded input generator
(``paper_2606_29027_b300.inputs``), which holds no arithmetic of the method.

Modules, in the order the method is built from them:

* ``grid``      -- uniform cell-centred grids, cell location, quadratic weights (Sec. 3.1)
* ``ht``        -- hierarchical-Tucker tensors for the two dimension trees used, entry
                   evaluation, densification, orthogonalisation and HSVD truncation
                   (Sec. 3.1; Supp. B.1)
* ``sl``        -- characteristic feet, the local SL-FD entry evaluator and the dense
                   full-tensor SL step (Sec. 3.1, Eq. SL_basic_formulation, Eq. tp_interp)
* ``cross``     -- adaptive cross approximation building the new HT (HTACA reading)
* ``field``     -- velocity moments and the spectral Poisson solver (Sec. 2; Sec. 3.2.3)
* ``lomac``     -- adaptive weight, weighted Gram-Schmidt, projection coefficients and the
                   reconstruction R(U) (Sec. 3.2.1-3.2.2; Supp. B)
* ``macro``     -- macroscopic residual G(U), JFNK, BE / BDF3 / DIRK3 (Sec. 3.2.3)
* ``precond``   -- block-circulant right preconditioner of the Newton-Krylov solve and the
                   preconditioned JFNK (an addition to the paper's plain JFNK)
* ``net``       -- the warm-start network: periodic convolutions, adjoints, losses, Adam
                   (an addition; the plain JFNK stays its fallback and judge)
* ``stepper``   -- SLAR, SLAR_VP (RKEI) and the LoMaC-coupled step (Fig. flowchart)
* ``dispersion``-- linear Landau / two-stream dispersion roots used as physics pins

Functions that could not be pinned to anything outside themselves say
"parity unpinned" in their docstring.
"""
