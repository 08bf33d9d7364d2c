"""FP64 CPU oracle for one Chebyshev-filtered subspace iteration (ChFSI) step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously
correct reference that the CUDA path is checked against.  Only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The library (``paper_1903_10959_gb300``)
never imports, links or calls anything here, and nothing here imports the
library: the two share no code.  Inputs (well centres, start blocks, Lanczos
start vectors) are passed in as arrays.

Every function cites the passage of arXiv:1903.10959 (DFT-FE) it follows:

* ``fe``          -- GLL / Gauss rules, Lagrange basis, cell stiffness, mass and
                     potential matrices, DOF maps (Sec. 2.4, Eqs. fem,
                     discreteHam, hep).
* ``hamiltonian`` -- V_eff from Gaussian wells, nonlocal projectors
                     (Eqs. nlps, nonlocalHamDiscrete), the action of
                     M^{-1/2} H M^{-1/2} (Eq. hep), dense assembly for tiny meshes.
* ``chfsi``       -- Chebyshev filter (Eq. chebFilter, Sec. 3.3), CholGS
                     (Algorithm CholGS, Sec. 3.4), Rayleigh-Ritz (Sec. 3.5),
                     bound estimate, residuals and the iteration loop.
* ``density``     -- spectrum-splitting Rayleigh-Ritz (Algorithm rr), Fermi
                     level and electron density (Algorithm dc, Eq. elecDensSP).
* ``matrix_free`` -- the cell action of Eq. discreteHam by sum factorisation
                     (the matrix-free alternative named in Sec. 3.3.1) and its
                     exact flop count.
* ``kpoints``     -- the Bloch-periodic Hamiltonian H~(k) of Eq. evp
                     (Eq. ksproblemPer), local part.
* ``scf``         -- Algorithm scf on Gaussian-charge systems: periodic
                     Poisson solve (Eq. ksproblemPer), LDA exchange, ChFSI
                     passes, Fermi-Dirac density and Anderson mixing (Sec. 3.6).

Parity status: every function is pinned by ``-m "not gpu"`` tests against
closed forms, textbook rules, brute-force dense diagonalisation or
library routines, except ``chfsi.lanczos_upper_bound``, whose output is a
heuristic bound: *parity unpinned* beyond the property b >= lambda_max
(checked against dense diagonalisation on small meshes).
"""
