"""FP64 CPU oracle for the PFC block-preconditioned Rosenbrock stage solve.

TEST INFRASTRUCTURE.  This package is a plain, slow restatement of Praetorius &
Voigt, "Development and Analysis of a Block-Preconditioner for the Phase-Field
Crystal Equation" (arXiv:1501.06852), written to check the CUDA library against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls it and shares no code
with it; the only common input is the seeded generator module ``synth``.

Modules (each function cites the paper's section or equation it follows):

* ``quadrature`` - Gauss-Jacobi rules (Golub-Welsch) and collapsed simplex rules.
* ``p2``         - P2 Lagrange basis on the reference simplex (Section 3).
* ``mesh``       - structured simplicial meshes and the P2 dof lattice (Section 3, Section 7).
* ``assembly``   - M, K, N(psi) and the load vector (psi^3, phi) (Section 3, Eq. 3.4).
* ``solvers``    - Jacobi-PCG, FGMRES(30) with modified Gram-Schmidt, and the
                   block preconditioner with the Cahn-Hilliard Schur approximation
                   (Sections 4, 4.2, 7 and Table 2).
* ``rosenbrock`` - Ros3Pw stages, stage matrix A^R and right-hand side, step
                   combination and embedded step-size control (Section 3.1, Table 1).
* ``analysis``   - closed forms of the spectral analysis (Section 6: Lemma 2,
                   Lemma 3, symbol eigenvalues).

Readings taken where the paper is silent or garbled are listed where they are
used, each marked "reading".  Parity of the step-size control formula is
unpinned (the paper defers it to the literature); see ``rosenbrock.step_error``.
"""
