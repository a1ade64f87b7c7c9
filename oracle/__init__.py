"""Plain FP64 CPU oracle for the mixed-basis H/S apply and eigensolve.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call,
link or execute anything in this package: only ``tests/``, the package's
``smoke()`` self-check and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` use it.  It shares no code, tables or helpers with the CUDA
library; the two meet only at the seeded inputs of
``paper_1406_4960_gb300.workloads``.

Modules follow the paper (Ren, Hsue, Chang, "A Mixed Basis Density
Functional Approach for Low Dimensional Systems with B-splines"):

* ``bspline``     §II.A, Eqs. (1)-(3): knots, Cox-de Boor recursion, derivative,
                  Gauss-Legendre planes along z.
* ``hamiltonian`` §II.B.1, Eqs. (6)-(9), (12)-(13), (16)-(17), (20): overlap,
                  kinetic, local and Kleinman-Bylander matrix elements; dense
                  assembly and a matrix-free apply written from the same
                  element formulas.
* ``eigen``       §II.C: dense generalized eigenproblem (the definition), the
                  Jacobi diagonalizer (plain C, ``jacobi.c``) and the
                  generalized Lanczos-Krylov iteration.

Units are Hartree and bohr throughout (the paper writes -nabla^2 in Rydberg).
"""
