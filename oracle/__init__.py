"""FP64 CPU oracle for the P4D DFN Newton linear systems.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It is a
plain, slow, obviously-correct restatement of the paper's discretization
(sections 2-4) in NumPy/SciPy, independent of the CUDA path: the two share no
code, only the seeded inputs of ``p4d_inputs``.

Modules
-------
fe        mesh bookkeeping, coefficients, residual and exact Jacobian
          (sections 2-3, eqs. ce-weak, phie-weak, phis-weak, L1, L2, L0, LR, FD)
blocks    scaling, block extraction and the particle Schur complement (section 4)
mg        plain geometric multigrid on one scalar 27-point block
krylov    plain right-preconditioned FGMRES(m) and the block preconditioner
newton    Newton with direct solves, time stepping

Parity pins (checked by ``tests/test_oracle_*.py``): dense-LU brute force,
central finite differences of the residual, the sphere series solution for
constant surface flux, discrete lithium conservation, charge balance and the
reduction of a laterally uniform cube to a 1D solve.  Iteration counts and
timings against the paper are "parity unpinned" (different multigrid,
hardware and sizes).
"""
