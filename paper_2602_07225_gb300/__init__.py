"""GB300-native (sm_103a) block-preconditioned Newton-Krylov hot path of the
pseudo-4D DFN battery model (arXiv 2602.07225).

The compute lives in the C-ABI library ``libp4d.so`` (``include/p4d.h``);
this package only marshals arguments: torch tensors on the CUDA device supply
memory and streams.  There is no CPU fallback.

One Newton linear solve of a cell::

    from p4d_inputs import make_case
    from paper_2602_07225_gb300 import P4DSolver
    case = make_case("cube8")                  # mesh, parameters, state
    s = P4DSolver(case, precision=1)           # FP32 preconditioner, FP64 FGMRES
    st = s.state_tensors(case["state"])        # device tensors of the state
    b = s.residual(st).neg_()                  # right-hand side -R(u)
    s.jacobian_update(st)                      # linearization, multigrid operators
    x, info = s.solve(b)                       # info: iterations, rel_res, timings

Many cells together: ``BatchSolver(cases).solve_all()`` (lockstep FGMRES
of all cells, autotuned smoother per grid shape).  Gradients of the
terminal voltage: ``terminal_voltage(sigma, Ds, eps, case, nsteps)`` is
differentiable through ``torch.autograd``.  One cell cut into z slabs
(domain decomposition, one handle per slab): ``SlabSolver(slab_cases(case,
nparts)).solve(...)``.
"""
from ._native import P4DError, load  # noqa: F401
from .solver import P4DSolver, SlabSolver, default_params, halo_plan  # noqa: F401
from .adjoint import TerminalVoltage, terminal_voltage  # noqa: F401
from .batch import BatchSolver, Autotuner  # noqa: F401
