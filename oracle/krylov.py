"""Plain right-preconditioned FGMRES(m) and the scaled block-preconditioned
Newton linear solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper solves every Newton linear system with GMRES(30) (restart 100 for
the jelly roll) preconditioned by the block preconditioners of section 4
(Appendix "Solver parameters").  Because the multigrid/particle
preconditioner may be applied in reduced precision on the GPU, the flexible
variant (Saad 1993) is used: the preconditioned directions Z are stored and
the update is x += Z y.  Modified Gram-Schmidt, Givens rotations, and the
stopping test ||b - A x||_2 <= rtol ||b||_2 on the Arnoldi estimate, confirmed
by a true residual at every restart.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .blocks import BlockPrecond, scaled_system


def fgmres(A, b, M, x0=None, rtol=1e-8, restart=30, maxit=1000):
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    it = 0
    hist = []
    while True:
        r = b - A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= rtol * bnorm or it >= maxit:
            return x, it, hist
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        kk = 0
        for k in range(m):
            Z[k] = M(V[k])
            w = A(Z[k])
            for i in range(k + 1):
                H[i, k] = V[i] @ w
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            breakdown = H[k + 1, k] == 0.0
            if not breakdown:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            kk = k + 1
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) <= rtol * bnorm or it >= maxit or breakdown:
                break
        y = sla.solve_triangular(H[:kk, :kk], g[:kk])
        x = x + Z[:kk].T @ y


class LinearSolve:
    """One Newton linear system J(u) delta = -R(u) at a state, solved either
    directly (sparse LU) or by scaled block-preconditioned FGMRES."""

    def __init__(self, disc, st):
        self.disc = disc
        self.st = st
        self.J = disc.jacobian(st)
        self.b = -disc.residual(st)

    def direct(self, b=None, refine=2):
        """Sparse LU of the symmetrically Jacobi-equilibrated matrix
        D^-1/2 J D^-1/2 (the unscaled J spans ~17 orders of magnitude across
        blocks), followed by `refine` steps of iterative refinement."""
        b = self.b if b is None else b
        sc = 1.0 / np.sqrt(self.J.diagonal())
        Js = (sp.diags(sc) @ self.J @ sp.diags(sc)).tocsc()
        lu = spla.splu(Js)
        bs = sc * b
        y = lu.solve(bs)
        for _ in range(refine):
            y = y + lu.solve(bs - Js @ y)
        return sc * y

    def fgmres(self, b=None, rtol=1e-8, restart=30, maxit=2000, combine="additive",
               order=(1, 0, 2), exact_macro=False, exact_schur=False, degree=2, coarse_max=128,
               ratio=10.0):
        b = self.b if b is None else b
        s, d, w = scaled_system(self.disc, self.J, b, self.disc.pack(self.st), rtol)
        P = BlockPrecond(self.disc, self.J, combine=combine, order=order, exact_macro=exact_macro,
                         exact_schur=exact_schur, degree=degree, coarse_max=coarse_max, ratio=ratio)
        sinv = 1.0 / s
        Ah = sp.diags(s) @ self.J @ sp.diags(s)
        x_hat, its, hist = fgmres(lambda v: Ah @ v, s * b, lambda v: sinv * P.apply(sinv * v),
                                  rtol=rtol, restart=restart, maxit=maxit)
        self.last_precond = P
        return s * x_hat, its, hist


def per_field_error(disc, x, ref):
    """max over fields of ||x_f - ref_f|| / ||ref_f||."""
    errs = []
    for sl in disc.field_slices():
        nr = np.linalg.norm(ref[sl])
        errs.append(np.linalg.norm(x[sl] - ref[sl]) / (nr if nr > 0 else 1.0))
    return max(errs), errs


def newton(disc, st, rtol=1e-10, maxit=20, linear="direct", **kw):
    """Newton's method on the monolithic residual.  The paper runs its
    nonlinear solver with default settings: full Newton steps (basic line
    search); a step is halved here only while the trial state leaves the
    kinetics' domain.  The residual is measured in the Jacobi-scaled norm
    ||D^-1/2 R|| with D = |diag J| at the initial guess (the rows of R span
    ~17 orders of magnitude, so the plain 2-norm sees only the potential
    rows).  Converged when that norm has dropped by rtol or when a full step
    is at most max(rtol, 1e-13) times the state in every field (the
    residual's rounding floor)."""
    st = dict(st)
    x = disc.pack(st)
    w = 1.0 / np.sqrt(np.abs(disc.jacobian(st).diagonal()))
    r0 = np.linalg.norm(w * disc.residual(st))
    hist = [r0]
    for it in range(maxit):
        if hist[-1] <= rtol * r0:
            break
        ls = LinearSolve(disc, st)
        if linear == "direct":
            dx = ls.direct()
        else:
            dx, _, _ = ls.fgmres(**kw)
        lam = 1.0
        for _ in range(9):
            trial = disc.with_values(st, x + lam * dx)
            try:
                rn = np.linalg.norm(w * disc.residual(trial))
            except ValueError:
                rn = np.inf
            if np.isfinite(rn):
                break
            lam *= 0.5
        x = x + lam * dx
        st = disc.with_values(st, x)
        hist.append(rn)
        stol = max(rtol, 1e-13)
        tiny = all(np.linalg.norm(dx[sl]) <= stol * np.linalg.norm(x[sl]) for sl in disc.field_slices()
                   if np.linalg.norm(x[sl]) > 0)
        if tiny and lam == 1.0:
            break
    return st, hist


def time_step(disc, st, **kw):
    """One backward-Euler step: the previous concentrations become the
    current state's, then Newton."""
    st = dict(st)
    st["ce_prev"] = st["ce"].copy()
    st["cs_prev"] = st["cs"].copy()
    return newton(disc, st, **kw)
