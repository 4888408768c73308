"""Scaling, particle Schur complement and the block preconditioner (plain).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 4 ("Linear system structure", "Preconditioning") of the paper: the
Newton Jacobian has a 4x4 block structure [phi_s, phi_e, c_e, c_s]; the c_s
block is block diagonal with one N_c x N_c tridiagonal per particle, and the
couplings to c_s touch only the particle surface node.  The paper applies
block Jacobi (eq. PJ) or block Gauss-Seidel (eq. PGS) with one multigrid
V-cycle per electrode-level block and an exact inverse of every particle
tridiagonal.

Here the particle block is eliminated exactly (block LU in c_s):
    y_c = T^-1 r_c,  r_m' = r_m - A_mc y_c,  z_m = P_macro^-1 r_m',
    z_c = y_c - T^-1 A_cm z_m,
with P_macro block Jacobi or block Gauss-Seidel over the diagonal blocks of
the Schur complement S = A_mm - A_mc T^-1 A_cm.  Because A_mc / A_cm only
touch the surface node, S differs from A_mm by a rank-one 3x3 term per
electrode node: -z_j b_j c_j^T with z_j = (T_j^-1)_NN.

Scaling (a reading: the paper states no norm).  With d = diag(J) > 0 and a
per-field weight w_f, the Krylov solve works on
    A^ = diag(s) J diag(s),  s_i = w_f(i) / sqrt(d_i),
    w_f = 1 / max(|| (b / sqrt(d))_f ||_2, (1e-14/rtol) || (sqrt(d) u)_f ||_2)
(u: the linearization state), so the scaled right-hand side has unit norm
in every field and every residual block counts equally, unless a field's
right-hand side lies below the rounding level of its own terms.  The block preconditioner P approximates
J^-1 itself (its multigrid needs the near-null vectors of the unscaled
blocks, the constants) and is mapped to the scaled space by
P^^-1 v = s^-1 * P^-1 (s^-1 * v).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mg import GMG


def field_weights(disc, J, b, u=None, rtol=1e-8):
    """d = diag(J) and w_f = 1 / max(||(b / sqrt(d))_f||, floor_f) with
    floor_f = (1e-14 / rtol) ||(sqrt(d) u)_f|| (u: the linearization state;
    0 if not given): every field's scaled right-hand side has unit norm,
    unless it lies below the rounding level of the field's own terms."""
    d = J.diagonal()
    if np.any(d <= 0):
        raise ValueError("non-positive Jacobian diagonal")
    bt = b / np.sqrt(d)
    w = np.ones(4)
    for f, sl in enumerate(disc.field_slices()):
        fl = 0.0 if u is None else (1e-14 / rtol) * np.linalg.norm((np.sqrt(d) * u)[sl])
        nf = max(np.linalg.norm(bt[sl]), fl)
        if nf > 0:
            w[f] = 1.0 / nf
    return d, w


def field_of_row(disc):
    f = np.empty(disc.ndof, np.int64)
    for k, sl in enumerate(disc.field_slices()):
        f[sl] = k
    return f


def thomas(lo, di, up, rhs):
    """Solve one tridiagonal system per row of the (n, nc) arrays (plain
    forward elimination and back substitution)."""
    n, nc = di.shape
    c = np.zeros((n, nc))
    dd = np.zeros((n, nc))
    c[:, 0] = up[:, 0] / di[:, 0]
    dd[:, 0] = rhs[:, 0] / di[:, 0]
    for i in range(1, nc):
        den = di[:, i] - lo[:, i] * c[:, i - 1]
        if i < nc - 1:
            c[:, i] = up[:, i] / den
        dd[:, i] = (rhs[:, i] - lo[:, i] * dd[:, i - 1]) / den
    x = np.zeros((n, nc))
    x[:, -1] = dd[:, -1]
    for i in range(nc - 2, -1, -1):
        x[:, i] = dd[:, i] - c[:, i] * x[:, i + 1]
    return x


class _EquilibratedLU:
    """Sparse LU of D^-1/2 A D^-1/2 (A's rows span many orders of magnitude)."""

    def __init__(self, A):
        self.sc = 1.0 / np.sqrt(np.abs(A.diagonal()))
        self.lu = spla.splu((sp.diags(self.sc) @ A @ sp.diags(self.sc)).tocsc())

    def solve(self, b):
        return self.sc * self.lu.solve(self.sc * b)


class BlockPrecond:
    """Exact particle elimination + BJ/BGS over multigrid (or exact) solves of
    the Schur diagonal blocks of the (unscaled) Jacobian J."""

    def __init__(self, disc, J, combine="additive", order=(1, 0, 2), exact_macro=False,
                 exact_schur=False, degree=2, coarse_max=128, ratio=10.0):
        nn, NE, nc = disc.nn, disc.NE, disc.nc
        self.disc, self.combine, self.order = disc, combine, tuple(order)
        Jt = sp.csr_matrix(J)
        m = 3 * nn
        self.Amm = Jt[:m, :m].tocsr()
        self.Amc = Jt[:m, m:].tocsr()
        self.Acm = Jt[m:, :m].tocsr()
        Acc = Jt[m:, m:].tocsr()
        idx = np.arange(NE)[:, None] * nc + np.arange(nc)[None, :]
        self.di = np.asarray(Acc[idx.ravel(), idx.ravel()]).reshape(NE, nc)
        self.lo = np.zeros((NE, nc))
        self.up = np.zeros((NE, nc))
        self.lo[:, 1:] = np.asarray(Acc[idx[:, 1:].ravel(), idx[:, :-1].ravel()]).reshape(NE, nc - 1)
        self.up[:, :-1] = np.asarray(Acc[idx[:, :-1].ravel(), idx[:, 1:].ravel()]).reshape(NE, nc - 1)
        eN = np.zeros((NE, nc))
        eN[:, -1] = 1.0
        self.z = thomas(self.lo, self.di, self.up, eN)[:, -1]
        # S = Amm - sum_j z_j b_j c_j^T  (b_j: column (j,N) of A_mc, c_j: row (j,N) of A_cm)
        colN = idx[:, -1]
        Bm = self.Amc[:, colN].tocsc()          # (m, NE)
        Cm = self.Acm[colN, :].tocsr()          # (NE, m)
        corr = Bm @ sp.diags(self.z) @ Cm
        self.S = (self.Amm - corr).tocsr()
        self.blocks = [[self.S[f * nn:(f + 1) * nn, g * nn:(g + 1) * nn].tocsr() for g in range(3)]
                       for f in range(3)]
        dims = (disc.nnx, disc.nny, disc.nnz)
        self.solvers = []
        for f in range(3):
            if exact_macro:
                self.solvers.append(_EquilibratedLU(self.blocks[f][f]).solve)
            elif f == 0:
                self.solvers.append(self._phis_solver(disc, dims, degree, coarse_max, ratio))
            else:
                mg = GMG(self.blocks[f][f], dims, degree=degree, coarse_max=coarse_max, ratio=ratio,
                         lengths=disc.lengths)
                self.solvers.append(mg.vcycle)
        self.idx = idx
        # exact_schur: the whole Schur complement solved by sparse LU, which
        # makes apply() the exact inverse of Jt (block LU in c_s).
        self.schur_lu = _EquilibratedLU(self.S) if exact_schur else None

    def _phis_solver(self, disc, dims, degree, coarse_max, ratio):
        """phi_s: one masked V-cycle per electrode (the two electrodes do not
        couple in S_phis,phis, and a shared coarse grid across the thin
        separator cannot represent their separate near-constant modes), plus
        the identity rows of the non-electrode and grounded nodes."""
        A = self.blocks[0][0]
        node_elec = np.full(disc.nn, -1)
        node_elec[disc.enodes] = disc.etype
        mgs = [GMG(A, dims, mask=disc.act & (node_elec == e), degree=degree,
                   coarse_max=coarse_max, ratio=ratio, lengths=disc.lengths) for e in (0, 1)]
        ina = ~disc.act
        dinv = 1.0 / A.diagonal()

        def solve(r):
            z = mgs[0].vcycle(r) + mgs[1].vcycle(r)
            z[ina] = r[ina] * dinv[ina]
            return z
        return solve

    def macro_apply(self, rm):
        if self.schur_lu is not None:
            return self.schur_lu.solve(rm)
        nn = self.disc.nn
        r = [rm[f * nn:(f + 1) * nn] for f in range(3)]
        z = [None] * 3
        if self.combine == "additive":
            for f in range(3):
                z[f] = self.solvers[f](r[f])
        else:
            done = []
            for f in self.order:
                rhs = r[f].copy()
                for g in done:
                    rhs -= self.blocks[f][g] @ z[g]
                z[f] = self.solvers[f](rhs)
                done.append(f)
        return np.concatenate(z)

    def macro_apply_transpose(self, rm):
        """Transpose of macro_apply: the V-cycles are symmetric, block
        Gauss-Seidel becomes upper triangular (reverse order, transposed
        couplings)."""
        if self.schur_lu is not None:
            raise NotImplementedError
        nn = self.disc.nn
        r = [rm[f * nn:(f + 1) * nn] for f in range(3)]
        z = [None] * 3
        if self.combine == "additive":
            for f in range(3):
                z[f] = self.solvers[f](r[f])
        else:
            done = []
            for f in reversed(self.order):
                rhs = r[f].copy()
                for g in done:
                    rhs -= self.blocks[g][f].T @ z[g]
                z[f] = self.solvers[f](rhs)
                done.append(f)
        return np.concatenate(z)

    def apply_transpose(self, r):
        """P^-T r: the transpose of ``apply`` (particle solves with T^T,
        A_mc and A_cm exchanged and transposed)."""
        m = 3 * self.disc.nn
        NE, nc = self.disc.NE, self.disc.nc
        loT = np.zeros_like(self.lo)
        upT = np.zeros_like(self.up)
        loT[:, 1:] = self.up[:, :-1]
        upT[:, :-1] = self.lo[:, 1:]
        rm, rc = r[:m], r[m:].reshape(NE, nc)
        yc = thomas(loT, self.di, upT, rc)
        rm2 = rm - self.Acm.T @ yc.ravel()
        zm = self.macro_apply_transpose(rm2)
        t = (self.Amc.T @ zm).reshape(NE, nc)
        zc = yc - thomas(loT, self.di, upT, t)
        return np.concatenate([zm, zc.ravel()])

    def apply(self, r):
        m = 3 * self.disc.nn
        NE, nc = self.disc.NE, self.disc.nc
        rm, rc = r[:m], r[m:].reshape(NE, nc)
        yc = thomas(self.lo, self.di, self.up, rc)
        rm2 = rm - self.Amc @ yc.ravel()
        zm = self.macro_apply(rm2)
        t = (self.Acm @ zm).reshape(NE, nc)
        zc = yc - thomas(self.lo, self.di, self.up, t)
        return np.concatenate([zm, zc.ravel()])


def scaled_system(disc, J, b, u=None, rtol=1e-8):
    """Return (s, d, w): s the Krylov scaling vector, d = diag J, w the
    per-field weights."""
    d, w = field_weights(disc, J, b, u, rtol)
    s = w[field_of_row(disc)] / np.sqrt(d)
    return s, d, w
