"""Plain geometric multigrid on one scalar block of the structured node grid.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper approximates the inverse of each electrode-level block by one
algebraic-multigrid V-cycle (section 4, "Preconditioning").  On the
structured box meshes used here the same role is played by a geometric
V-cycle, written out plainly:

* coarsening by two (an odd count keeps its last fine node as a coarse
  node) along the axes with at least two elements -- given the axes'
  physical lengths, only along those whose mean element size is at most
  twice the smallest among them (see ``coarsen_flags``) -- until at most
  ``coarse_max`` nodes remain;
* trilinear prolongation P (Kronecker product of 1D linear interpolations),
  with the rows of masked-out fine nodes set to zero (phi_s has unknowns
  only at non-grounded electrode nodes);
* Galerkin coarse operators A_c = P^T A P, coarse nodes without support get
  an identity row;
* Chebyshev smoothing of degree ``degree`` on D^-1 A (D = diag A) over the
  interval [lam/ratio, lam], lam = max_i sum_j |A_ij| / A_ii (Gershgorin);
* a dense LU solve on the coarsest level;
* the result is zero on masked-out fine unknowns.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def interp_1d(n_fine_nodes, coarsen):
    """1D linear interpolation from the coarse to the fine node line.  The
    coarse nodes are the even fine nodes and, when the element count is odd,
    also the last fine node (that coarse element spans one fine element)."""
    if not coarsen:
        return sp.identity(n_fine_nodes, format="csr")
    ne = n_fine_nodes - 1
    nc = (ne + 1) // 2 + 1
    rows, cols, vals = [], [], []
    for i in range(n_fine_nodes):
        if ne % 2 == 1 and i == ne:
            rows.append(i); cols.append(nc - 1); vals.append(1.0)
        elif i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_fine_nodes, nc))


def coarsen_flags(dims, lengths=None):
    """Axes coarsened from a level with node counts ``dims``.  Without
    ``lengths``: every axis with at least two elements.  With the axes'
    physical lengths: of those, only the axes whose mean element size
    L_a / (n_a - 1) is at most twice the smallest.  The Q1 stiffness couples
    most strongly across the short element edges and a point smoother
    removes only errors that are smooth along the weak directions, so the
    weakly coupled axes are left fine until the elements are near isotropic
    (the structured-grid counterpart of algebraic coarsening along strong
    connections, which the paper's AMG performs)."""
    can = [(n - 1) >= 2 for n in dims]
    if lengths is None or not any(can):
        return tuple(can)
    h = [float(L) / (n - 1) if n >= 2 else 0.0 for L, n in zip(lengths, dims)]
    hmin = min(ha for ha, c in zip(h, can) if c)
    return tuple(c and ha <= 2.0 * hmin for c, ha in zip(can, h))


def coarse_dims(dims, flags):
    return tuple((n - 1 + 1) // 2 + 1 if f else n for n, f in zip(dims, flags))


def chebyshev(A, dinv, b, x, degree, lam, ratio):
    """Chebyshev iteration for A x = b preconditioned by D^-1 on
    [lam/ratio, lam] (the classical three-term recurrence)."""
    beta = lam
    alpha = lam / ratio
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = dinv * (b - A @ x)
    d = r / theta
    x = x + d
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = dinv * (b - A @ x)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        x = x + d
        rho = rho_new
    return x


class GMG:
    def __init__(self, A, dims, mask=None, degree=2, coarse_max=128, ratio=10.0, max_levels=20, lengths=None):
        self.degree = degree
        self.ratio = ratio
        A = sp.csr_matrix(A)
        n = A.shape[0]
        mask = np.ones(n, bool) if mask is None else np.asarray(mask, bool)
        mask0 = mask
        self.A, self.P, self.dinv, self.lam, self.dims = [], [], [], [], []
        while True:
            self._add_level(A, dims)
            flags = coarsen_flags(dims, lengths)
            if A.shape[0] <= coarse_max or not any(flags) or len(self.A) >= max_levels:
                break
            cd = coarse_dims(dims, flags)
            Pz = interp_1d(dims[2], flags[2])
            Py = interp_1d(dims[1], flags[1])
            Px = interp_1d(dims[0], flags[0])
            P = sp.kron(Pz, sp.kron(Py, Px), format="csr")
            P = sp.diags(mask.astype(float)) @ P
            Ac = (P.T @ A @ P).tocsr()
            cmask = np.asarray(abs(P).sum(axis=0)).ravel() > 0
            Ac = (Ac + sp.diags((~cmask).astype(float))).tocsr()
            self.P.append(P.tocsr())
            A, dims, mask = Ac, cd, cmask
        self.lu = sla.lu_factor(self.A[-1].toarray())
        self.mask0 = mask0

    def _add_level(self, A, dims):
        d = A.diagonal()
        self.A.append(A)
        self.dims.append(dims)
        self.dinv.append(1.0 / d)
        self.lam.append(float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / d)))

    @property
    def nlevels(self):
        return len(self.A)

    def vcycle(self, b, level=0):
        if level == self.nlevels - 1:
            x = sla.lu_solve(self.lu, b)
            if level == 0:
                x[~self.mask0] = 0.0
            return x
        A = self.A[level]
        x = chebyshev(A, self.dinv[level], b, np.zeros_like(b), self.degree, self.lam[level], self.ratio)
        r = b - A @ x
        P = self.P[level]
        x = x + P @ self.vcycle(P.T @ r, level + 1)
        x = chebyshev(A, self.dinv[level], b, x, self.degree, self.lam[level], self.ratio)
        if level == 0:
            x[~self.mask0] = 0.0          # the V-cycle acts on the masked-in unknowns only
        return x
