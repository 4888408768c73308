"""Known-answer pins of the oracle's block preconditioner (paper section 4,
eqs. PJ and PGS).

Block Gauss-Seidel over the electrode-level blocks, with each diagonal block
solved exactly and the particle blocks eliminated exactly, is forward block
substitution.  It is therefore the exact inverse of any Jacobian whose
Schur complement S = A_mm - A_mc A_cc^-1 A_cm is block lower triangular in
the elimination order, and FGMRES preconditioned by it must converge in one
iteration; its transpose must do the same for J^T.  With the order reversed,
the same Jacobian is block upper triangular for the preconditioner, which
is then no longer exact: more than one iteration.

The triangular Jacobian is built here without the oracle's block code: the
Schur correction A_mc A_cc^-1 A_cm is formed densely with numpy, and the
upper blocks of A_mm (in the chosen order) are replaced by the matching
blocks of that correction, so that those blocks of S vanish.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from p4d_inputs import make_box_case
from oracle.fe import Disc
from oracle.blocks import BlockPrecond, scaled_system
from oracle.krylov import fgmres

ORDERS = list(itertools.permutations((0, 1, 2)))


def _case():
    case = make_box_case(3, 3, (3, 2, 3), 30e-6, (40e-6, 20e-6, 40e-6), 4, 21)
    d = Disc(case["mesh"], case["params"])
    st = d.state_from_case(case["state"])
    return d, st


def _lower_triangular(d, J, order):
    """J with the Schur complement's blocks above the diagonal (in `order`)
    made zero, by dense arithmetic independent of oracle.blocks."""
    nn = d.nn
    m = 3 * nn
    Jd = J.toarray()
    corr = Jd[:m, m:] @ np.linalg.solve(Jd[m:, m:], Jd[m:, :m])
    pos = {f: i for i, f in enumerate(order)}
    Jn = Jd.copy()
    for f in range(3):
        for g in range(3):
            if pos[g] > pos[f]:
                rf, cg = slice(f * nn, (f + 1) * nn), slice(g * nn, (g + 1) * nn)
                Jn[rf, cg] = corr[rf, cg]
    return sp.csr_matrix(Jn), Jn


def _solve(d, J, b, P, transpose):
    A = (J.T if transpose else J).tocsr()
    s, _, _ = scaled_system(d, A, b)
    Ah = sp.diags(s) @ A @ sp.diags(s)
    apply = P.apply_transpose if transpose else P.apply
    x, its, _ = fgmres(lambda v: Ah @ v, s * b, lambda v: apply(v / s) / s, rtol=1e-10,
                       restart=30, maxit=60)
    return s * x, its


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("transpose", [False, True])
def test_bgs_exact_blocks_invert_block_lower_triangular_jacobian(order, transpose):
    d, st = _case()
    Jt, Jd = _lower_triangular(d, d.jacobian(st), order)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(d.ndof) * np.sqrt(np.abs(np.diag(Jd)))
    P = BlockPrecond(d, Jt, combine="multiplicative", order=order, exact_macro=True)
    x, its = _solve(d, Jt, b, P, transpose)
    assert its == 1
    ref = np.linalg.solve(Jd.T if transpose else Jd, b)
    for sl in d.field_slices():
        assert np.linalg.norm(x[sl] - ref[sl]) <= 1e-8 * np.linalg.norm(ref[sl])
    # the reversed order sees the same Jacobian as block upper triangular
    Pr = BlockPrecond(d, Jt, combine="multiplicative", order=tuple(reversed(order)), exact_macro=True)
    assert _solve(d, Jt, b, Pr, transpose)[1] > 1
    # block Jacobi drops the lower couplings as well
    Pj = BlockPrecond(d, Jt, combine="additive", exact_macro=True)
    assert _solve(d, Jt, b, Pj, transpose)[1] > 1


@pytest.mark.parametrize("mistake", ["swapped_coupling", "coupling_sign"])
def test_bgs_pin_catches_planted_mistakes(mistake):
    """A preconditioner with a transposed coupling block or a flipped sign
    of the couplings is not exact and fails the one-iteration pin."""
    order = (1, 0, 2)
    d, st = _case()
    Jt, Jd = _lower_triangular(d, d.jacobian(st), order)
    b = np.random.default_rng(6).standard_normal(d.ndof) * np.sqrt(np.abs(np.diag(Jd)))
    P = BlockPrecond(d, Jt, combine="multiplicative", order=order, exact_macro=True)
    blk = P.blocks
    if mistake == "swapped_coupling":
        P.blocks = [[blk[g][f] if f != g else blk[f][f] for g in range(3)] for f in range(3)]
    else:
        P.blocks = [[-blk[f][g] if f != g else blk[f][f] for g in range(3)] for f in range(3)]
    assert _solve(d, Jt, b, P, False)[1] > 1
