"""The two readings of the diffusion-potential term of eq. phie-weak.

The paper integrates kappa_eff (2RT(1 - t+)/F) grad(c_e)/c_e . grad(v) without
saying how the quotient is discretized.  The oracle and the CUDA path use
grad(ln c_e) with ln c_e replaced by its Q1 nodal interpolant (the "ln"
form).  The alternative is the quotient grad(c_h)/c_h of the Q1 field at the
2x2x2 Gauss points (the "quad" form), also in the oracle for this comparison.

What separates them, pinned here:
* the ln form keeps the electrolyte's discrete equilibrium exact: when
  phi_e + gamma ln c_e is the same at every node, the ionic flux vanishes
  identically, as it does in the continuous problem; the quad form leaves a
  spurious current of second order in the nodal variation of c_e;
* on smooth fields (a transient from rest) the two forms' solutions differ
  by a vanishing fraction of the discretization error, and the difference
  falls faster than that error under refinement.
The quad form's Jacobian is itself pinned by central differences.
"""
import numpy as np
import pytest

from p4d_inputs import make_box_case, make_tiny_case
from oracle.fe import Disc
from oracle.krylov import time_step


def test_quad_form_jacobian_matches_central_differences():
    case = make_tiny_case()
    d = Disc(case["mesh"], case["params"], diffpot_form="quad")
    st = d.state_from_case(case["state"])
    J = d.jacobian(st).toarray()
    x0 = d.pack(st)
    nn = d.nn
    for c in range(2 * nn, 3 * nn):              # the c_e columns carry the quotient's derivative
        h = 1e-6 * abs(x0[c])
        xp = x0.copy(); xp[c] += h
        xm = x0.copy(); xm[c] -= h
        fd = (d.residual(d.with_values(st, xp)) - d.residual(d.with_values(st, xm))) / (2 * h)
        scale = np.max(np.abs(J[:, c]))
        assert np.max(np.abs(fd - J[:, c])) <= 1e-6 * scale


def _equilibrium_state(d, st, rng):
    """phi_e = C - gamma ln c_e at every node, with phi_s = phi_e + U(theta)
    at electrode nodes so that every reaction current is zero."""
    st = dict(st)
    st["ce"] = 1000.0 * (1.0 + rng.uniform(-0.05, 0.05, d.nn))
    st["phie"] = -0.1 - d._gamma() * np.log(st["ce"])
    theta = st["cs"][:, -1] / d.cmax
    phis = np.zeros(d.nn)
    phis[d.enodes] = st["phie"][d.enodes] + d.u0 + d.u1 * theta
    st["phis"] = np.where(d.act, phis, 0.0)
    return st


def test_ln_form_keeps_discrete_equilibrium():
    case = make_box_case(3, 3, (3, 2, 3), 30e-6, (40e-6, 20e-6, 40e-6), 4, 31)
    # no grounded face: every electrode node carries a free phi_s, so zero
    # overpotential gives zero reaction current everywhere
    case["mesh"]["gamma_n"] = np.zeros_like(case["mesh"]["gamma_n"])
    out = {}
    for form in ("ln", "quad"):
        d = Disc(case["mesh"], case["params"], diffpot_form=form)
        st = _equilibrium_state(d, d.state_from_case(case["state"]), np.random.default_rng(8))
        nn = d.nn
        r_e = d.residual(st)[nn:2 * nn]
        # the conduction term alone: same phi_e with a uniform c_e
        flat = dict(st, ce=np.full(nn, 1000.0))
        out[form] = (np.linalg.norm(r_e), np.linalg.norm(d.residual(flat)[nn:2 * nn]))
    ln, scale = out["ln"]
    quad, _ = out["quad"]
    assert ln <= 1e-12 * scale
    assert quad >= 1e-5 * scale


def _transient(nz_layers, form, nsteps=4, crate=5.0):
    case = make_box_case(2, 2, nz_layers, 100e-6, (100e-6, 25e-6, 100e-6), 6, 5, state="initial")
    case["params"]["i_app"] *= crate
    d = Disc(case["mesh"], case["params"], diffpot_form=form)
    st = d.state_from_case(case["state"])
    for _ in range(nsteps):
        st, _ = time_step(d, st, rtol=1e-12)
    return d, st


@pytest.mark.slow
def test_forms_differ_far_below_discretization_error():
    """A 5C transient from rest on a laterally uniform cell at element counts
    (10, 4, 10), (20, 8, 20) and (40, 16, 40) in z: at each of the two
    coarser meshes the ln and quad solutions differ by less than 1e-4 of
    the change under one refinement, per field (phi_s, phi_e, c_e at the
    coarse nodes), and that difference shrinks by more than 4x per
    refinement while the discretization error shrinks by about 3x."""
    levels = ((10, 4, 10), (20, 8, 20), (40, 16, 40))
    sol = {(l, f): _transient(levels[l], f) for l in range(3) for f in ("ln", "quad")}
    form_diff = {}
    for lev in (0, 1):
        for f in ("phis", "phie", "ce"):
            d0, s0 = sol[lev, "ln"]
            _, sq = sol[lev, "quad"]
            _, s1 = sol[lev + 1, "ln"]
            coarse = s0[f]
            fine = s1[f].reshape(2 * d0.nz + 1, d0.nny, d0.nnx)[::2].ravel()
            fd = np.linalg.norm(coarse - sq[f])
            de = np.linalg.norm(coarse - fine)
            assert fd < 1e-4 * de, (lev, f, fd, de)
            form_diff[lev, f] = fd
    for f in ("phis", "phie", "ce"):
        assert form_diff[1, f] < form_diff[0, f] / 4.0
