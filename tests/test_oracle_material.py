"""Pins of the paper's nonlinear material laws in the oracle (Appendix
"Model Parameters": eqs. ocp_cathode, ocp_anode, De_app, kappa_app).

* closed-form values of kappa(c_e) and D_e(c_e) at 1 mol/L;
* the OCP curves against the input generator's own transcription of the
  same equations (two independent transcriptions, one of them used only to
  draw the linear secants), and dU/dtheta against central differences;
* the exact Jacobian with the nonlinear laws against central differences
  of the residual;
* charge balance and lithium conservation still hold exactly after a
  Newton-converged step (they follow from the structure, not the laws).
"""
import math

import numpy as np
import pytest

from p4d_inputs import make_box_case, make_tiny_case
from p4d_inputs import generators as gen
from oracle.fe import Disc, ocp_paper, transport_paper, radial_operator
from oracle.krylov import time_step


def test_transport_closed_form_at_one_molar():
    kap, dkap, De, dDe = transport_paper(np.array([1000.0]))
    assert kap[0] == pytest.approx(0.0911 + 1.9101 - 1.052 + 0.1554, rel=1e-15)
    assert De[0] == pytest.approx(5.34e-10 * math.exp(-0.65), rel=1e-15)
    h = 1e-3
    kp, _, Dp, _ = transport_paper(np.array([1000.0 + h]))
    km, _, Dm, _ = transport_paper(np.array([1000.0 - h]))
    assert dkap[0] == pytest.approx((kp[0] - km[0]) / (2 * h), rel=1e-7)
    assert dDe[0] == pytest.approx((Dp[0] - Dm[0]) / (2 * h), rel=1e-7)


def test_ocp_matches_independent_transcription_and_its_derivative():
    u_p, u_n = gen.ocp_curve_p, gen.ocp_curve_n
    th = np.linspace(0.05, 0.95, 37)
    Up, dUp = ocp_paper(th, True)
    Un, dUn = ocp_paper(th, False)
    for t, a, b in zip(th, Up, Un):
        assert a == pytest.approx(u_p(t), rel=1e-14, abs=1e-14)
        assert b == pytest.approx(u_n(t), rel=1e-14, abs=1e-14)
    h = 1e-7
    for cath, dU in ((True, dUp), (False, dUn)):
        fd = (ocp_paper(th + h, cath)[0] - ocp_paper(th - h, cath)[0]) / (2 * h)
        assert np.allclose(dU, fd, rtol=1e-6, atol=1e-6 * np.max(np.abs(fd)))


def test_jacobian_with_paper_laws_matches_central_differences():
    case = make_tiny_case()
    d = Disc(case["mesh"], case["params"], material="paper")
    st = d.state_from_case(case["state"])
    J = d.jacobian(st).toarray()
    x0 = d.pack(st)
    for c in range(d.ndof):
        h = 1e-6 * max(abs(x0[c]), 1e-3)
        xp = x0.copy(); xp[c] += h
        xm = x0.copy(); xm[c] -= h
        fd = (d.residual(d.with_values(st, xp)) - d.residual(d.with_values(st, xm))) / (2 * h)
        scale = np.max(np.abs(J[:, c])) + 1e-300
        assert np.max(np.abs(fd - J[:, c])) <= 1e-6 * scale, c


def test_conservation_with_paper_laws():
    case = make_box_case(3, 3, (3, 2, 3), 30e-6, (40e-6, 20e-6, 40e-6), 5, 11, state="initial")
    d = Disc(case["mesh"], case["params"], material="paper")
    st0 = d.state_from_case(case["state"])
    st1, hist = time_step(d, st0, rtol=1e-13)
    assert hist[-1] < 1e-10 * hist[0]
    p = d.p
    phis_l = np.where(d.act, st1["phis"], 0.0)
    i_n, *_ = d.kinetics(phis_l, st1["phie"], st1["ce"], st1["cs"][:, -1])
    I = p["i_app"] * d.gpw.sum()
    an = d.etype == 0
    assert np.sum(d.A[~an] * i_n[~an]) == pytest.approx(I, rel=1e-9)
    assert np.sum(d.A[an] * i_n[an]) == pytest.approx(-I, rel=1e-9)
    from oracle.fe import MREF
    me = (d.eps * d.vol)[:, None, None] * MREF[None]
    tot = lambda ce: np.sum(np.einsum("elm,em->el", me, ce[d.conn]))
    assert tot(st1["ce"]) == pytest.approx(tot(st0["ce"]), rel=1e-12)
