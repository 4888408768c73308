"""Plain adjoint sensitivities of the terminal voltage after a backward-Euler
discharge, with respect to per-element bulk solid conductivity sigma,
solid diffusivity D_s and porosity eps.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Objective: V = mean of phi_s over the applied-current face Gamma_p at the
final step (phi_s = 0 on the grounded face).  Discrete adjoint of the step
residuals R_n(u_n; u_{n-1}, p) = 0:
    J_N^T lam_N = dV/du_N,   J_n^T lam_n = -(dR_{n+1}/du_n)^T lam_{n+1},
    dV/dp = -sum_n lam_n^T dR_n/dp.
dR_n/dp is written out per element from the same element matrices the
residual uses; D_s enters through the volume-weighted node means.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe import Disc, KREF, MREF, radial_operator
from .krylov import time_step


def _with_params(case, sigma_e=None, Ds_e=None, eps_e=None):
    mesh = dict(case["mesh"])
    if sigma_e is not None:
        mesh["sigma_e"] = np.asarray(sigma_e, float)
    if Ds_e is not None:
        mesh["Ds_e"] = np.asarray(Ds_e, float)
    if eps_e is not None:
        mesh["eps"] = np.asarray(eps_e, float)
    return mesh


def voltage_weights(d):
    q = np.zeros(d.ndof)
    q[:d.nn] = d.gpw / d.gpw.sum()
    return q


def forward(case, nsteps, sigma_e=None, Ds_e=None, eps_e=None, rtol=1e-13, material=None, **disc_kw):
    d = Disc(_with_params(case, sigma_e, Ds_e, eps_e), case["params"], material=material, **disc_kw)
    st = d.state_from_case(case["state"])
    states = [st]
    for _ in range(nsteps):
        st, _ = time_step(d, st, rtol=rtol, maxit=30)
        states.append(st)
    V = voltage_weights(d) @ d.pack(states[-1])
    return d, states, V


def _elem_K(d):
    Ke = np.zeros((d.nelem, 8, 8))
    for a in range(3):
        Ke += (d.vol / d.h[:, a] ** 2)[:, None, None] * KREF[a][None]
    return Ke


def dR_dp_dot(d, st, lam):
    """lam^T dR/dp for every element: (sigma, D_s, eps)."""
    p = d.p
    b = p["brug"]
    nn = d.nn
    Ke = _elem_K(d)
    Me = d.vol[:, None, None] * MREF[None]
    lam_s = np.where(d.act, lam[:nn], 0.0)[d.conn]
    lam_e = lam[nn:2 * nn][d.conn]
    lam_c = lam[2 * nn:3 * nn][d.conn]
    phis_l = np.where(d.act, st["phis"], 0.0)[d.conn]
    gam = p["diffpot_sign"] * 2 * p["R"] * p["T"] * (1 - p["tplus"]) / p["F"]
    ue = (st["phie"] + gam * np.log(st["ce"]))[d.conn]
    uc = st["ce"][d.conn]
    dc = (st["ce"] - st["ce_prev"])[d.conn]
    form = lambda l, M, u: np.einsum("el,elm,em->e", l, M, u)
    g_sig = np.where(d.el, d.eps_s_e ** b * form(lam_s, Ke, phis_l), 0.0)
    # d(eps^b coef(c_e))/d eps = (b / eps) eps^b coef(c_e)
    kap_eff, D_eff, _, _ = d.transport(st["ce"])
    g_eps = ((b / d.eps) * kap_eff * form(lam_e, Ke, ue) + form(lam_c, Me, dc) / p["dt"]
             + (b / d.eps) * D_eff * form(lam_c, Ke, uc))
    # D_s: dR_cs,j/dD_j = -M_j (L_h c_j)/D_j without the flux; dD_j/dD_e = (vol_e/8)/M_j
    lo, di, up, beta = radial_operator(d.r, d.Ds, p["F"])
    c = st["cs"]
    L = di * c
    L[:, 1:] += lo[:, 1:] * c[:, :-1]
    L[:, :-1] += up[:, :-1] * c[:, 1:]
    lcs = lam[3 * nn:].reshape(d.NE, d.nc)
    Pj = -np.sum(lcs * L, axis=1) / d.Ds          # lam^T dR_cs,j / dD_j divided by M_j
    Pn = np.zeros(nn)
    Pn[d.enodes] = Pj
    g_D = np.where(d.el, d.vol / 8.0 * Pn[d.conn].sum(axis=1), 0.0)
    return g_sig, g_D, g_eps


def gradient(case, nsteps, sigma_e=None, Ds_e=None, eps_e=None, rtol=1e-13, material=None, **disc_kw):
    """Returns (V, dV/dsigma_e, dV/dDs_e, dV/deps_e)."""
    d, states, V = forward(case, nsteps, sigma_e, Ds_e, eps_e, rtol, material, **disc_kw)
    nn = d.nn
    rhs = voltage_weights(d)
    g = [np.zeros(d.nelem) for _ in range(3)]
    for n in range(nsteps, 0, -1):
        st = dict(states[n])
        J = d.jacobian(st)
        sc = 1.0 / np.sqrt(np.abs(J.diagonal()))
        JT = (sp.diags(sc) @ J.T @ sp.diags(sc)).tocsc()
        lam = sc * spla.spsolve(JT, sc * rhs)
        for gi, v in zip(g, dR_dp_dot(d, st, lam)):
            gi -= v
        # previous-level coupling: R_n depends on c_e^{n-1} (mass) and c_s^{n-1}
        Mg = np.zeros((d.nelem, 8))
        lam_c = lam[2 * nn:3 * nn][d.conn]
        Mg = np.einsum("elm,el->em", (d.eps * d.vol)[:, None, None] * MREF[None], lam_c) / d.p["dt"]
        rhs = np.zeros(d.ndof)
        rhs[2 * nn:3 * nn] = np.bincount(d.conn.ravel(), weights=Mg.ravel(), minlength=nn)
        rhs[3 * nn:] = (d.M[:, None] / d.p["dt"] * lam[3 * nn:].reshape(d.NE, d.nc)).ravel()
    return V, g[0], g[1], g[2]
