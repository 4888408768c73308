"""Pins of the oracle's electrode-level discretization and solvers.

* exact Jacobian vs central finite differences of the residual;
* sparse direct solve vs dense LU brute force;
* charge balance, electrolyte and solid lithium conservation after a
  Newton-converged backward-Euler step (consequences of eqs. phis-weak,
  phie-weak, ce-weak and FD);
* a laterally uniform cube reproduces an independent 1D (P2D) solve;
* exact particle elimination + exact Schur solve = one FGMRES iteration;
* multigrid convergence factor on a Poisson-type block;
* FGMRES solution vs the direct solve.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from p4d_inputs import make_case, make_box_case
from oracle.fe import Disc, radial_operator
from oracle.krylov import LinearSolve, per_field_error, newton, time_step
from oracle.mg import GMG

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _disc(case):
    d = Disc(case["mesh"], case["params"])
    return d, d.state_from_case(case["state"])


def _tiny_tab_shell(nc=4):
    """4x2 lateral tiny box with tab strips (first element column) on both
    faces and collector shells on both."""
    case = make_case("tiny", nx=4, ny=2, nc=nc)
    m = case["mesh"]
    col = np.arange(4 * 2) % 4
    m["gamma_p"] = (col < 1).astype(np.uint8)
    m["gamma_n"] = (col < 1).astype(np.uint8)
    m["shell_sigma_t_p"], m["shell_sigma_t_n"] = 3.0, 5.0
    return case


@pytest.mark.parametrize("name", ["tiny", "tiny_void", "tiny_tab_shell"])
def test_jacobian_matches_central_differences(name):
    if name == "tiny":
        case = make_case("tiny")
    elif name == "tiny_tab_shell":
        case = _tiny_tab_shell()
    else:
        case = make_case("tiny", nc=3)
        # make one electrolyte-only element inside the cathode layer and vary eps
        m = case["mesh"]
        m["region"] = m["region"].copy()
        m["region"][-1] = 3
        m["eps"] = m["eps"].copy()
        m["eps"][-1] = 1.0
        m["eps_s"] = m["eps_s"].copy()
        m["eps_s"][-1] = 0.0
    d, st = _disc(case)
    J = d.jacobian(st).toarray()
    x0 = d.pack(st)
    rng = np.random.default_rng(3)
    cols = rng.choice(d.ndof, size=min(d.ndof, 120), replace=False)
    for c in cols:
        h = 1e-6 * max(abs(x0[c]), 1e-3)
        xp = x0.copy(); xp[c] += h
        xm = x0.copy(); xm[c] -= h
        fd = (d.residual(d.with_values(st, xp)) - d.residual(d.with_values(st, xm))) / (2 * h)
        scale = np.max(np.abs(J[:, c])) + 1e-300
        assert np.max(np.abs(fd - J[:, c])) <= 1e-6 * scale, (c, np.max(np.abs(fd - J[:, c])) / scale)


def test_direct_matches_dense_lu():
    d, st = _disc(make_case("tiny"))
    ls = LinearSolve(d, st)
    x = ls.direct()
    Jd = ls.J.toarray()
    sc = 1 / np.sqrt(np.diag(Jd))
    xd = sc * np.linalg.solve(sc[:, None] * Jd * sc[None, :], sc * ls.b)
    assert per_field_error(d, x, xd)[0] < 1e-11


def _converged_step(nxy=3, layers=(3, 2, 3), nc=5, hetero=False):
    case = make_box_case(nxy, nxy, layers, 30e-6, (40e-6, 20e-6, 40e-6), nc, 11, state="initial",
                         hetero=hetero)
    d, st = _disc(case)
    st1, hist = time_step(d, st, rtol=1e-13)
    assert hist[-1] < 1e-10 * hist[0]
    return d, st, st1


def test_charge_balance_and_lithium_conservation():
    d, st0, st1 = _converged_step()
    p = d.p
    phis_l = np.where(d.act, st1["phis"], 0.0)
    i_n, *_ = d.kinetics(phis_l, st1["phie"], st1["ce"], st1["cs"][:, -1])
    area = d.gpw.sum()
    I = p["i_app"] * area
    an = d.etype == 0
    ca = ~an
    assert np.sum(d.A[ca] * i_n[ca]) == pytest.approx(I, rel=1e-9)
    assert np.sum(d.A[an] * i_n[an]) == pytest.approx(-I, rel=1e-9)
    # electrolyte lithium (consistent mass row sums): unchanged over the step
    from oracle.fe import MREF
    me = (d.eps * d.vol)[:, None, None] * MREF[None]
    tot = lambda ce: np.sum(np.einsum("elm,em->el", me, ce[d.conn]))
    assert tot(st1["ce"]) == pytest.approx(tot(st0["ce"]), rel=1e-12)
    # solid lithium: w-weighted particle averages change by -(I/F) dt per electrode
    dc = st1["cs"] - st0["cs"]
    lith = np.zeros(2)
    for j in range(d.NE):
        lo, di, up, beta = radial_operator(d.r[j:j + 1], d.Ds[j:j + 1], p["F"])
        L = np.diag(di[0]) + np.diag(lo[0, 1:], -1) + np.diag(up[0, :-1], 1)
        w = np.linalg.svd(L.T)[2][-1]
        w = w / w.sum()
        lith[d.etype[j]] += d.S[j] * (w @ dc[j])
    dt = p["dt"]
    assert lith[1] == pytest.approx(-I / p["F"] * dt, rel=1e-8)
    assert lith[0] == pytest.approx(I / p["F"] * dt, rel=1e-8)
    assert I < 0 and lith[1] > 0          # discharge: lithium enters the cathode


def test_collector_shell_energy_and_patch():
    """The shell adds sig_t times the 2D Q1 face stiffness to the phi_s rows:
    for phi = x (resp. y) over the all-active z = Lz face, phi^T dJ phi equals
    sig_t |grad phi|^2 times the face area (exact for bilinear elements), and
    a linear phi leaves the rows of interior face nodes at zero (patch test);
    on non-square faces a swapped b/a <-> a/b fails both."""
    base = make_box_case(5, 3, (2, 1, 2), (50e-6, 18e-6), (20e-6, 10e-6, 20e-6), 3, 4, state="initial")
    d0, st = _disc(base)
    m = dict(base["mesh"])
    m["shell_sigma_t_p"] = 7.0
    d1 = Disc(m, base["params"])
    dJ = (d1.jacobian(st) - d0.jacobian(st)).tocsr()[:d0.nn, :d0.nn]
    hx, hy = np.asarray(m["hx"]), np.asarray(m["hy"])
    X = np.concatenate([[0.0], np.cumsum(hx)])
    Y = np.concatenate([[0.0], np.cumsum(hy)])
    kk, jj, ii = np.indices((d0.nnz, d0.nny, d0.nnx))
    top = kk.ravel() == d0.nz
    Lx, Ly = X[-1], Y[-1]
    for coord, grad2 in ((X[ii.ravel()], 1.0), (Y[jj.ravel()], 1.0)):
        phi = np.where(top, coord, 0.0)
        assert phi @ (dJ @ phi) == pytest.approx(7.0 * grad2 * Lx * Ly, rel=1e-12)
        r = dJ @ phi
        inner = top & (ii.ravel() > 0) & (ii.ravel() < d0.nx) & (jj.ravel() > 0) & (jj.ravel() < d0.ny)
        assert np.max(np.abs(r[inner])) <= 1e-12 * np.max(np.abs(r))
    assert abs(dJ[~top][:, ~top]).sum() == 0.0      # only face rows and columns change


def test_tab_charge_balance():
    """With the applied current and the ground on tab strips and the current
    spread by collector shells, a converged step still balances charge: the
    cathode reaction current equals i_app times the tab area."""
    from p4d_inputs import make_slab_case
    case = make_slab_case(nx=8, ny=2, layers=(3, 2, 3), nc=5, tab=2, crate=1.0, h_lat=8e-6,
                          L_layers=(30e-6, 15e-6, 30e-6))
    d, st = _disc(case)
    st1, hist = time_step(d, st, rtol=1e-13)
    phis_l = np.where(d.act, st1["phis"], 0.0)
    i_n, *_ = d.kinetics(phis_l, st1["phie"], st1["ce"], st1["cs"][:, -1])
    tab_area = 2 * 2 * 8e-6 * 8e-6
    assert d.gpw.sum() == pytest.approx(tab_area, rel=1e-14)
    I = case["params"]["i_app"] * tab_area
    ca = d.etype == 1
    assert np.sum(d.A[ca] * i_n[ca]) == pytest.approx(I, rel=1e-9)
    assert np.sum(d.A[~ca] * i_n[~ca]) == pytest.approx(-I, rel=1e-9)
    # the grounded nodes are exactly the tab's bottom nodes
    assert d.dirichlet.sum() == 3 * 3


def _p2d_residual(z_h, region, p, nc, R, D, u, prev, eps_e=0.3, eps_s=(0.6, 0.5)):
    """Independent 1D restatement (per unit area) of the same equations on a
    line of linear elements: used only to pin the 3D assembly."""
    nz = len(z_h)
    nn = nz + 1
    b = p["brug"]
    an_n = np.zeros(nn, bool); ca_n = np.zeros(nn, bool)
    for e in range(nz):
        if region[e] == 0: an_n[e] = an_n[e + 1] = True
        if region[e] == 2: ca_n[e] = ca_n[e + 1] = True
    en = np.flatnonzero(an_n | ca_n)
    NE = len(en)
    phis, phie, ce = u[:nn], u[nn:2 * nn], u[2 * nn:3 * nn]
    cs = u[3 * nn:].reshape(NE, nc)
    cep, csp = prev
    act = an_n | ca_n
    act[0] = False                                  # grounded face z = 0
    phis_l = np.where(act, phis, 0.0)
    Rs = np.zeros(nn); Re = np.zeros(nn); Rc = np.zeros(nn)
    Mw = np.zeros(nn); Sw = np.zeros(nn)
    kp = p["diffpot_sign"] * 2 * p["R"] * p["T"] * (1 - p["tplus"]) / p["F"]
    for e in range(nz):
        h = z_h[e]
        el = region[e] in (0, 2)
        eps = eps_e if el else 1.0
        es = eps_s[0] if region[e] == 0 else (eps_s[1] if region[e] == 2 else 0.0)
        sig = es ** b * (p["sigma_n"] if region[e] == 0 else p["sigma_p"]) if el else 0.0
        kap = eps ** b * p["kappa"]
        De = eps ** b * p["De"]
        k2 = np.array([[1, -1], [-1, 1]]) / h
        m2 = np.array([[2, 1], [1, 2]]) * h / 6
        ix = [e, e + 1]
        Rs[ix] += sig * k2 @ phis_l[ix]
        Re[ix] += kap * k2 @ phie[ix]
        Rc[ix] += eps * m2 @ (ce[ix] - cep[ix]) / p["dt"] + De * k2 @ ce[ix]
        Re[ix] += kap * kp * k2 @ np.log(ce[ix])
        if el:
            Mw[ix] += h / 2
            Sw[ix] += es * h / 2
    A = 3 * Sw[en] / R
    M = Mw[en]
    an = an_n[en]
    kr = np.where(an, p["k_n"], p["k_p"]); cm = np.where(an, p["cmax_n"], p["cmax_p"])
    u0 = np.where(an, p["ocp_n"][0], p["ocp_p"][0]); u1 = np.where(an, p["ocp_n"][1], p["ocp_p"][1])
    cN = cs[:, -1]
    f = p["F"] / (p["R"] * p["T"])
    eta = phis_l[en] - phie[en] - (u0 + u1 * cN / cm)
    i_n = 2 * kr * np.sqrt(ce[en] * (cm - cN) * cN) * np.sinh(0.5 * f * eta)
    tau = (1 - p["tplus"]) / p["F"]
    Rs[en] += A * i_n; Re[en] -= A * i_n; Rc[en] -= tau * A * i_n
    Rs[-1] -= p["i_app"]
    Rs[~act] = phis[~act]
    r = np.linspace(0, R, nc)
    lo, di, up, beta = radial_operator(np.tile(r, (NE, 1)), np.full(NE, D), p["F"])
    L = di * cs
    L[:, 1:] += lo[:, 1:] * cs[:, :-1]
    L[:, :-1] += up[:, :-1] * cs[:, 1:]
    L[:, -1] -= beta * i_n
    Rp = M[:, None] * ((cs - csp) / p["dt"] - L)
    return np.concatenate([Rs, Re, Rc, Rp.ravel()]), en


def test_laterally_uniform_cube_is_p2d():
    layers, nc = (3, 2, 3), 4
    Lz = (30e-6, 12e-6, 30e-6)
    case = make_box_case(2, 2, layers, 20e-6, Lz, nc, 5, state="initial")
    d, st = _disc(case)
    st1, hist = time_step(d, st, rtol=1e-13)
    p = d.p
    z_h = case["mesh"]["hz"]
    region = case["mesh"]["region"][::4]
    nz = len(z_h); nn1 = nz + 1
    # 1D initial state = one column of the 3D state
    col = lambda a: a.reshape(nz + 1, 3, 3)[:, 0, 0]
    an_n = np.zeros(nn1, bool); ca_n = np.zeros(nn1, bool)
    for e in range(nz):
        if region[e] == 0: an_n[e] = an_n[e + 1] = True
        if region[e] == 2: ca_n[e] = ca_n[e + 1] = True
    en1 = np.flatnonzero(an_n | ca_n)
    cs0 = np.where(an_n[en1], 0.8 * p["cmax_n"], 0.6 * p["cmax_p"])[:, None] * np.ones(nc)
    u = np.concatenate([col(st["phis"]), col(st["phie"]), col(st["ce"]), cs0.ravel()])
    prev = (col(st["ce"]), cs0.copy())
    for _ in range(30):
        F0, _ = _p2d_residual(z_h, region, p, nc, 5e-6, 1e-14, u, prev)
        n = u.size
        Jn = np.zeros((n, n))
        for c in range(n):
            h = 1e-7 * max(abs(u[c]), 1e-2)
            up_ = u.copy(); up_[c] += h
            um_ = u.copy(); um_[c] -= h
            Jn[:, c] = (_p2d_residual(z_h, region, p, nc, 5e-6, 1e-14, up_, prev)[0]
                        - _p2d_residual(z_h, region, p, nc, 5e-6, 1e-14, um_, prev)[0]) / (2 * h)
        sc = 1 / np.sqrt(np.abs(np.diag(Jn)))
        du = -sc * np.linalg.solve(sc[:, None] * Jn * sc[None, :], sc * F0)
        u = u + du
        if np.max(np.abs(du[:nn1])) < 1e-13 and np.max(np.abs(du[3 * nn1:] / 1e4)) < 1e-13:
            break
    for f, key in enumerate(["phis", "phie", "ce"]):
        a3 = st1[key].reshape(nz + 1, 3, 3)
        # laterally uniform
        assert np.max(np.abs(a3 - a3[:, :1, :1])) <= 1e-9 * (np.max(np.abs(a3)) + 1e-3)
        ref = u[f * nn1:(f + 1) * nn1]
        assert np.max(np.abs(a3[:, 0, 0] - ref)) <= 1e-8 * (np.max(np.abs(ref)) + 1e-3), key
    cs3 = st1["cs"][np.searchsorted(d.enodes, np.array([(k * 9) for k in en1]))]
    assert np.max(np.abs(cs3 - u[3 * nn1:].reshape(-1, nc))) <= 1e-8 * 1e4


def test_exact_schur_preconditioner_is_inverse():
    d, st = _disc(make_case("cube8"))
    ls = LinearSolve(d, st)
    x, its, hist = ls.fgmres(rtol=1e-10, exact_schur=True)
    assert its == 1


@pytest.mark.parametrize("combine", ["additive", "multiplicative"])
def test_fgmres_matches_direct(combine):
    d, st = _disc(make_case("cube8"))
    ls = LinearSolve(d, st)
    xd = ls.direct()
    x, its, hist = ls.fgmres(rtol=1e-10, combine=combine)
    assert per_field_error(d, x, xd)[0] <= 1e-9
    assert its < 60


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("block,limit", [(1, 0.25), (2, 0.25), ("phis_anode", 0.3), ("phis_cathode", 0.3)])
def test_multigrid_convergence_factor(block, limit, odd):
    """V(2,2) Chebyshev multigrid as a stationary iteration: textbook
    convergence factors on the electrolyte blocks (Q1 Laplacian plus mass or
    reaction) and on each electrode's masked phi_s block; also with odd
    element counts (coarse grids keeping the last fine node)."""
    if odd:
        case = make_box_case(15, 13, (7, 3, 7), 100e-6, (45e-6, 20e-6, 45e-6), 3, 1, state="initial")
    else:
        case = make_box_case(16, 16, (6, 4, 6), 100e-6, (40e-6, 25e-6, 40e-6), 3, 1, state="initial")
    d, st = _disc(case)
    J = d.jacobian(st)
    nn = d.nn
    f = block if isinstance(block, int) else 0
    A = J[f * nn:(f + 1) * nn, f * nn:(f + 1) * nn].tocsr()
    mask = None
    if not isinstance(block, int):
        e = 0 if block == "phis_anode" else 1
        node_elec = np.full(nn, -1)
        node_elec[d.enodes] = d.etype
        mask = d.act & (node_elec == e)
    mg = GMG(A, (d.nnx, d.nny, d.nnz), mask=mask)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(nn)
    if mask is not None:
        x[~mask] = 0.0
    e0 = np.linalg.norm(x)
    for _ in range(10):
        x = x + mg.vcycle(-(A @ x))
    rho = (np.linalg.norm(x) / e0) ** 0.1
    # odd element counts leave one coarse element of half width per axis and
    # level, which costs a few hundredths in the factor
    assert rho < limit + (0.05 if odd else 0.0), rho


def test_printed_parameters_and_dof_counts():
    g = json.load(open(os.path.join(GOLDEN, "paper_printed_values.json")))
    for side in ("cathode", "anode"):
        v = g[side]
        assert 3 * v["eps_s"] / v["R_s"] == pytest.approx(v["a"], rel=1e-12)
    for case in ("case_I_mesh", "case_III_mesh"):
        v = g[case]
        ex, ey, ez = v["elements_xyz"]
        nelem = ex * ey * ez
        assert nelem == pytest.approx(v["elements"], rel=0.01)
        assert 3 * (ex + 1) * (ey + 1) * (ez + 1) == pytest.approx(v["electrode_dofs"], rel=0.03)
        assert v["N_c"] * nelem == pytest.approx(v["particle_dofs"], rel=0.01)
        assert 3 * (ex + 1) * (ey + 1) * (ez + 1) + v["N_c"] * nelem == pytest.approx(v["total_dofs"], rel=0.01)


@pytest.mark.parametrize("combine", ["additive", "multiplicative"])
def test_preconditioner_transpose_is_adjoint(combine):
    """<P^-1 x, y> = <x, P^-T y>: the V-cycles are symmetric and the
    transposed block elimination is the exact adjoint."""
    case = make_box_case(4, 4, (4, 2, 4), 30e-6, (40e-6, 15e-6, 40e-6), 4, 3)
    d, st = _disc(case)
    from oracle.blocks import BlockPrecond
    P = BlockPrecond(d, d.jacobian(st), combine=combine, coarse_max=16)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(d.ndof)
    y = rng.standard_normal(d.ndof)
    a = P.apply(x) @ y
    b = x @ P.apply_transpose(y)
    assert abs(a - b) <= 1e-10 * (abs(a) + np.linalg.norm(P.apply(x)) * np.linalg.norm(y) * 1e-6)


def test_coarsening_follows_strong_coupling():
    """The coarsening rule: an axis with >= 2 elements is coarsened only while
    its mean element size is within twice the smallest; without lengths every
    such axis is."""
    from oracle.mg import coarsen_flags, coarse_dims
    L = (100e-6, 100e-6, 225e-6)                       # cube128: 0.78 / 0.78 / 2.34 um
    assert coarsen_flags((129, 129, 97), L) == (True, True, False)
    assert coarsen_flags((65, 65, 97), L) == (True, True, True)
    assert coarsen_flags((129, 129, 97)) == (True, True, True)
    assert coarsen_flags((9, 9, 13), (1.0, 1.0, 1.5)) == (True, True, True)   # isotropic enough
    assert coarsen_flags((9, 2, 13), (1.0, 5.0, 1.0)) == (True, False, True)  # one element: kept
    assert coarsen_flags((2, 2, 2), (1.0, 1.0, 1.0)) == (False, False, False)
    # slab-like: z kept for two levels, then everything
    dims, seq = (2049, 17, 49), []
    Ls = (2048 * 100e-6 / 128, 16 * 100e-6 / 128, 225e-6)
    for _ in range(3):
        f = coarsen_flags(dims, Ls)
        seq.append(f)
        dims = coarse_dims(dims, f)
    assert seq == [(True, True, False), (True, True, False), (True, True, True)]


def test_multigrid_factor_with_anisotropic_coarsening():
    """V-cycle convergence factor on the phi_e block of a box with 3.2:1
    elements (the bench's aspect ratio): with x, y-only coarsening on the
    first level it is well below the factor with full coarsening."""
    from oracle.mg import GMG
    case = make_box_case(32, 32, (10, 4, 10), 100e-6, (100e-6, 25e-6, 100e-6), 3, 1, state="initial")
    d, st = _disc(case)
    J = d.jacobian(st)
    nn = d.nn
    A = J[nn:2 * nn, nn:2 * nn].tocsr()
    rho = {}
    for name, lengths in (("full", None), ("strong", d.lengths)):
        mg = GMG(A, (d.nnx, d.nny, d.nnz), degree=2, ratio=10.0, lengths=lengths)
        x = np.random.default_rng(0).standard_normal(nn)
        e0 = np.linalg.norm(x)
        for _ in range(10):
            x = x + mg.vcycle(-(A @ x))
        rho[name] = (np.linalg.norm(x) / e0) ** 0.1
    # measured: 0.46 with full coarsening, 0.24 with the rule
    assert rho["strong"] < 0.3 and rho["strong"] < 0.6 * rho["full"], rho


def test_tpms_cell_charge_balance():
    """The voxelised interpenetrating gyroid (the paper's Case IV): the
    electrodes never share a node, and a converged step balances charge."""
    from p4d_inputs import make_tpms_cell
    case = make_tpms_cell(8, 8, 6, state="initial")
    d, st0 = _disc(case)
    st1, hist = time_step(d, st0, rtol=1e-13)
    p = d.p
    phis_l = np.where(d.act, st1["phis"], 0.0)
    i_n, *_ = d.kinetics(phis_l, st1["phie"], st1["ce"], st1["cs"][:, -1])
    I = p["i_app"] * d.gpw.sum()
    an = d.etype == 0
    assert np.sum(d.A[~an] * i_n[~an]) == pytest.approx(I, rel=1e-8)
    assert np.sum(d.A[an] * i_n[an]) == pytest.approx(-I, rel=1e-8)


@pytest.mark.parametrize("cell", ["cube8", "tpms"])
def test_masked_galerkin_operator_rank(cell):
    """The phi_s multigrid of one electrode (masked to its unknowns): the
    Galerkin operator P^T A P of the symmetric positive definite fine block
    is symmetric positive semidefinite, and definite exactly when the
    masked prolongation has full column rank.  On the layered cube it has;
    on the voxelised gyroid the anode's grounded nodes leave coarse columns
    that reach the anode only where it is one element thick, the columns
    become dependent and the coarse operator singular."""
    from p4d_inputs import make_tpms_cell
    from oracle.blocks import BlockPrecond
    case = make_case("cube8") if cell == "cube8" else make_tpms_cell(8, 8, 6)
    d, st = _disc(case)
    A = BlockPrecond(d, d.jacobian(st), coarse_max=16).blocks[0][0]
    node_elec = np.full(d.nn, -1)
    node_elec[d.enodes] = d.etype
    mask = d.act & (node_elec == 0)
    Af = A[mask][:, mask].toarray()
    assert np.abs(Af - Af.T).max() <= 1e-12 * np.abs(Af).max()
    assert np.linalg.eigvalsh(Af).min() > 0
    mg = GMG(A, (d.nnx, d.nny, d.nnz), mask=mask, coarse_max=16, lengths=d.lengths)
    P = mg.P[0].tocsc()
    cols = np.flatnonzero(np.asarray(abs(P).sum(axis=0)).ravel() > 0)
    Ac = mg.A[1][cols][:, cols].toarray()
    ev = np.linalg.eigvalsh(0.5 * (Ac + Ac.T))
    assert np.abs(Ac - Ac.T).max() <= 1e-12 * np.abs(Ac).max()
    assert ev.min() >= -1e-12 * ev.max()
    full_rank = np.linalg.matrix_rank(P[:, cols].toarray()[mask]) == len(cols)
    assert full_rank == (cell == "cube8")
    assert (ev.min() > 1e-10 * ev.max()) == full_rank, (ev.min() / ev.max(), full_rank)
