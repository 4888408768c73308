"""Slab domain decomposition on the GPU (p4d_dd_*): the cell cut into z
slabs, one handle per slab on one stream, ghost planes exchanged before
every operator application and every inner product reduced over the slabs.

* The decomposed JVP is the cell's JVP on every owned row.
* The decomposed FGMRES (restricted additive Schwarz over the slabs, with
  or without the two-level coarse correction) converges to the cell's
  solution: the oracle's direct solve, within the bounds of the single-cell
  parity tests.
* The coarse space and a wider overlap cut the iteration count.
* One slab is the single-cell solve."""
import numpy as np
import pytest
import torch

from oracle.fe import Disc
from oracle.krylov import LinearSolve, per_field_error
from p4d_inputs import make_box_case, make_case, make_slab_case, make_tpms_cell, slab_cases, slab_node_rows

pytestmark = pytest.mark.gpu

CELLS = {
    "cube8": lambda: make_case("cube8"),
    "hetero": lambda: make_box_case(8, 8, (6, 4, 6), 60e-6, (60e-6, 25e-6, 60e-6), 6, 1234, hetero=True, rs_cv=0.3),
    "tabshell": lambda: make_slab_case(nx=12, ny=3, layers=(3, 2, 3), nc=5, seed=55, tab=3, crate=1.0, h_lat=8e-6,
                                       shell=(40.0, 60.0), state="seeded"),
    "tpms": lambda: make_tpms_cell(16, 16, 8),
    "paper_laws": lambda: make_case("cube8"),
}
LAWS = {"paper_laws": (dict(material="paper", ocp="paper"), dict(ocp_model=1, transport_model=1))}


def _maps(case, slabs, parts, d):
    """Per slab: (slab rows, cell rows) of its owned rows, and the cell row of
    every slab row."""
    m = case["mesh"]
    nxy = (m["nx"] + 1) * (m["ny"] + 1)
    out = []
    for sl, p in zip(slabs, parts):
        off = sl["e_lo"] * nxy
        glob, loc = slab_node_rows(sl, nxy)
        nns, nc = p.nn, p.nc
        en = np.asarray(p.enodes, np.int64)
        own_e = np.flatnonzero(np.isin(en, loc))
        ecell = d.eidx[en + off]
        assert (ecell >= 0).all()
        rs = [f * nns + loc for f in range(3)] + [3 * nns + own_e * nc + i for i in range(nc)]
        rc = [f * d.nn + glob for f in range(3)] + [3 * d.nn + ecell[own_e] * nc + i for i in range(nc)]
        full = np.concatenate([f * d.nn + off + np.arange(nns) for f in range(3)] +
                              [3 * d.nn + ecell * nc + i for i in range(nc)])
        order = np.concatenate([f * nns + np.arange(nns) for f in range(3)] +
                               [3 * nns + np.arange(p.NE) * nc + i for i in range(nc)])
        out.append((np.concatenate(rs), np.concatenate(rc), order, full))
    return out


def _gather(maps, ys, ndof):
    out = np.full(ndof, np.nan)
    for (rs, rc, _, _), y in zip(maps, ys):
        out[rc] = y.cpu().numpy()[rs]
    assert not np.isnan(out).any()
    return out


def _scatter(maps, g, parts):
    xs = []
    for (_, _, order, full), p in zip(maps, parts):
        v = np.zeros(p.ndof)
        v[order] = g[full]
        xs.append(torch.tensor(v, device="cuda"))
    return xs


def _setup(name, nparts, coarse=2, ghosts=1, **opts):
    from paper_2602_07225_gb300 import P4DSolver, SlabSolver
    case = CELLS[name]()
    okw, lkw = LAWS.get(name, ({}, {}))
    d = Disc(case["mesh"], case["params"], **okw)
    slabs = slab_cases(case, nparts, ghosts)
    dd = SlabSolver(slabs, coarse=coarse, **lkw, **opts)
    maps = _maps(case, slabs, dd.parts, d)
    cell = P4DSolver(case, **lkw, **opts)
    return case, d, slabs, dd, maps, cell


@pytest.mark.parametrize("name,nparts,ghosts", [("cube8", 2, 1), ("cube8", 3, 1), ("cube8", 3, 3), ("hetero", 2, 1),
                                                ("tabshell", 2, 1), ("tpms", 2, 2), ("paper_laws", 2, 1),
                                                ("paper_laws", 4, 2)])
def test_dd_jvp_is_the_cells(name, nparts, ghosts):
    case, d, slabs, dd, maps, cell = _setup(name, nparts, ghosts=ghosts, precision=0)
    sts = dd.state_tensors()
    dd.jacobian_update(sts)
    stc = cell.state_tensors(case["state"])
    cell.jacobian_update(stc)
    g = np.random.default_rng(11).standard_normal(d.ndof)
    ys = dd.jvp(_scatter(maps, g, dd.parts))
    y = _gather(maps, ys, d.ndof)
    yc = cell.jvp(torch.tensor(g, device="cuda")).cpu().numpy()
    for sl in d.field_slices():
        assert np.abs(y[sl] - yc[sl]).max() <= 1e-14 * max(np.abs(yc[sl]).max(), 1e-300)
    # the owned rows of the slab residuals are the cell's residual
    r = _gather(maps, dd.residual(sts), d.ndof)
    rc = cell.residual(stc).cpu().numpy()
    assert np.abs(r - rc).max() <= 1e-14 * np.abs(rc).max()


@pytest.mark.parametrize("name,nparts,ghosts", [("cube8", 2, 1), ("cube8", 3, 1), ("cube8", 3, 2), ("hetero", 2, 1),
                                                ("tpms", 2, 2), ("paper_laws", 2, 1)])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("coarse", [0, 2])
def test_dd_fgmres_matches_direct(name, nparts, ghosts, precision, refine, coarse):
    rtol = 1e-12 if precision == 0 else 1e-10
    case, d, slabs, dd, maps, cell = _setup(name, nparts, ghosts=ghosts, precision=precision, mode=1, rtol=rtol,
                                            maxit=1500, cgs_refine=refine, coarse=coarse)
    sts = dd.state_tensors()
    dd.jacobian_update(sts)
    bs = [-r for r in dd.residual(sts)]
    xs, info = dd.solve(bs)
    x = _gather(maps, xs, d.ndof)
    ref = d.state_from_case(case["state"])
    x_ref = LinearSolve(d, ref).direct()
    err = per_field_error(d, x, x_ref)[0]
    assert info["status"] == 0, info
    assert info["rel_res"] <= 2 * rtol, info
    assert err <= (1e-9 if precision == 0 else 1e-7), (err, info)
    if refine == 0:
        assert info["reorth"] == 0


def test_coarse_space_cuts_iterations():
    # the slab preconditioners leave the long-range potential modes to
    # FGMRES; the coarse space (constants and linear-in-z functions per slab
    # and block) carries them
    from paper_2602_07225_gb300 import SlabSolver
    case = make_box_case(16, 16, (20, 8, 20), 100e-6, (100e-6, 25e-6, 100e-6), 6, 1007)
    its = {}
    for coarse in (0, 1, 2):
        dd = SlabSolver(slab_cases(case, 4, 2), coarse=coarse, precision=1, mode=1, rtol=1e-8, maxit=1500)
        sts = dd.state_tensors()
        dd.jacobian_update(sts)
        _, info = dd.solve([-r for r in dd.residual(sts)])
        assert info["status"] == 0, info
        its[coarse] = info["iters"]
        dd.close()
    assert its[2] < its[0], its


@pytest.mark.parametrize("name", ["cube8", "paper_laws"])
def test_one_slab_is_the_cell_solve(name):
    rtol = 1e-10
    case, d, slabs, dd, maps, cell = _setup(name, 1, precision=0, mode=1, rtol=rtol, maxit=600)
    sts = dd.state_tensors()
    dd.jacobian_update(sts)
    xs, info = dd.solve([-r for r in dd.residual(sts)])
    stc = cell.state_tensors(case["state"])
    cell.jacobian_update(stc)
    x1, info1 = cell.solve(-cell.residual(stc))
    assert info["iters"] == info1["iters"], (info, info1)
    a, b = xs[0].cpu().numpy(), x1.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_wider_overlap_cuts_iterations():
    from paper_2602_07225_gb300 import SlabSolver
    case = make_box_case(16, 16, (20, 8, 20), 100e-6, (100e-6, 25e-6, 100e-6), 6, 1007)
    its = {}
    for ghosts in (2, 4):
        dd = SlabSolver(slab_cases(case, 4, ghosts), coarse=2, precision=1, mode=1, rtol=1e-8, maxit=1500)
        sts = dd.state_tensors()
        dd.jacobian_update(sts)
        _, info = dd.solve([-r for r in dd.residual(sts)])
        assert info["status"] == 0, info
        its[ghosts] = info["iters"]
        dd.close()
    assert its[4] < its[2], its


def test_dd_rejects_mismatched_slabs():
    from paper_2602_07225_gb300 import P4DSolver, _native as N
    import ctypes as C
    a = P4DSolver(make_case("cube8"))
    b = P4DSolver(CELLS["tabshell"]())                     # another nx, ny
    lib = a.lib
    out = C.c_void_p()
    hs = (C.c_void_p * 2)(a.h.value, b.h.value)
    assert lib.p4d_dd_create(hs, 2, 1, C.byref(out)) == N.INVALID_ARG
    hs = (C.c_void_p * 2)(a.h.value, a.h.value)
    assert lib.p4d_dd_create(hs, 2, 1, C.byref(out)) == N.INVALID_ARG
