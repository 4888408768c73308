"""Slab partition of a cell along z for domain decomposition (index
bookkeeping only: the slabs' meshes, parameters and states are slices of the
cell's arrays).

The node planes 0..nz are split into ``nparts`` contiguous owned ranges
``[p_r, p_{r+1})`` of nearly equal size.  With ``g`` ghost planes per
interior side, slab r is built from the elements
``[max(p_r - g, 0), min(p_{r+1} - 1 + g, nz))``, so its node planes run from
``max(p_r - g, 0)`` to ``min(p_{r+1} - 1 + g, nz)``.  The lowest ``g`` of
them are ghost planes (owned by slab r - 1) for every slab but the first,
the highest ``g`` (owned by slab r + 1) for every slab but the last.  Gamma_n, the grounded z = 0 face, and its
foil belong to the first slab; Gamma_p, the z = Lz face carrying the
applied current, and its foil to the last.
"""
import numpy as np

_ELEM_KEYS = ("region", "eps", "eps_s", "sigma_e", "Ds_e")
_NODE_KEYS = ("Rs", "Ds")
_STATE_NODE = ("phis", "phie", "ce", "ce_prev")
_STATE_CS = ("cs_node", "cs_prev_node")


def owned_plane_bounds(nz, nparts):
    """[p_0 = 0, p_1, ..., p_P = nz + 1]: slab r owns node planes [p_r, p_{r+1})."""
    if not 1 <= nparts <= nz:
        raise ValueError("need 1 <= nparts <= nz")
    return [round(r * (nz + 1) / nparts) for r in range(nparts + 1)]


def slab_cases(case, nparts, ghosts=1):
    """The cell ``case`` cut into ``nparts`` z slabs with ``ghosts`` ghost
    planes per interior side.  Returns a list of dicts, bottom to top:
    ``case`` (mesh, params and state of the slab, same keys as the cell's),
    ``e_lo`` (first element layer = first node plane of the slab in the
    cell), ``own`` (owned local node planes [lo, hi)), ``nplanes`` and
    ``ghosts``."""
    m = case["mesh"]
    nx, ny, nz = int(m["nx"]), int(m["ny"]), int(m["nz"])
    nxy_e, nxy_n = nx * ny, (nx + 1) * (ny + 1)
    bounds = owned_plane_bounds(nz, nparts)
    if ghosts < 1 or (nparts > 1 and min(b1 - b0 for b0, b1 in zip(bounds, bounds[1:])) < ghosts):
        raise ValueError("every slab must own at least `ghosts` >= 1 node planes")
    out = []
    for r in range(nparts):
        e_lo, e_hi = max(bounds[r] - ghosts, 0), min(bounds[r + 1] - 1 + ghosts, nz)
        sm = dict(m)
        sm["nz"] = e_hi - e_lo
        sm["hz"] = np.asarray(m["hz"], float)[e_lo:e_hi].copy()
        for k in _ELEM_KEYS:
            if m.get(k) is not None:
                sm[k] = np.asarray(m[k])[e_lo * nxy_e:e_hi * nxy_e].copy()
        for k in _NODE_KEYS:
            sm[k] = np.asarray(m[k])[e_lo * nxy_n:(e_hi + 1) * nxy_n].copy()
        zero = np.zeros(nxy_e, np.uint8)
        sm["gamma_n"] = np.asarray(m["gamma_n"], np.uint8).copy() if r == 0 else zero
        sm["gamma_p"] = np.asarray(m["gamma_p"], np.uint8).copy() if r == nparts - 1 else zero.copy()
        if r > 0:
            sm["shell_sigma_t_n"] = 0.0
        if r < nparts - 1:
            sm["shell_sigma_t_p"] = 0.0
        st = case["state"]
        sst = {k: np.asarray(st[k])[e_lo * nxy_n:(e_hi + 1) * nxy_n].copy() for k in _STATE_NODE + _STATE_CS}
        nplanes = e_hi - e_lo + 1
        own = (bounds[r] - e_lo, bounds[r + 1] - e_lo)
        out.append(dict(case=dict(mesh=sm, params=dict(case["params"]), state=sst), e_lo=e_lo, own=own,
                        nplanes=nplanes, ghosts=ghosts))
    return out


def slab_node_rows(slab, nxy):
    """Cell node indices of the slab's owned nodes, and their local indices."""
    lo, hi = slab["own"]
    loc = np.arange(lo * nxy, hi * nxy)
    return loc + slab["e_lo"] * nxy, loc
