"""Slab domain decomposition on the host.

The decomposed solve rests on one fact: the rows a slab owns, assembled on
the slab's own sub-mesh (its elements plus the element layers of its ghost
planes), are the cell's rows.  The oracle checks that here for the
residual and the Jacobian of several cells (section 4 eqs.), so that a
wrong slice (an element layer too few, Gamma_n or Gamma_p on the wrong
slab, a shifted node plane) fails.  The library's halo plan is checked
against the partition, and its messages are exchanged between two gloo
ranks on the CPU the way the slabs exchange ghost planes."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from oracle.fe import Disc
from p4d_inputs import make_box_case, make_case, make_slab_case, slab_cases, slab_node_rows, owned_plane_bounds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CELLS = {
    "cube8": lambda: make_case("cube8"),
    "hetero": lambda: make_box_case(8, 8, (6, 4, 6), 60e-6, (60e-6, 25e-6, 60e-6), 6, 1234, hetero=True, rs_cv=0.3),
    "tabshell": lambda: make_slab_case(nx=12, ny=3, layers=(3, 2, 3), nc=5, seed=55, tab=3, crate=1.0, h_lat=8e-6,
                                       shell=(40.0, 60.0), state="seeded"),
}


def _row_maps(d_cell, d_slab, slab, nxy):
    """Cell rows of the slab's owned rows (all four fields) and the cell
    column of every slab column."""
    glob, loc = slab_node_rows(slab, nxy)
    off = slab["e_lo"] * nxy
    nn_c, nn_s, nc = d_cell.nn, d_slab.nn, d_cell.nc
    rows_s, rows_c = [], []
    for f in range(3):
        rows_s.append(f * nn_s + loc)
        rows_c.append(f * nn_c + glob)
    own_e = np.flatnonzero(np.isin(d_slab.enodes, loc))
    ecell = d_cell.eidx[d_slab.enodes[own_e] + off]
    assert (ecell >= 0).all()
    for i in range(nc):
        rows_s.append(3 * nn_s + own_e * nc + i)
        rows_c.append(3 * nn_c + ecell * nc + i)
    colmap = np.empty(d_slab.ndof, np.int64)
    for f in range(3):
        colmap[f * nn_s:(f + 1) * nn_s] = f * nn_c + np.arange(nn_s) + off
    ec_all = d_cell.eidx[d_slab.enodes + off]
    assert (ec_all >= 0).all()      # a slab's electrode node is one of the cell's
    for i in range(nc):
        colmap[3 * nn_s + np.arange(d_slab.NE) * nc + i] = 3 * nn_c + ec_all * nc + i
    return np.concatenate(rows_s), np.concatenate(rows_c), colmap


@pytest.mark.parametrize("name", list(CELLS))
@pytest.mark.parametrize("nparts,ghosts", [(2, 1), (3, 1), (2, 2)])
@pytest.mark.parametrize("material", [None, "paper"])
def test_owned_rows_of_a_slab_are_the_cells(name, nparts, ghosts, material):
    case = CELLS[name]()
    kw = dict(material="paper", ocp="paper") if material else {}
    d = Disc(case["mesh"], case["params"], **kw)
    st = d.state_from_case(case["state"])
    R = d.residual(st)
    J = d.jacobian(st).tocsr()
    m = case["mesh"]
    nxy = (m["nx"] + 1) * (m["ny"] + 1)
    slabs = slab_cases(case, nparts, ghosts)
    covered = np.zeros(d.ndof, int)
    for sl in slabs:
        ds = Disc(sl["case"]["mesh"], sl["case"]["params"], **kw)
        ss = ds.state_from_case(sl["case"]["state"])
        rs, rc, colmap = _row_maps(d, ds, sl, nxy)
        covered[rc] += 1
        Rs = ds.residual(ss)
        scale = np.abs(R).max()
        assert np.abs(Rs[rs] - R[rc]).max() <= 1e-13 * scale
        Js = ds.jacobian(ss).tocsr()[rs].tocoo()
        A = np.zeros((len(rs), d.ndof))
        np.add.at(A, (Js.row, colmap[Js.col]), Js.data)
        B = J[rc].toarray()
        assert np.abs(A - B).max() <= 1e-12 * np.abs(B).max()
    assert (covered == 1).all()     # every row of the cell owned by exactly one slab


@pytest.mark.parametrize("nz,nparts", [(24, 2), (24, 3), (8, 8), (5, 2), (97, 4)])
def test_slabs_partition_the_node_planes(nz, nparts):
    b = owned_plane_bounds(nz, nparts)
    assert b[0] == 0 and b[-1] == nz + 1 and all(b[r + 1] > b[r] for r in range(nparts))


@pytest.mark.parametrize("ghosts", [1, 2, 3])
def test_plan_matches_partition(ghosts):
    from paper_2602_07225_gb300 import halo_plan
    case = make_case("cube8")
    for nparts in (1, 2, 3, 5):
        slabs = slab_cases(case, nparts, ghosts)
        plan = halo_plan([s["nplanes"] for s in slabs], ghosts)
        assert len(plan) == 2 * (nparts - 1)
        got = set()
        for src, sp, dst, dp in plan:
            for t in range(ghosts):
                lo, hi = slabs[src]["own"]
                assert lo <= sp + t < hi                                      # an owned plane ...
                assert not slabs[dst]["own"][0] <= dp + t < slabs[dst]["own"][1]  # ... into a ghost plane
                assert slabs[src]["e_lo"] + sp + t == slabs[dst]["e_lo"] + dp + t  # of the same cell plane
                got.add((dst, dp + t))
        want = {(r, p) for r, s in enumerate(slabs) for p in range(s["nplanes"])
                if not s["own"][0] <= p < s["own"][1]}
        assert got == want
        for r, s in enumerate(slabs):                       # the library's ownership rule
            assert s["own"] == (ghosts if r > 0 else 0, s["nplanes"] - (ghosts if r < nparts - 1 else 0))


def test_plan_rejects_slabs_without_owned_planes():
    from paper_2602_07225_gb300 import halo_plan
    with pytest.raises(ValueError):
        halo_plan([1, 3])
    with pytest.raises(ValueError):
        halo_plan([3, 2, 3])
    with pytest.raises(ValueError):
        halo_plan([5, 5], ghosts=4)        # one owned plane each, fewer than the neighbour's ghosts
    with pytest.raises(ValueError):
        halo_plan([5, 5], ghosts=0)
    with pytest.raises(ValueError):
        slab_cases(make_case("cube8"), 8, ghosts=4)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q, ghosts):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    from paper_2602_07225_gb300 import halo_plan
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = make_case("cube8")
        m = case["mesh"]
        nxy = (m["nx"] + 1) * (m["ny"] + 1)
        nn = nxy * (m["nz"] + 1)
        rng = np.random.default_rng(5)
        g = rng.standard_normal(3 * nn)                     # a cell vector (fields 0..2)
        slabs = slab_cases(case, world, ghosts)
        me = slabs[rank]
        nns = me["nplanes"] * nxy
        off = me["e_lo"] * nxy
        x = np.zeros(3 * nns)
        glob, loc = slab_node_rows(me, nxy)
        for f in range(3):
            x[f * nns + loc] = g[f * nn + glob]             # owned rows only
        plan = halo_plan([s["nplanes"] for s in slabs], ghosts)
        ln = ghosts * nxy                                   # `ghosts` consecutive planes per message
        reqs = []
        for src, sp, dst, dp in plan:                       # pack and send
            if src == rank:
                buf = torch.tensor(np.concatenate([x[f * nns + sp * nxy:f * nns + sp * nxy + ln] for f in range(3)]))
                reqs.append(dist.isend(buf, dst))
        for src, sp, dst, dp in plan:                       # receive and unpack
            if dst == rank:
                buf = torch.empty(3 * ln, dtype=torch.float64)
                dist.recv(buf, src)
                for f in range(3):
                    x[f * nns + dp * nxy:f * nns + dp * nxy + ln] = buf[f * ln:(f + 1) * ln].numpy()
        for r in reqs:
            r.wait()
        want = np.concatenate([g[f * nn + off:f * nn + off + nns] for f in range(3)])
        halo_ok = bool(np.array_equal(x, want))             # every plane of the slab, ghosts included
        part = torch.tensor([float(np.dot(x[f * nns + loc], x[f * nns + loc])) for f in range(3)], dtype=torch.float64)
        dist.all_reduce(part)                               # owned-row partial sums
        full = [float(np.dot(g[f * nn:(f + 1) * nn], g[f * nn:(f + 1) * nn])) for f in range(3)]
        q.put((rank, halo_ok, part.tolist(), full))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ghosts", [1, 2])
def test_two_ranks_exchange_ghost_planes_and_reduce(ghosts):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, ghosts)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, halo_ok, part, full in out:
        assert halo_ok
        assert np.allclose(part, full, rtol=1e-13, atol=0)
