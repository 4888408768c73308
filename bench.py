"""Benchmark: Newton linear solves/s and FGMRES iterations/s to a 1e-8
relative residual on the 128x128x96 homogeneous cube (40/16/40 elements,
N_c = 20, ~32M unknowns), mixed precision (FP32 multigrid/particle
preconditioner inside FP64 FGMRES) vs the all-FP64 GPU path.

The workload is a 1C constant-current discharge from rest (theta_n = 0.8,
theta_p = 0.6, c_e = 1000 mol/m^3, open-circuit potentials): one step = one
backward-Euler time step of 10 s, solved by Newton's method (scaled residual
reduced by 1e-8) whose linear systems are solved by block-preconditioned
FGMRES to 1e-8.  `--steps K` times K consecutive time steps from rest (the
default K = 20 is the whole 200 s transient); the warm-up steps run the
same transient from rest beforehand.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
Under torchrun (N > 1) every rank solves its own cell (independent problems,
weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton linear solves/s & FGMRES iters/s to 1e-8 rel. residual; mixed vs FP64"
WORKLOAD = "cube128"
# unknowns of cube128: 3 fields on 129*129*97 nodes + N_c = 20 radial nodes on
# the 82 electrode node layers (41 anode + 41 cathode)
# DRAM bytes per row of one level-0 Chebyshev step (k_mf_level0, all four
# hierarchies), from an ncu capture of that launch on cube128 itself
# (dram__bytes_read.sum + dram__bytes_write.sum = 110.79 + 16.98 MB for
# 4,576,275 rows; a one-pass metric set, so the full-size capture is safe)
TRAFFIC_PER_ROW = (110.79e6 + 16.98e6) / 4576275
TRAFFIC_SOURCE = ("ncu dram__bytes_read+write of one level-0 k_mf_level0 launch on cube128 (1.16 x the "
                  "24 B/row algorithmic bytes), per row x rows")
FP64_TFLOPS = 1.25    # GB300 nominal non-tensor FP64
CHEB = (2, 10.0)      # Chebyshev degree (V(d,d) cycles) and eigenvalue ratio, both arms
# FGMRES rtol of the precision study's second set: the scaled residual's
# error amplification on hetero128 is ~17 (1.72e-7 at 1e-8), so 3e-9 keeps
# the solution error within 1e-7
PRECISION_RTOL = 3e-9
CYCLE = "V(%d,%d) Chebyshev (eigenvalue ratio %g), coarsening along the strongly coupled axes" % (
    CHEB[0], CHEB[0], CHEB[1])
WORKLOAD_DESC = {"cube128": "cube128: Q1 hex 128x128x96 (anode/sep/cathode 40/16/40), N_c=20",
                 "cube96": "cube96 (profiling case): Q1 hex 96x96x72 (anode/sep/cathode 30/12/30), N_c=20",
                 "tpms128": "tpms128: the paper's interpenetrating gyroid electrodes (Case IV) voxelised on "
                            "128x128x64 hex elements of a 1 x 1 x 0.5 mm box, N_c=6"}
CUBE128_DOF = 3 * 129 * 129 * 97 + 20 * 82 * 129 * 129


COMBINE_DESC = {"bj": "block Jacobi", "bgs": "block Gauss-Seidel in the order phi_e, phi_s, c_e"}
CGS_DESC = {0: "classical Gram-Schmidt without refinement", 1: "classical Gram-Schmidt, second pass when needed",
            2: "classical Gram-Schmidt twice"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--laws", default="linear", choices=["linear", "paper"],
                    help="material laws: linear OCP and constant transport (the workload definition), or the "
                         "paper's OCP curves and kappa(c_e), D_e(c_e)")
    ap.add_argument("--stepwise", action="store_true",
                    help="launch every solve kernel by kernel instead of through CUDA graphs (the same work; for "
                         "profilers that cannot see kernels inside conditional graph nodes)")
    ap.add_argument("--combine", default="bj", choices=["bj", "bgs"],
                    help="block Jacobi, or block Gauss-Seidel in the paper's order (phi_e, phi_s, c_e; c_s eliminated)")
    ap.add_argument("--cgs-refine", type=int, default=0, choices=[0, 1, 2],
                    help="second Gram-Schmidt pass: 0 never (the paper's GMRES setting), 1 when needed, 2 always")
    ap.add_argument("--slab-nx", type=int, default=2048, help="slab2048: elements along the long axis")
    ap.add_argument("--slab-steps", type=int, default=30, help="slab2048: backward-Euler steps")
    ap.add_argument("--slab-fd", type=int, default=6, help="slab2048: directional finite-difference checks")
    ap.add_argument("--slab-geometry", default="cube", choices=["cube", "paper"],
                    help="slab2048: the cube's element scale without collector foils, or the paper's jelly roll "
                         "(1 m x 5 cm, 50/20/50 um layers) with aluminium and copper foils as collector shells")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nme, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# generator seeds of the named workloads; rank r > 0 of a multi-GPU run
# solves its own cell of the same shape, seeded SEEDS[name] + 7919 r
SEEDS = {"cube8": 1001, "cube128": 1002, "cube96": 1002, "hetero128": 1003, "tpms128": 1006}


def make_workload(name, rank=0, **kw):
    from p4d_inputs import make_case, make_tpms_cell
    if name == "tpms128":
        return make_tpms_cell(128, 128, 64, seed=SEEDS[name] + 7919 * rank, **kw)
    if rank == 0:
        return make_case(name, **kw)
    return make_case(name, seed=SEEDS[name] + 7919 * rank, **kw)


def shard(n, rank, world):
    """Units of this rank: round-robin over the ranks, every unit once."""
    return list(range(rank, n, world))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(ms, iters, world, device=None):
    """(max over ranks of the timed milliseconds, sum of their iterations).
    The ranks' units are independent, so this timing reduction is the only
    exchange between them."""
    if world == 1:
        return ms, iters
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters)], device=device, dtype=torch.float64)
    dist.all_reduce(it)
    return t.item(), it.item()


NEWTON_RTOL = 1e-8    # scaled nonlinear residual reduction per backward-Euler step
NEWTON_MAXIT = 20
STEP_FIELDS = ("phis", "phie", "ce", "cs")


def be_step(solver, st):
    """One backward-Euler step in place on st: the current concentrations
    become the previous time level, then Newton.  Returns (Newton iterations,
    info of the step: last linear solve, plus nsolves / iters_total)."""
    st["ce_prev"].copy_(st["ce"])
    st["cs_prev"].copy_(st["cs"])
    it, info = solver.newton(st, rtol=NEWTON_RTOL, maxit=NEWTON_MAXIT)
    return it, info


def run_transient(solver, st0, work, nsteps):
    """nsteps backward-Euler steps from st0 (copied into work first)."""
    for k in st0:
        work[k].copy_(st0[k])
    tot = {"solves": 0, "iters": 0, "newton": 0, "rel_res": 0.0, "rel_res_unscaled": 0.0,
           "rel_res_block_unscaled": [0.0] * 4, "reorth": 0}
    for _ in range(nsteps):
        it, info = be_step(solver, work)
        tot["solves"] += info["nsolves"]
        tot["iters"] += info["iters_total"]
        tot["newton"] += it
        tot["reorth"] += info["reorth"]
        tot["rel_res"] = max(tot["rel_res"], info["rel_res"])
        tot["rel_res_unscaled"] = max(tot["rel_res_unscaled"], info["rel_res_unscaled"])
        tot["rel_res_block_unscaled"] = [max(a, b) for a, b in zip(tot["rel_res_block_unscaled"],
                                                                   info["rel_res_block_unscaled"])]
    return tot


def gpu_leg(args, rank, world, local):
    import torch
    from paper_2602_07225_gb300 import P4DSolver
    from paper_2602_07225_gb300 import build as pbuild

    pbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = make_workload(args.workload, rank, state="initial")
    opts = dict(mode=1, combine=0 if args.combine == "bj" else 1, order=(1, 0, 2), rtol=1e-8, restart=30, maxit=600,
                cheb_degree=CHEB[0], cheb_ratio=CHEB[1], cgs_refine=args.cgs_refine, profile=int(args.stepwise))
    if args.laws == "paper":
        opts.update(ocp_model=1, transport_model=1)
    s = P4DSolver(case, device=dev, precision=1, **opts)
    st0 = s.state_tensors(case["state"])
    work = {k: v.clone() for k, v in st0.items()}
    ndof = s.ndof
    lib = s.lib

    run_transient(s, st0, work, args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in st0:
        work[k].copy_(st0[k])
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        l0 = lib.p4d_launch_count()
        e0.record(stream)
        tot = {"solves": 0, "iters": 0, "newton": 0, "rel_res": 0.0, "rel_res_unscaled": 0.0,
               "rel_res_block_unscaled": [0.0] * 4, "reorth": 0}
        for _ in range(args.steps):
            it, info = be_step(s, work)
            tot["solves"] += info["nsolves"]
            tot["iters"] += info["iters_total"]
            tot["newton"] += it
            tot["reorth"] += info["reorth"]
            tot["rel_res"] = max(tot["rel_res"], info["rel_res"])
            tot["rel_res_unscaled"] = max(tot["rel_res_unscaled"], info["rel_res_unscaled"])
            tot["rel_res_block_unscaled"] = [max(a, b) for a, b in zip(tot["rel_res_block_unscaled"],
                                                                       info["rel_res_block_unscaled"])]
        e1.record(stream)
        torch.cuda.synchronize()
        launches = lib.p4d_launch_count() - l0
        barrier(world)
    ms_all = e0.elapsed_time(e1)
    ms, solves_all = aggregate(ms_all, tot["solves"], world, dev)
    _, iters_all = aggregate(0.0, tot["iters"], world, dev)
    final = {k: work[k].clone() for k in STEP_FIELDS}

    # ---- end-to-end through the C ABI with the state in pinned host memory:
    # every step copies the state to the device and the new state back
    host = {k: st0[k].cpu().pin_memory() for k in STEP_FIELDS}
    host0 = {k: v.clone() for k, v in host.items()}
    dbuf = {k: torch.empty_like(v) for k, v in st0.items()}
    h2d = sum(host[k].numel() * 8 for k in STEP_FIELDS)
    d2h = h2d

    def e2e_step():
        for k in STEP_FIELDS:
            dbuf[k].copy_(host[k], non_blocking=True)
        be_step(s, dbuf)
        for k in STEP_FIELDS:
            host[k].copy_(dbuf[k], non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    for k in STEP_FIELDS:
        host[k].copy_(host0[k])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    # ---- roofline: one profiled Newton linear solve at the final state
    roof = roofline_smooth(s, work, case)
    fp64_rate = measure_fp64(s)

    # ---- FP64 GPU path of the same transient
    fp64 = None
    if not args.no_fp64:
        s64 = P4DSolver(case, device=dev, precision=0, **opts)
        w64 = {k: v.clone() for k, v in st0.items()}
        run_transient(s64, st0, w64, 1)
        torch.cuda.synchronize()
        e0.record(stream)
        t64 = run_transient(s64, st0, w64, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        dev64 = max(float(((w64[k] - final[k]).norm() / final[k].norm()).item()) for k in STEP_FIELDS)
        fp64 = {"solves_per_s": t64["solves"] / (ms64 / 1e3), "fgmres_iters_per_s": t64["iters"] / (ms64 / 1e3),
                "linear_solves": t64["solves"], "fgmres_iters": t64["iters"], "newton_iters": t64["newton"],
                "ms_per_step": ms64 / args.steps, "rel_res_max": t64["rel_res"],
                "final_state_rel_diff_vs_mixed": dev64}
        s64.close()
    return dict(ms_per_step=ms / args.steps, solves_per_s=solves_all / (ms / 1e3),
                iters_per_s=iters_all / (ms / 1e3), tot=tot, ndof=ndof, e2e_ms=e2e_ms, h2d=h2d, d2h=d2h,
                clocks=clk.summary(), roof=roof, fp64=fp64, launches=launches, nn=s.nn, NE=s.NE, nc=s.nc,
                fp64_rate=fp64_rate)


def measure_fp64(s):
    """Measured FP64 FMA rate of this GPU (TFLOP/s, p4d_fp64_fma_rate)."""
    import ctypes as C
    v = C.c_double(0.0)
    st = s.lib.p4d_fp64_fma_rate(C.byref(v))
    return v.value if st == 0 else None


# Algorithmic bytes of one level-0 Chebyshev step per node and field: the
# method's minimum for a matrix-free fine-level smoothing step (read x, b,
# 1/diag and d, write d and x_out: 6 x 4 B of FP32 vectors).
ALG_BYTES_SMOOTH0 = 24
# Bytes the matrix-free level-0 step reads and writes per node and field:
# x, b, 1/diag, d and the variable diagonal in, d and x_out out (7 x 4 B),
# the element coefficients (~4 B per node; 8 for c_e) and the phi_s label
# byte, ~33 B; ncu measures ~25 B of DRAM traffic per row on cube128 (part of
# the x tiles' halo and the coefficients come from L2).
KERNEL_BYTES_SMOOTH0 = 33


def n_grounded(m):
    """Nodes of the grounded faces (z = 0 faces flagged in gamma_n): they are
    anode electrode nodes without a phi_s unknown."""
    import numpy as np
    nx, ny = int(m["nx"]), int(m["ny"])
    g = np.asarray(m["gamma_n"]).reshape(ny, nx).astype(bool)
    nodes = np.zeros((ny + 1, nx + 1), bool)
    for dj in (0, 1):
        for di in (0, 1):
            nodes[dj:dj + ny, di:di + nx] |= g
    return int(nodes.sum())


def roofline_smooth(s, st, case):
    """Level-0 Chebyshev steps that apply the fine-level operator (the
    largest kernel class of a step in the ncu launch list), averaged over
    one profiled Newton linear solve at state st.  Rows per launch: the
    active phi_s nodes plus every phi_e and c_e node.  Also the phases of the
    same solve and its reduced FP64 JVP."""
    b = s.residual(st)
    b.neg_()
    s.jacobian_update(st)
    s.set_options(profile=1)
    _, info = s.solve(b)
    s.set_options(profile=0)
    n_act = s.NE - n_grounded(case["mesh"])
    rows = n_act + 2 * s.nn
    ms = info["ms_smooth0"] / max(1, info["n_smooth0"])
    # reduced FP64 JVP of the same solve (k_jvp_combine + k_jvp_macro): FP64
    # FMAs per launch = 27 per active phi_s node (K_sigma) + 2 x 27 per node
    # (K_kappa, C) + 1 per node (u = x_phie + gamma/c_e x_ce) + 10 per
    # electrode node (Schur coupling)
    fma = 27 * n_act + 55 * s.nn + 10 * s.NE
    jvp_ms = info["ms_jvp"] / max(1, info["n_jvp"])
    return {"kernel": "k_mf_level0: level-0 Chebyshev step, matrix-free (FP32, 4 hierarchies)", "ms": ms,
            "rows": rows,
            "bytes": ALG_BYTES_SMOOTH0 * rows, "kernel_bytes": KERNEL_BYTES_SMOOTH0 * rows,
            "gbs": ALG_BYTES_SMOOTH0 * rows / (ms * 1e-3) / 1e9,
            "kernel_gbs": KERNEL_BYTES_SMOOTH0 * rows / (ms * 1e-3) / 1e9, "launches": info["n_smooth0"],
            "solve": {"iters": info["iters"], "reorth": info["reorth"], "rel_res": info["rel_res"],
                      "rel_res_unscaled": info["rel_res_unscaled"]},
            "phases_ms": {"precond": info["ms_precond"], "jvp": info["ms_jvp"], "ortho": info["ms_ortho"],
                          "total": info["ms_total"]},
            "jvp": {"ms": jvp_ms, "flops": 2 * fma, "tflops": 2 * fma / (jvp_ms * 1e-3) / 1e12,
                    "launches": info["n_jvp"]}}


def roofline_jvp(s, st, dev):
    """Average duration of the FP64 coupled JVP (full layout) over repeated
    launches on the solver's stream, and its algorithmic bytes: the three
    27-point FP64 stencils, x and y over every unknown, the per-node factor
    gamma/c_e and the electrode-node coupling scalars."""
    import torch
    x = torch.randn(s.ndof, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        s.jvp(x, out=y)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        s.jvp(x, out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nn, NE, nc = s.nn, s.NE, s.nc
    bytes_ = 3 * 27 * 8 * nn + 2 * 8 * s.ndof + 8 * nn + (8 * 9) * NE
    return {"kernel": "coupled JVP (k_jvp_macro + k_jvp_particle)", "ms": ms, "bytes": bytes_,
            "gbs": bytes_ / (ms * 1e-3) / 1e9}


def cpu_oracle_leg(full_dof, sample_lat=16, seconds_hint=30.0, combine="bj"):
    """The oracle's plain Newton method with block-preconditioned FGMRES
    linear solves (same V(2,2) cycle, rtol 1e-8) on a bounded sample of the
    workload: the first backward-Euler step from rest of a 16x16 lateral
    column block of the 128x128x96 cube (same z layering, spacings, N_c and
    physics), its Newton linear solves/s scaled to the full workload by the
    number of unknowns."""
    from p4d_inputs import make_box_case
    from oracle.fe import Disc
    from oracle.krylov import time_step
    L = 100e-6 * sample_lat / 128
    case = make_box_case(sample_lat, sample_lat, (40, 16, 40), L, (100e-6, 25e-6, 100e-6), 20, 1002,
                         state="initial")
    d = Disc(case["mesh"], case["params"])
    st = d.state_from_case(case["state"])
    counts = {"solves": 0, "iters": 0}
    import oracle.krylov as ok

    class Counting(ok.LinearSolve):
        def fgmres(self, *a, **kw):
            x, its, hist = super().fgmres(*a, **kw)
            counts["solves"] += 1
            counts["iters"] += its
            return x, its, hist

    t0 = time.perf_counter()
    steps = 0
    saved = ok.LinearSolve
    ok.LinearSolve = Counting
    try:
        while True:
            st, _ = time_step(d, st, rtol=NEWTON_RTOL, linear="fgmres", degree=CHEB[0], ratio=CHEB[1],
                              combine="additive" if combine == "bj" else "multiplicative", order=(1, 0, 2))
            steps += 1
            if time.perf_counter() - t0 > seconds_hint * 0.5 or steps >= 2:
                break
    finally:
        ok.LinearSolve = saved
    dt = time.perf_counter() - t0
    return {"sample_dof": d.ndof, "s_per_solve": dt / max(1, counts["solves"]),
            "iters_per_solve": counts["iters"] / max(1, counts["solves"]), "solves": counts["solves"],
            "steps": steps, "scaled_solves_per_s": counts["solves"] / dt * d.ndof / full_dof}


def batched_leg(args, rank=0, world=1, local=0):
    """64 gyroid cells of uneven sizes (16x16x24 ... 64x64x96 elements,
    N_c 10-20): one Newton linear solve per cell per step (linearization on
    a host thread pool, then all cells' FGMRES in lockstep through one
    libp4d batch: one CUDA graph per Krylov column over all cells).  Under
    torchrun every rank takes its round-robin share of the cells.  At N=1
    also one host thread per cell solve and the cells one after another."""
    import torch
    from p4d_inputs import make_gyroid_batch
    from paper_2602_07225_gb300 import BatchSolver
    from paper_2602_07225_gb300 import build as pbuild
    pbuild.build()
    torch.cuda.set_device(local)
    allc = make_gyroid_batch(64, seed=1004)
    cells = [allc[i] for i in shard(len(allc), rank, world)]
    t0 = time.perf_counter()
    bs = BatchSolver(cells, threads=16, device=torch.device("cuda", local), precision=1, mode=1, rtol=1e-8,
                     maxit=600, cgs_refine=args.cgs_refine, tune_setup=True)
    setup_s = time.perf_counter() - t0
    ndof = sum(s.ndof for s in bs.solvers)
    lib = bs.solvers[0].lib

    def timed(mode, steps):
        for _ in range(max(1, args.warmup // 2)):
            bs.solve_all(mode)
        barrier(world)
        l0 = lib.p4d_launch_count()
        t0 = time.perf_counter()
        its = 0
        out = None
        for _ in range(steps):
            out = bs.solve_all(mode)
            its += sum(info["iters"] for _, info in out)
        el = time.perf_counter() - t0
        barrier(world)
        return el / steps, its / steps, lib.p4d_launch_count() - l0, out

    with ClockSampler(local) as clk:
        lock_s, its, launches, out = timed("lockstep", args.steps)
    bad = sum(1 for _, info in out if info["status"] != 0)
    ms, its_all = aggregate(lock_s * 1e3, its, world, torch.device("cuda", local))
    _, nd_all = aggregate(0.0, ndof, world, torch.device("cuda", local))
    _, bad_all = aggregate(0.0, bad, world, torch.device("cuda", local))
    thr_s = seq_s = None
    if world == 1:
        thr_s, _, _, _ = timed("threads", max(1, args.steps // 2))
        seq_s, _, _, _ = timed("sequential", 1)
    return dict(ncells=len(allc), ndof=int(nd_all), lock_s=ms / 1e3, thr_s=thr_s, seq_s=seq_s, its=its_all,
                launches=launches, setup_s=setup_s, tuned={"%dx%dx%d" % k[:3]: list(v) for k, v in bs.tuned.items()},
                failed=int(bad_all), clocks=clk.summary())


def _field_errors(x, ref, nn):
    """Per-field relative 2-norm errors (phi_s, phi_e, c_e, c_s)."""
    sl = [slice(0, nn), slice(nn, 2 * nn), slice(2 * nn, 3 * nn), slice(3 * nn, x.numel())]
    out = []
    for q in sl:
        nr = float(ref[q].norm())
        out.append(float((x[q] - ref[q]).norm()) / (nr if nr > 0 else 1.0))
    return out


def precision_study(args):
    """Mixed-precision contract on the heterogeneous cube (hetero128): one
    Newton linear solve with the FP64, FP32 and FP32 + BF16-level
    preconditioners, at FGMRES rtol 1e-8 and at the tighter rtol that keeps
    the solution error within 1e-7; each solution's per-field error against
    the FP64 GPU path solved to 1e-12, its iteration count and time.  On a
    64x64x48 heterogeneous box of the same physics (N_c = 10, ~2.2M
    unknowns) the same solves are compared with the oracle's FGMRES solved to
    1e-12."""
    import torch
    from p4d_inputs import make_case, make_box_case
    from paper_2602_07225_gb300 import P4DSolver
    from paper_2602_07225_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    names = {0: "fp64", 1: "fp32", 2: "fp32+bf16 levels"}
    rtols = (1e-8, PRECISION_RTOL)

    def solve_set(case, ref_fn):
        rows = []
        ref = None
        for prec in (0, 1, 2):
            s = P4DSolver(case, device=dev, precision=prec, mode=1, combine=0, rtol=1e-8, restart=30, maxit=600,
                          cheb_degree=CHEB[0], cheb_ratio=CHEB[1])
            st = s.state_tensors(case["state"])
            b = s.residual(st).neg_()
            s.jacobian_update(st)
            if ref is None:
                ref = ref_fn(s, b)
            for rtol in rtols:
                s.set_options(rtol=rtol)
                x, info = s.solve(b)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(3):
                    x, info = s.solve(b)
                e1.record()
                torch.cuda.synchronize()
                err = _field_errors(x, ref, s.nn)
                rows.append({"precision": names[prec], "rtol": rtol, "iters": info["iters"],
                             "ms_per_solve": e0.elapsed_time(e1) / 3, "rel_res": info["rel_res"],
                             "rel_res_unscaled": info["rel_res_unscaled"], "err_phis_phie_ce_cs": err,
                             "max_err": max(err)})
            s.close()
        base = {r["rtol"]: r["iters"] for r in rows if r["precision"] == "fp64"}
        for r in rows:
            r["delta_iters_vs_fp64"] = r["iters"] - base[r["rtol"]]
        return rows

    def gpu_ref(s, b):
        s.set_options(rtol=1e-12, maxit=2000)
        x, info = s.solve(b)
        s.set_options(rtol=1e-8, maxit=600)
        return x.clone()

    full = solve_set(make_case("hetero128"), gpu_ref)

    from oracle.fe import Disc
    from oracle.krylov import LinearSolve
    mid = make_box_case(64, 64, (20, 8, 20), 100e-6, (100e-6, 25e-6, 100e-6), 10, 1003, hetero=True, rs_cv=0.3)
    d = Disc(mid["mesh"], mid["params"])
    t0 = time.perf_counter()
    x_or, its_or, _ = LinearSolve(d, d.state_from_case(mid["state"])).fgmres(rtol=1e-12, degree=CHEB[0],
                                                                               ratio=CHEB[1])
    t_or = time.perf_counter() - t0
    ref_or = torch.tensor(x_or, device=dev)
    midrows = solve_set(mid, lambda s, b: ref_or)
    fp32 = [r for r in full if r["precision"] == "fp32"]
    out = {"study": "precision", "metric": METRIC, "unit": "solves/s",
           "value": 1e3 / fp32[-1]["ms_per_solve"], "n_gpus": 1, "higher_is_better": True,
           "dtype": "f64 outer / {f64, f32, f32+bf16} preconditioner", "data": "synthetic",
           "config": {"workload": "hetero128: Q1 hex 128x128x96 (40/16/40), lognormal porosity (mean 0.3, CV 0.2, "
                                  "correlation 8 elements), lognormal R_s (CV 0.3), N_c=20, seed 1003; REDUCED, BJ, "
                                  + CYCLE + ", FGMRES(30) at rtol 1e-8 and %g; value = FP32 preconditioner at %g"
                                  % (PRECISION_RTOL, PRECISION_RTOL),
                      "reference": "FP64 GPU path solved to rtol 1e-12"},
           "results": full,
           "oracle_box": {"workload": "64x64x48 (20/8/20) heterogeneous box of hetero128's physics, N_c = 10 "
                                      "(seed 1003), %d unknowns" % d.ndof,
                          "reference": "oracle FGMRES to rtol 1e-12 (%d iterations, %.1f s)" % (its_or, t_or),
                          "results": midrows}}
    print(json.dumps(out))


def ordering_study(args):
    """Block Gauss-Seidel over the three macro blocks in each of the 6 orders
    (the particle block is eliminated exactly, so the paper's 24 orderings of
    four blocks reduce to these), against block Jacobi: iterations and time of
    one Newton linear solve to 1e-8 on cube128 and hetero128."""
    import itertools
    import torch
    from p4d_inputs import make_case
    from paper_2602_07225_gb300 import P4DSolver
    from paper_2602_07225_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    fields = ("phi_s", "phi_e", "c_e")
    out = {"study": "bgs_orderings", "metric": METRIC, "unit": "solves/s", "n_gpus": 1, "data": "synthetic",
           "higher_is_better": True, "dtype": "f64 outer / f32 preconditioner", "results": {}}
    for wl in ("cube128", "hetero128"):
        case = make_case(wl)
        s = P4DSolver(case, device=dev, precision=1, mode=1, combine=0, rtol=1e-8, restart=30, maxit=600,
                      cheb_degree=CHEB[0], cheb_ratio=CHEB[1])
        st = s.state_tensors(case["state"])
        b = s.residual(st).neg_()
        s.jacobian_update(st)
        rows = []
        for combine, order in [(0, (1, 0, 2))] + [(1, o) for o in itertools.permutations(range(3))]:
            s.set_options(combine=combine, order=order)
            s.solve(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(3):
                x, info = s.solve(b)
            e1.record()
            torch.cuda.synchronize()
            rows.append({"combine": "BJ" if combine == 0 else "BGS", "order": [fields[i] for i in order] if combine else None,
                         "iters": info["iters"], "ms_per_solve": e0.elapsed_time(e1) / 3, "rel_res": info["rel_res"]})
        s.close()
        out["results"][wl] = rows
    best = min(out["results"]["cube128"], key=lambda r: r["ms_per_solve"])
    out["value"] = 1e3 / best["ms_per_solve"]
    out["config"] = {"workload": "cube128 and hetero128, REDUCED, " + CYCLE + ", FGMRES(30) rtol 1e-8; value = the "
                                 "fastest combination on cube128 (linear solve only)"}
    print(json.dumps(out))


def slab_study(args):
    """cube128 (seeded linearization, seed 1002) cut into 1, 2, 4 and 8 z
    slabs on this one GPU (p4d_dd_*): one handle per slab, ghost planes
    exchanged before every operator application, every inner product reduced
    over the slabs, restricted additive Schwarz over the slabs (1, 4 or 8
    ghost planes) with and without the two-level coarse correction.  Iterations,
    time of one
    Newton linear solve to 1e-8 and the solution's per-field difference from
    the undecomposed solve; what one slab per GPU would add (the transfers
    and allreduces over the interconnect) is not in these times."""
    import numpy as np
    import torch
    from p4d_inputs import make_case, slab_cases, slab_node_rows
    from paper_2602_07225_gb300 import P4DSolver, SlabSolver
    from paper_2602_07225_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    case = make_case("cube128")
    m = case["mesh"]
    nxy = (m["nx"] + 1) * (m["ny"] + 1)
    opts = dict(precision=1, mode=1, combine=0, rtol=1e-8, restart=30, maxit=1000, cheb_degree=CHEB[0],
                cheb_ratio=CHEB[1], cgs_refine=args.cgs_refine)

    def timed(fn, reps=3):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / reps

    s = P4DSolver(case, device=dev, **opts)
    st = s.state_tensors(case["state"])
    b = s.residual(st).neg_()
    s.jacobian_update(st)
    (x1, info1), ms1 = timed(lambda: s.solve(b))
    x1 = x1.cpu().numpy()
    nn = s.nn
    s.close()
    del st, b
    torch.cuda.empty_cache()
    rows = [{"slabs": 1, "driver": "single cell", "iters": info1["iters"], "ms_per_solve": ms1,
             "rel_res": info1["rel_res"]}]
    for nparts, coarse, ghosts in ((1, 0, 1), (2, 0, 1), (2, 0, 4), (2, 2, 4), (4, 0, 4), (4, 2, 4), (4, 2, 8),
                                   (8, 0, 4), (8, 2, 4), (8, 2, 8)):
        slabs = slab_cases(case, nparts, ghosts)
        dd = SlabSolver(slabs, device=dev, coarse=coarse, **opts)
        sts = dd.state_tensors()
        bs = [r.neg_() for r in dd.residual(sts)]
        dd.jacobian_update(sts)
        (xs, info), ms = timed(lambda: dd.solve(bs, check=False), reps=2)
        diff = 0.0
        for i, (sl, xp) in enumerate(zip(slabs, xs)):
            glob, loc = slab_node_rows(sl, nxy)
            xv, nns = xp.cpu().numpy(), dd.parts[i].nn
            for f in range(3):
                ref = x1[f * nn:(f + 1) * nn]
                diff = max(diff, float(np.abs(xv[f * nns + loc] - ref[glob]).max() / np.abs(ref).max()))
        rows.append({"slabs": nparts, "driver": "decomposed", "ghost_planes": ghosts,
                     "coarse": ["none", "constants", "constants + z"][coarse], "status": info["status"],
                     "iters": info["iters"], "ms_per_solve": ms,
                     "rel_res": info["rel_res"], "rel_res_unscaled": info["rel_res_unscaled"],
                     "max_field_diff_vs_cell": diff})
        print("slabs %d ghosts %d coarse %d: %d iterations, status %d" % (nparts, ghosts, coarse, info["iters"],
                                                                         info["status"]), file=sys.stderr)
        dd.close()
        del dd, sts, bs, xs
        torch.cuda.empty_cache()
    out = {"study": "slab_decomposition", "metric": METRIC, "unit": "solves/s", "n_gpus": 1, "data": "synthetic",
           "higher_is_better": True, "dtype": "f64 outer / f32 preconditioner", "results": rows,
           "value": 1e3 / rows[4]["ms_per_solve"],
           "config": {"workload": "cube128 seeded linearization (seed 1002) as 1-8 z slabs on one GPU, REDUCED, "
                                  + CYCLE + ", FGMRES(30) rtol 1e-8, " + CGS_DESC[args.cgs_refine]
                                  + "; restricted additive Schwarz over the slabs with 1, 4 or 8 ghost planes, with "
                                    "or without the coarse correction; value = two slabs, 4 ghost planes, coarse "
                                    "correction (linear solve only)"}}
    print(json.dumps(out))


def slab_adjoint(args):
    """Adjoint of the flattened jelly-roll slab: 2048x16x48 elements
    (20/8/20), N_c = 15, tabs on the first 64 element columns (applied
    current on the cathode face, ground on the anode face), 2C, 30
    backward-Euler steps of 10 s.  Gradient of the terminal voltage after
    the last step with respect to per-element sigma_s, D_s and eps through
    the torch.autograd.Function with checkpoints every 5 steps, checked
    against central differences (relative step 1e-5, Newton to 1e-12).  A
    single element's sensitivity here moves V by ~1e-12 V, below the FP64
    resolution of V (~4e-16 x 3.7 V) plus the Newton floor, so the checks
    are directional: each perturbs one parameter on a seeded block of
    16x16x4 electrode elements and compares g . dp with the central
    difference along dp."""
    import numpy as np
    import torch
    from p4d_inputs import make_slab_case
    from paper_2602_07225_gb300 import terminal_voltage
    from paper_2602_07225_gb300 import build as pbuild
    pbuild.build()
    nx = args.slab_nx
    nsteps = args.slab_steps
    tab = max(1, 64 * nx // 2048)
    if args.slab_geometry == "paper":
        # the paper's jelly roll: 1 m x 5 cm, 50/20/50 um layers; the foils as thin
        # shells: aluminium 3.77e7 S/m x 15 um (cathode), copper 5.96e7 S/m x 10 um (anode)
        geo = dict(h_lat=1.0 / nx, width=0.05, L_layers=(50e-6, 20e-6, 50e-6), shell=(565.5, 596.0))
    else:
        geo = {}
    case = make_slab_case(nx=nx, ny=16, layers=(20, 8, 20), nc=15, seed=1005, tab=tab, crate=2.0, **geo)
    m, p = case["mesh"], case["params"]
    region = m["region"]
    nz = int(m["nz"])
    sig0 = np.where(region == 0, p["sigma_n"], np.where(region == 2, p["sigma_p"], 0.0))
    D0 = np.full(region.size, 1e-14)
    eps0 = np.asarray(m["eps"], float).copy()
    # FGMRES(100): the restart length of the paper's jelly-roll runs.  With the
    # foils the rows span ~1e8 more in stiffness: FGMRES stagnates below ~1e-9
    # there (the FP64 resolution of the foil-dominated system), so the paper
    # geometry runs at 1e-8 / Newton 1e-10
    tight = args.slab_geometry != "paper"
    opts = dict(precision=1, mode=1, rtol=1e-10 if tight else 1e-8, restart=100, maxit=1500,
                newton_rtol=1e-12 if tight else 1e-10, newton_maxit=30, cheb_degree=CHEB[0], cheb_ratio=CHEB[1])

    def V_of(s_, d_, e_):
        with torch.no_grad():
            return terminal_voltage(torch.tensor(s_), torch.tensor(d_), torch.tensor(e_), case, nsteps, 5,
                                    **dict(opts)).item()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    V0 = V_of(sig0, D0, eps0)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t = [torch.tensor(a, requires_grad=True) for a in (sig0, D0, eps0)]
    t0 = time.perf_counter()
    V = terminal_voltage(*t, case, nsteps, 5, **dict(opts))
    V.backward()
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    grads = [ti.grad.numpy() for ti in t]
    rng = np.random.default_rng(1005)
    checks = []
    h = 1e-5
    ei_, ej_, ek_ = np.meshgrid(np.arange(nx), np.arange(16), np.arange(nz), indexing="ij")
    for c in range(args.slab_fd):
        k = c % 3
        base = (sig0, D0, eps0)[k]
        reg = 0 if rng.random() < 0.5 else 2
        layers = np.flatnonzero(region.reshape(nz, 16, nx)[:, 0, 0] == reg)
        i0 = int(rng.integers(0, max(1, nx - 16)))
        k0 = int(layers[rng.integers(0, max(1, len(layers) - 4))])
        blk = ((ei_ >= i0) & (ei_ < i0 + 16) & (ek_ >= k0) & (ek_ < k0 + 4)).transpose(2, 1, 0).ravel()
        blk &= region == reg
        dp = np.where(blk, base, 0.0)
        vals = []
        for sgn in (1, -1):
            pp = [sig0, D0, eps0]
            pp[k] = base + sgn * h * dp
            vals.append(V_of(*pp))
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = float(grads[k] @ dp)
        checks.append({"param": ("sigma_s", "D_s", "eps")[k], "region": ("anode", "", "cathode")[reg],
                       "block": [i0, k0], "elements": int(blk.sum()), "adjoint": ad, "fd": float(fd),
                       "rel_err": float(abs(ad - fd) / max(abs(fd), 1e-300))})
    out = {"study": "adjoint_slab", "metric": METRIC, "unit": "gradients/s", "value": 1.0 / t_grad, "n_gpus": 1,
           "higher_is_better": True, "data": "synthetic", "dtype": "f64 outer / f32 preconditioner",
           "config": {"workload": "jelly-roll slab %dx16x48 (20/8/20), N_c=15, tabs on %d columns, 2C, %d BE steps "
                                  "x 10 s, checkpoints every 5" % (nx, tab, nsteps)
                                  + (", the paper's geometry (1 m x 5 cm, 50/20/50 um) with collector foils "
                                     "(565.5 and 596 S shells)" if args.slab_geometry == "paper" else
                                     ", 0.78 um lateral elements, 100/25/100 um layers, no foils"),
                      "unknowns": int(3 * (nx + 1) * 17 * 49 + 15 * (nx + 1) * 17 * 42)},
           "V_final": V0, "forward_s": t_fwd, "gradient_s": t_grad, "fd_checks": checks,
           "max_rel_err": max(c["rel_err"] for c in checks) if checks else None}
    print(json.dumps(out))

def main():
    args = parse()
    if args.workload == "slab2048" and args.impl == "gpu":
        slab_adjoint(args)
        return
    if args.workload == "slabs128" and args.impl == "gpu":
        slab_study(args)
        return
    if args.workload == "orderings" and args.impl == "gpu":
        ordering_study(args)
        return
    if args.workload == "hetero128" and args.impl == "gpu":
        precision_study(args)
        return
    if args.workload == "gyroid64" and args.impl == "gpu":
        rank, world, local = dist_env()
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        r = batched_leg(args, rank, world, local)
        if rank != 0:
            return
        seq = {} if r["seq_s"] is None else {
            "threads_solves_per_s": r["ncells"] / r["thr_s"],
            "sequential_solves_per_s": r["ncells"] / r["seq_s"],
            "speedup_vs_sequential": r["seq_s"] / r["lock_s"]}
        out = {"metric": METRIC, "value": r["ncells"] / r["lock_s"], "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["lock_s"] * 1e3,
               "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
               "dtype": "f64 outer / f32 preconditioner", "data": "synthetic",
               "config": {"workload": "gyroid64: 64 gyroid cells 16x16x24..64x64x96, N_c 10-20, one Newton "
                                      "linear solve per cell per step, lockstep batch (one CUDA graph per "
                                      "Krylov column over all cells), autotuned smoother, block combination, "
                                      "coarsening threshold and level-0 tile depth per shape, "
                                      + CGS_DESC[args.cgs_refine],
                          "unknowns": r["ndof"], "l2": "inputs larger than L2"},
               "fgmres_iters_per_s": r["its"] / r["lock_s"], **seq, "setup_s": r["setup_s"], "tuned": r["tuned"],
               "failed_cells": r["failed"], "gpu_launches": r["launches"], "clocks": r["clocks"]}
        print(json.dumps(out))
        return
    args = args
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        if args.impl == "gpu":
            dist.init_process_group("nccl")
        else:
            if rank != 0:
                return
    if args.impl == "reference":
        if rank != 0:
            return
        reference_main(args)
        return
    r = gpu_leg(args, rank, world, local)
    if rank != 0:
        return
    pk, src = peaks()
    peak = pk.get("hbm_gbs", 6800.0)
    cpu = None
    if not args.no_cpu and world == 1:
        try:
            cores = os.cpu_count()
            c = cpu_oracle_leg(r["ndof"], combine=args.combine)
            cpu = {"value": c["scaled_solves_per_s"], "unit": "solves/s", "cores": cores, "kind": "oracle",
                   "sample": "oracle Newton with FGMRES linear solves (BJ, " + CYCLE + ", FP64) for %d backward-"
                             "Euler step(s) from rest of a 16x16x96 column block of the cube128 workload "
                             "(%d unknowns, %d linear solves, %.1f s/solve, %.1f its/solve), scaled by unknowns"
                             % (c["steps"], c["sample_dof"], c["solves"], c["s_per_solve"], c["iters_per_solve"])}
        except Exception as e:  # pragma: no cover
            cpu = {"value": None, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "failed: %s" % e}
    tot = r["tot"]
    roof = r["roof"]
    f64 = r["fp64_rate"]
    traffic = TRAFFIC_PER_ROW * roof["rows"] if args.workload == "cube128" else None
    out = {
        "metric": METRIC,
        "value": r["solves_per_s"],
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 outer / f32 preconditioner",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload) +
                               ", 1C discharge from rest (theta_n 0.8, theta_p 0.6, c_e 1000), "
                               "one step = one backward-Euler step of 10 s by Newton (scaled residual 1e-8), "
                               "REDUCED Schur mode, " + COMBINE_DESC[args.combine] + ", " + CYCLE
                               + ", FGMRES(30) rtol 1e-8, "
                               + CGS_DESC[args.cgs_refine]
                               + (", the paper's OCP curves and kappa(c_e), D_e(c_e)" if args.laws == "paper" else ""),
                   "time_steps": args.steps, "unknowns": r["ndof"],
                   "l2": "inputs larger than L2 (Krylov basis and stencils > 129 MB)"},
        "fgmres_iters_per_s": r["iters_per_s"],
        "linear_solves": tot["solves"],
        "newton_iters": tot["newton"],
        "fgmres_iters": tot["iters"],
        "iters_per_solve": tot["iters"] / max(1, tot["solves"]),
        "dof_iters_per_s": r["iters_per_s"] * r["ndof"],
        "rel_res": tot["rel_res"],
        "rel_res_unscaled": tot["rel_res_unscaled"],
        "rel_res_block_unscaled": tot["rel_res_block_unscaled"],
        "reorth": tot["reorth"],
        "fp64_path": r["fp64"],
        "e2e": {"value": tot["solves"] / (r["e2e_ms"] * args.steps / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"],
        "roofline": {"bound": "hbm", "achieved": roof["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": roof["gbs"] / peak, "traffic": traffic,
                     "traffic_source": TRAFFIC_SOURCE,
                     "kernel": roof["kernel"], "peak_source": src, "ms_per_launch": roof["ms"],
                     "bytes_per_launch": roof["bytes"],
                     "bytes_note": "%d B per node and field (the method's algorithmic bytes of a fine-level "
                                   "Chebyshev step: x, b, 1/diag, d in, d and x out) x %d rows"
                                   % (ALG_BYTES_SMOOTH0, roof["rows"]),
                     "kernel_bytes_per_launch": roof["kernel_bytes"],
                     "kernel_gbs": roof["kernel_gbs"], "kernel_frac": roof["kernel_gbs"] / peak},
        "solve_phases_ms": roof["phases_ms"],
        "profiled_solve": roof["solve"],
        "roofline_fp64": {"kernel": "k_jvp_combine + k_jvp_macro (reduced FP64 JVP inside FGMRES)", "bound": "alu",
                          "achieved": roof["jvp"]["tflops"], "peak": f64 or FP64_TFLOPS, "unit": "TFLOP/s",
                          "frac": roof["jvp"]["tflops"] / (f64 or FP64_TFLOPS),
                          "ms_per_launch": roof["jvp"]["ms"],
                          "peak_source": "measured FP64 FMA chain (p4d_fp64_fma_rate), this run" if f64 else
                                         "GB300 nominal FP64 (non-tensor)"},
        "cpu_baseline": cpu,
        "clocks": r["clocks"],
    }
    print(json.dumps(out))


def reference_main(args):
    """--impl reference: the FP64 oracle (plain Newton with block-preconditioned
    FGMRES linear solves), on the host cores, on bounded samples of the same
    workload: each step is the first backward-Euler step from rest of a
    16x16x96 column block of the cube, its linear solves/s scaled by unknowns."""
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        pass
    vals = []
    its = []
    for _ in range(max(1, args.steps)):
        c = cpu_oracle_leg(CUBE128_DOF, seconds_hint=10.0, combine=args.combine)
        vals.append(c["scaled_solves_per_s"])
        its.append(c["iters_per_solve"])
        if time.perf_counter() - t0 > 150:
            break
    v = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": 0,
           "steps": len(vals), "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "cube128 1C discharge from rest (bounded 16x16x96 column samples: the first "
                                  "backward-Euler step, Newton + FGMRES, scaled by unknowns)"},
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "first backward-Euler step of a 16x16x96 column block of cube128 per step"},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
