"""Many independent cells of uneven sizes solved together.

Each cell owns a libp4d handle and a CUDA stream.  A pool of host threads
linearizes the cells (ctypes releases the GIL during library calls); the
solves then run in lockstep through one libp4d batch (p4d_batch_*): one CUDA
graph per Krylov column holds every cell's Arnoldi step under a conditional
node, so the small launches of small cells overlap on the GPU and the host
synchronizes once per column for the whole batch.  The "threads" mode
(each thread also drives its cell's solve) and "sequential" mode are kept
for comparison.  An autotuner picks the
Chebyshev degree and interval per (mesh shape, precision) by timing one
solve of the first cell of each grid shape (N_c does not enter the
multigrid: the particle blocks are eliminated exactly), then the block
combination (block Jacobi or block Gauss-Seidel in each order of the fields)
with that smoother, then the two options fixed when a handle is set up: the
coarsening threshold coarse_max (the multigrid's level count) and the z
depth of the matrix-free level-0 tile (mf_zchunk), each candidate on a
handle built for it; results are cached in memory and optionally in a JSON
file.
"""
import concurrent.futures as cf
import ctypes as C
import itertools
import json
import os

import torch

from . import _native as N
from .solver import P4DSolver

CANDIDATES = ((1, 4.0), (2, 10.0), (3, 10.0), (3, 20.0), (4, 20.0))
# block combinations after the smoother: block Jacobi, then block
# Gauss-Seidel in every order of the fields (0 phi_s, 1 phi_e, 2 c_e)
BJ = (0, (1, 0, 2))
COMBOS = (BJ,) + tuple((1, o) for o in itertools.permutations((0, 1, 2)))
# (coarse_max, mf_zchunk), the library defaults first.  No coarsest level
# larger than the default's: timed on one cell a larger dense coarsest solve
# looks free (the GPU is idle around it), but with all cells of a batch in
# flight it doubled the time per Arnoldi step
SETUP_DEFAULT = (128, 8)
SETUP_CANDIDATES = (SETUP_DEFAULT, (32, 8), (64, 8), (128, 4), (128, 16))


class Autotuner:
    def __init__(self, path=None):
        self.path = path
        self.cache = {}
        if path and os.path.exists(path):
            with open(path) as fh:
                self.cache = {tuple(json.loads(k)): tuple(v) for k, v in json.load(fh).items()}

    @staticmethod
    def key(solver, case):
        # the smoother acts on the electrode-level grid only: N_c does not enter
        m = case["mesh"]
        return (int(m["nx"]), int(m["ny"]), int(m["nz"]), int(solver.params.precision))

    @staticmethod
    def _time(solver, b):
        """Device time of one FGMRES solve with the current options (the first
        solve after an option change captures the CUDA graphs and is not
        timed); inf when it does not converge."""
        solver.solve(b, check=False)
        _, info = solver.solve(b, check=False)
        return info["ms_total"] if info["status"] == 0 else float("inf")

    def tune(self, solver, state, b):
        """(cheb_degree, cheb_ratio, combine, order) for this solver's shape:
        first the Chebyshev smoother under block Jacobi, then the block
        combination with that smoother, each by device time of one FGMRES
        solve (the linearization is shared)."""
        best_s, best_ms = (2, 10.0), float("inf")
        for deg, ratio in CANDIDATES:
            solver.set_options(cheb_degree=deg, cheb_ratio=ratio, combine=BJ[0], order=BJ[1])
            ms = self._time(solver, b)
            if ms < best_ms:
                best_s, best_ms = (deg, ratio), ms
        best = best_s + BJ
        for combine, order in COMBOS[1:]:
            solver.set_options(cheb_degree=best_s[0], cheb_ratio=best_s[1], combine=combine, order=order)
            ms = self._time(solver, b)
            if ms < best_ms:
                best, best_ms = best_s + (combine, order), ms
        return best

    def tune_setup(self, build, runtime):
        """(coarse_max, mf_zchunk): build(coarse_max, mf_zchunk) returns a
        linearized solver of the shape and its right-hand side; each
        candidate runs with the runtime options chosen before."""
        best, best_ms = SETUP_DEFAULT, float("inf")
        for cm, zc in SETUP_CANDIDATES:
            s, b = build(cm, zc)
            s.set_options(**runtime)
            ms = self._time(s, b)
            if hasattr(s, "close"):
                s.close()
            if ms < best_ms:
                best, best_ms = (cm, zc), ms
        return best

    def get(self, solver, case, state, b, build=None):
        """(cheb_degree, cheb_ratio, combine, order, coarse_max, mf_zchunk);
        without build the setup options stay at the library defaults."""
        k = self.key(solver, case)
        if k not in self.cache or (build is not None and len(self.cache[k]) < 6):
            got = self.cache[k][:4] if k in self.cache else self.tune(solver, state, b)
            deg, ratio, combine, order = got
            setup = SETUP_DEFAULT
            if build is not None:
                setup = self.tune_setup(build, dict(cheb_degree=deg, cheb_ratio=ratio, combine=combine,
                                                    order=tuple(order)))
            self.cache[k] = tuple(got) + tuple(setup)
            if self.path:
                with open(self.path, "w") as fh:
                    json.dump({json.dumps(list(kk)): list(v) for kk, v in self.cache.items()}, fh)
        v = self.cache[k]
        return tuple(v) + (tuple(SETUP_DEFAULT) if len(v) < 6 else ())


class BatchSolver:
    """cases: list of generator cases; opts: P4DSolver options.  With
    tune_setup the autotuner also searches coarse_max and mf_zchunk (each
    candidate builds a handle of the shape's first cell)."""

    def __init__(self, cases, threads=16, autotune=True, tuner=None, device="cuda", tune_setup=False, **opts):
        self.cases = cases
        self.threads = threads
        self.opts = dict(opts)
        self.device = device
        self.solvers, self.states = [], []
        for c in cases:
            s, stt = self._make(c, opts)
            self.solvers.append(s)
            self.states.append(stt)
        torch.cuda.synchronize()
        self._batch = None
        self.tuner = tuner or (Autotuner() if autotune else None)
        self.tuned = {}
        if self.tuner:
            for i, c in enumerate(self.cases):
                s = self.solvers[i]
                k = Autotuner.key(s, c)
                if k not in self.tuned:
                    with torch.cuda.stream(s.stream):
                        b = s.residual(self.states[i]).neg_()
                        s.jacobian_update(self.states[i])
                        build = (lambda cm, zc, c=c: self._build_linearized(c, cm, zc)) if tune_setup else None
                        self.tuned[k] = self.tuner.get(s, c, self.states[i], b, build=build)
                deg, ratio, combine, order, cm, zc = self.tuned[k]
                want = dict(coarse_max=cm, mf_zchunk=zc)
                if (int(s.params.coarse_max), int(s.params.mf_zchunk) or SETUP_DEFAULT[1]) != (cm, zc):
                    s.close()
                    s, self.states[i] = self._make(c, {**opts, **want})
                    self.solvers[i] = s
                s.set_options(cheb_degree=deg, cheb_ratio=ratio, combine=combine, order=tuple(order))
        torch.cuda.synchronize()

    def _make(self, c, opts):
        st = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(st):
            s = P4DSolver(c, device=self.device, stream=st, **opts)
            return s, s.state_tensors(c["state"])

    def _build_linearized(self, c, coarse_max, mf_zchunk):
        s, stt = self._make(c, {**self.opts, "coarse_max": coarse_max, "mf_zchunk": mf_zchunk})
        with torch.cuda.stream(s.stream):
            b = s.residual(stt).neg_()
            s.jacobian_update(stt)
        return s, b

    def _linearize(self, i):
        s, st = self.solvers[i], self.states[i]
        with torch.cuda.stream(s.stream):
            b = s.residual(st).neg_()
            s.jacobian_update(st)
        return b

    def _solve_one(self, i):
        s = self.solvers[i]
        b = self._linearize(i)
        with torch.cuda.stream(s.stream):
            x, info = s.solve(b)
        return x, info

    def _order(self):
        # largest cells first: the long solves start while the small ones
        # fill the gaps (longest-processing-time-first order)
        return sorted(range(len(self.solvers)), key=lambda i: -self.solvers[i].ndof)

    def _batch_handle(self):
        if self._batch is None:
            lib = self.solvers[0].lib
            n = len(self.solvers)
            hs = (C.c_void_p * n)(*[s.h for s in self.solvers])
            out = C.c_void_p()
            N.check(lib.p4d_batch_create(hs, n, C.byref(out)), "p4d_batch_create")
            self._batch = out
        return self._batch

    def solve_batched(self, rhs, adjoint=False):
        """Lockstep FGMRES over all cells: rhs a list of device tensors;
        returns [(x, info)]."""
        lib = self.solvers[0].lib
        n = len(self.solvers)
        xs = [torch.zeros_like(b) for b in rhs]
        bp = (C.c_void_p * n)(*[b.data_ptr() for b in rhs])
        xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        infos = (N.Info * n)()
        fn = lib.p4d_batch_adjoint_solve if adjoint else lib.p4d_batch_fgmres_solve
        st = fn(self._batch_handle(), bp, xp, infos)
        out = []
        for i in range(n):
            out.append((xs[i], infos[i].as_dict()))
        if st not in (N.OK, N.NOT_CONVERGED, N.BREAKDOWN, N.NONFINITE):
            raise N.P4DError(st, "p4d_batch_fgmres_solve")
        return out

    def solve_all(self, mode="lockstep"):
        """One Newton linear solve per cell; returns [(x, info)].
        mode: "lockstep" (one batch), "threads" (one host thread per cell
        solve) or "sequential" (cells one after another)."""
        n = len(self.solvers)
        if mode == "sequential":
            out = [self._solve_one(i) for i in range(n)]
        elif mode == "threads":
            order = self._order()
            out = [None] * n
            with cf.ThreadPoolExecutor(max_workers=self.threads) as ex:
                for i, r in zip(order, ex.map(self._solve_one, order)):
                    out[i] = r
        elif mode == "lockstep":
            order = self._order()
            rhs = [None] * n
            with cf.ThreadPoolExecutor(max_workers=self.threads) as ex:
                for i, b in zip(order, ex.map(self._linearize, order)):
                    rhs[i] = b
            out = self.solve_batched(rhs)
        else:
            raise ValueError("mode: lockstep, threads or sequential")
        torch.cuda.synchronize()
        return out

    def close(self):
        if self._batch is not None:
            self.solvers[0].lib.p4d_batch_destroy(self._batch)
            self._batch = None
        for s in self.solvers:
            s.close()
