"""Many independent cells of uneven sizes solved together.

Each cell owns a libp4d handle and a CUDA stream; a pool of host threads
drives the per-cell Newton linear solves (ctypes releases the GIL during
library calls), so the many small launches of small cells overlap on the
GPU instead of running one cell after another.  An autotuner picks the
Chebyshev degree and interval per (mesh shape, N_c, precision) by timing
one solve of the first cell of each grid shape (N_c does not enter the
multigrid); results are cached in memory and optionally in a JSON file.
"""
import concurrent.futures as cf
import json
import os

import torch

from .solver import P4DSolver

CANDIDATES = ((1, 4.0), (2, 10.0), (3, 10.0), (3, 20.0), (4, 20.0))


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

    def tune(self, solver, state, b):
        """Best (cheb_degree, cheb_ratio) for this solver's shape by device time
        of one FGMRES solve per candidate (the linearization is shared)."""
        best, best_ms = None, float("inf")
        for deg, ratio in CANDIDATES:
            solver.set_options(cheb_degree=deg, cheb_ratio=ratio)
            _, info = solver.solve(b, check=False)
            if info["status"] == 0 and info["ms_total"] < best_ms:
                best, best_ms = (deg, ratio), info["ms_total"]
        return best if best is not None else (2, 10.0)

    def get(self, solver, case, state, b):
        k = self.key(solver, case)
        if k not in self.cache:
            self.cache[k] = self.tune(solver, state, b)
            if self.path:
                with open(self.path, "w") as fh:
                    json.dump({json.dumps(list(kk)): list(v) for kk, v in self.cache.items()}, fh)
        return self.cache[k]


class BatchSolver:
    """cases: list of generator cases; opts: P4DSolver options."""

    def __init__(self, cases, threads=16, autotune=True, tuner=None, device="cuda", **opts):
        self.cases = cases
        self.threads = threads
        self.solvers, self.states = [], []
        for c in cases:
            st = torch.cuda.Stream(device=device)
            with torch.cuda.stream(st):
                s = P4DSolver(c, device=device, stream=st, **opts)
                self.solvers.append(s)
                self.states.append(s.state_tensors(c["state"]))
        torch.cuda.synchronize()
        self.tuner = tuner or (Autotuner() if autotune else None)
        self.tuned = {}
        if self.tuner:
            for i, (s, c) in enumerate(zip(self.solvers, self.cases)):
                k = Autotuner.key(s, c)
                if k not in self.tuned:
                    with torch.cuda.stream(s.stream):
                        b = s.residual(self.states[i]).neg_()
                        s.jacobian_update(self.states[i])
                        self.tuned[k] = self.tuner.get(s, c, self.states[i], b)
                deg, ratio = self.tuned[k]
                s.set_options(cheb_degree=deg, cheb_ratio=ratio)
        torch.cuda.synchronize()

    def _solve_one(self, i):
        s, st = self.solvers[i], self.states[i]
        with torch.cuda.stream(s.stream):
            b = s.residual(st).neg_()
            s.jacobian_update(st)
            x, info = s.solve(b)
        return x, info

    def solve_all(self, concurrent=True):
        """One Newton linear solve per cell; returns [(x, info)]."""
        if not concurrent:
            out = [self._solve_one(i) for i in range(len(self.solvers))]
        else:
            # largest cells first: the long solves start while the small ones
            # fill the gaps (longest-processing-time-first order)
            order = sorted(range(len(self.solvers)), key=lambda i: -self.solvers[i].ndof)
            out = [None] * len(self.solvers)
            with cf.ThreadPoolExecutor(max_workers=self.threads) as ex:
                for i, r in zip(order, ex.map(self._solve_one, order)):
                    out[i] = r
        torch.cuda.synchronize()
        return out

    def close(self):
        for s in self.solvers:
            s.close()
