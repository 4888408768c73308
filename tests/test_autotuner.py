"""The batch autotuner's search on the host (a fake solver, no GPU): every
candidate is solved once to capture its graphs and timed on a second solve;
the smoother is chosen under block Jacobi first, then the block combination
with that smoother; non-converging candidates never win; results are cached
per shape and precision and round-trip through the JSON cache file; the
setup-time options (coarse_max, mf_zchunk) are searched last, each on a
handle built for it."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2602_07225_gb300.batch import (BJ, CANDIDATES, COMBOS, SETUP_CANDIDATES, SETUP_DEFAULT,  # noqa: E402
                                          Autotuner)


class _Params:
    precision = 1


class FakeSolver:
    """solve() reports the time of the current options from a table; the
    first solve after an option change is slower (graph capture)."""

    def __init__(self, ms, fail=()):
        self.ms, self.fail = ms, set(fail)
        self.params = _Params()
        self.opts = {}
        self.fresh = True
        self.calls = []

    def set_options(self, **o):
        self.opts = dict(o)
        self.fresh = True

    def key(self):
        o = self.opts
        return (o["cheb_degree"], o["cheb_ratio"], o["combine"], tuple(o["order"]))

    def solve(self, b, check=True):
        k = self.key()
        self.calls.append((k, self.fresh))
        ms = self.ms.get(k, 10.0) + (100.0 if self.fresh else 0.0)
        self.fresh = False
        return None, {"status": 1 if k in self.fail else 0, "ms_total": ms}


def _case(n=16):
    return {"mesh": {"nx": n, "ny": n, "nz": int(1.5 * n)}}


def test_two_stage_search_and_warm_timing():
    best_s = (2, 10.0)
    ms = {s + BJ: 9.0 for s in CANDIDATES}
    ms[best_s + BJ] = 5.0
    order = (0, 1, 2)
    ms[best_s + (1, order)] = 4.0                 # one BGS order beats block Jacobi
    ms[(4, 20.0) + (1, order)] = 1.0              # never tried: not the chosen smoother
    fs = FakeSolver(ms)
    got = Autotuner().tune(fs, None, None)
    assert got == best_s + (1, order)
    # every candidate: one capture solve, then one timed solve
    assert len(fs.calls) == 2 * (len(CANDIDATES) + len(COMBOS) - 1)
    assert all(fresh for _, fresh in fs.calls[0::2]) and not any(fresh for _, fresh in fs.calls[1::2])
    # stage 2 runs with the stage-1 smoother only
    stage2 = {k for k, _ in fs.calls[2 * len(CANDIDATES):]}
    assert {k[:2] for k in stage2} == {best_s}


def test_failed_candidates_never_win_and_cache_round_trip(tmp_path):
    ms = {s + BJ: 9.0 for s in CANDIDATES}
    ms[(1, 4.0) + BJ] = 0.5
    fs = FakeSolver(ms, fail={(1, 4.0) + BJ})
    path = str(tmp_path / "tune.json")
    tuner = Autotuner(path)
    got = tuner.get(fs, _case(), None, None)
    assert got[:2] != (1, 4.0) and got[2:4] == BJ and got[4:] == SETUP_DEFAULT
    # cached: no further solves for the same shape and precision
    n = len(fs.calls)
    assert tuner.get(fs, _case(), None, None) == got and len(fs.calls) == n
    # a new tuner reads the file
    again = Autotuner(path)
    key = Autotuner.key(fs, _case())
    assert list(again.cache[key][:3]) == list(got[:3]) and list(again.cache[key][3]) == list(got[3])
    json.load(open(path))


def test_setup_stage_builds_each_candidate_and_keeps_the_runtime_choice(tmp_path):
    ms = {s + BJ: 9.0 for s in CANDIDATES}
    ms[(3, 10.0) + BJ] = 5.0
    fs = FakeSolver(ms)
    built, closed = [], []

    class Built(FakeSolver):
        def close(self):
            closed.append(self.setup)

    speed = {c: 7.0 for c in SETUP_CANDIDATES}
    speed[(64, 8)] = 3.0
    speed[(32, 8)] = 2.0
    fail = (32, 8)                                 # the fastest does not converge: never chosen

    def build(cm, zc):
        b = Built({}, fail={(3, 10.0) + BJ} if (cm, zc) == fail else ())
        b.setup = (cm, zc)
        b.ms = {(3, 10.0) + BJ: speed[(cm, zc)]}
        built.append((cm, zc))
        return b, None

    tuner = Autotuner(str(tmp_path / "t.json"))
    got = tuner.get(fs, _case(24), None, None, build=build)
    assert got == (3, 10.0) + BJ + (64, 8)
    assert built == list(SETUP_CANDIDATES) and closed == built


def test_cached_runtime_choice_gains_setup_options(tmp_path):
    path = str(tmp_path / "old.json")
    key = [16, 16, 24, 1]
    json.dump({json.dumps(key): [2, 10.0, 0, [1, 0, 2]]}, open(path, "w"))
    tuner = Autotuner(path)
    fs = FakeSolver({})
    assert tuner.get(fs, _case(), None, None) == (2, 10.0, 0, [1, 0, 2]) + SETUP_DEFAULT
    assert fs.calls == []                          # no runtime search for a cached shape

    def build(cm, zc):
        b = FakeSolver({(2, 10.0, 0, (1, 0, 2)): 1.0 if (cm, zc) == (128, 16) else 4.0})
        return b, None

    got = tuner.get(fs, _case(), None, None, build=build)
    assert got[:4] == (2, 10.0, 0, [1, 0, 2]) and got[4:] == (128, 16) and fs.calls == []
