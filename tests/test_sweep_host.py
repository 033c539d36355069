"""The sweep's agreement rule on the host (no GPU): each stated class, the order
in which they are checked, and the continuation of the run that stopped first.
The continuation itself is replaced by a stand-in that records its arguments."""
import math

import pytest

from paper_1906_11027_gb300 import sweep

INF = float("inf")


def arm(us, steps):
    return {"obs": [{"max_u": u} for u in us], "steps": list(steps), "states64": {}, "batch": None}


@pytest.fixture
def continued(monkeypatch):
    calls = []
    table = {}

    def fake(d, f, nsteps):
        calls.append((d["i"], f, nsteps))
        return table[d["i"]]

    monkeypatch.setattr(sweep, "_continued_max_u", fake)
    monkeypatch.setattr(sweep, "batched_state", lambda a, i: ("fp32 state", i))
    return calls, table


def test_classes_in_order(continued):
    calls, table = continued
    doms = [{"i": i} for i in range(9)]
    a = arm([1e-3, INF, 5e-7, 5e-7, 2e-3, 1e-3, INF, 1e-3, 3e-3],
            [100, 200, 300, 300, 4000, 9000, 500, 800, 900])
    ref = arm([1.04e-3, INF, 8e-7, 3e-4, 1e-3, 2e-3, 1e-3, INF, 2e-3],
              [100, 200, 300, 300, 9000, 4000, 500, 800, 900])
    ref["states"] = [None, None, None, None, None, ("fp64 state", 5), None, None, None]
    table[4] = 1.02e-3   # the batched run continued to 9000 steps agrees with 1e-3
    table[5] = 1.2e-3    # the FP64 run continued to 9000 steps is still 2x off
    cls = sweep.classify(doms, a, ref)
    assert cls == ["within_5pct", "diverged_both", "below_resolution", "other_basin", "stopped_early",
                   "unexplained", "unexplained", "unexplained", "unexplained"]
    # the run that stopped first is the one continued, by the step difference
    assert calls == [(4, ("fp32 state", 4), 5000), (5, ("fp64 state", 5), 5000)]
    n = sweep.counts(cls)
    assert sum(n.values()) == len(doms) and n["unexplained"] == 4


def test_tanh_start_divergence_only_for_the_learned_start():
    doms = [{"i": 0}, {"i": 1}]
    warm = arm([1e-3, 1e-3], [100, 100])
    ref = arm([INF, INF], [200000, 200000])
    tanh = arm([INF, 2e-3], [100, 100])
    ref["states"] = [None, None]
    assert sweep.classify(doms, warm, ref, tanh_arm=tanh) == ["tanh_start_diverged", "unexplained"]
    assert sweep.classify(doms, warm, ref) == ["unexplained", "unexplained"]


def test_keep_states_only_for_misses():
    keep = sweep.misses_5pct(arm([1e-3, 1e-3, INF], [1, 1, 1]), arm([1e-3, 2e-3, 1e-3], [1, 1, 1]))
    assert not keep(0, 1.01e-3)
    assert keep(1, 1.01e-3)      # the second arm misses
    assert keep(2, 1e-3)         # the first arm diverged
    assert keep(0, math.inf)


class _FakeBatch:
    """Stands in for lbm.Batch: every domain's outcome is scripted by its "i"."""
    script = {}   # (precision, i) -> (steps, max_u)
    made = []

    def __init__(self, doms, precision=None):
        self.doms, self.precision = doms, precision
        _FakeBatch.made.append(([d["i"] for d in doms], precision))

    def run_to_steady(self, tol, max_steps, k):
        out = [self.script[(self.precision, d["i"])] for d in self.doms]
        return [s for s, _ in out], [{"max_u": u} for _, u in out], True

    def get_f(self, j):
        return ("f", self.precision, self.doms[j]["i"])

    def set_f(self, j, f):
        pass

    def close(self):
        pass

    def schedule_report(self):
        return {}


def test_learned_start_that_diverges_runs_again_from_tanh(monkeypatch):
    from paper_1906_11027_gb300 import lbm, warmstart
    monkeypatch.setattr(lbm, "Batch", _FakeBatch)
    monkeypatch.setattr(warmstart, "batch_warm_init", lambda b, doms, net: 0)
    monkeypatch.setattr(sweep, "_sync", lambda: None)
    _FakeBatch.made = []
    F32, F64 = lbm.LBM_FP32_SHIFTED, lbm.LBM_FP64
    # domain 0 settles from the learned start; domain 1 diverges from it after
    # 100 steps and settles from the tanh start in 6000; domain 2 diverges from both
    _FakeBatch.script = {(F32, 0): (5000, 1e-3), (F32, 1): (100, INF), (F32, 2): (200, INF)}
    first = dict(_FakeBatch.script)
    runs = {"n": 0}

    def run(self, tol, max_steps, k):
        runs["n"] += 1
        if runs["n"] == 2:  # the restart batch of the diverged domains
            self.script = {(F32, 1): (6000, 2e-3), (F32, 2): (300, INF)}
        else:
            self.script = first
        return _FakeBatch.__dict__["_run"](self, tol, max_steps, k)

    monkeypatch.setattr(_FakeBatch, "_run", _FakeBatch.run_to_steady, raising=False)
    monkeypatch.setattr(_FakeBatch, "run_to_steady", run)
    doms = [{"i": i} for i in range(3)]
    arm = sweep.batched(doms, net=object())
    assert [m[0] for m in _FakeBatch.made] == [[0, 1, 2], [1, 2]]
    assert arm["restarted"] == 2
    assert arm["steps"] == [5000, 6100, 500]          # the diverged prefix counts
    assert arm["evolved"] == [5000, 6000, 300]        # the final state's own run
    assert [o["max_u"] for o in arm["obs"]] == [1e-3, 2e-3, INF]
    assert sweep.batched_state(arm, 1) == ("f", F32, 1)
    # from the tanh start nothing is restarted
    _FakeBatch.made, runs["n"] = [], 0
    arm = sweep.batched(doms)
    assert arm["restarted"] == 0 and [m[0] for m in _FakeBatch.made] == [[0, 1, 2]]
