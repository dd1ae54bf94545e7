"""Host logic of the plan tuner (``engine.tune_plan``) with the plans faked:
the fastest candidate whose calibrated error meets the bar is kept open, the
others are closed, a candidate with no measured error (-1) or above the bar
is never kept, and no candidate within the bar is an error."""
import types

import numpy as np
import pytest

from paper_2406_18889_gb300 import engine as E


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = 0.0

    def record(self, stream=None):
        self.t = _FakeTorch.clock

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeTorch:
    clock = 0.0
    complex128 = "complex128"

    class cuda:
        Event = _FakeEvent

        @staticmethod
        def current_stream():
            return None

        @staticmethod
        def synchronize():
            pass

    @staticmethod
    def empty(shape, dtype=None, device=None):
        return np.zeros(shape)


def _fake_plan_class(table, log):
    class FakePlan:
        def __init__(self, tn, tree, prec="c64", flags=0, max_slice_batch=64, hilo_tol=0.0, **kw):
            self.prec, self.max_slice_batch = prec, max_slice_batch
            self.ms, self.err, self.nh = table[(prec, max_slice_batch)]
            self.G, self.J = 1, 1
            self.closed = False
            log.append(self)

        def autotune(self, ids, reps=3):
            return None

        def contract(self, ids, out=None):
            _FakeTorch.clock += self.ms
            return out

        def precision(self):
            return dict(rel_l2_chosen=self.err, rel_l2_none=self.err, n_tc_steps=4, n_hilo_steps=self.nh)

        def close(self):
            self.closed = True
    return FakePlan


def _run(monkeypatch, table, **kw):
    log = []
    monkeypatch.setattr(E, "Plan", _fake_plan_class(table, log))
    monkeypatch.setattr(E, "_torch", lambda: _FakeTorch)
    tree = types.SimpleNamespace(sliced_edges=[0, 1, 2])
    plan, rows = E.tune_plan(None, tree, tol=3e-3, precs=("fp16", "bf16"), batches=(4, 8), reps=2, **kw)
    return plan, rows, log


def test_keeps_the_fastest_within_the_bar(monkeypatch):
    # (prec, batch) -> (ms per call, calibrated error, split steps)
    table = {("fp16", 4): (2.0, 1e-3, 0), ("fp16", 8): (1.5, 1e-3, 0),
             ("bf16", 4): (1.0, 5e-3, 0),   # fastest, but above the bar
             ("bf16", 8): (1.2, -1.0, 2)}   # not measured: never kept
    plan, rows, log = _run(monkeypatch, table)
    assert (plan.prec, plan.max_slice_batch) == ("fp16", 8) and not plan.closed
    assert all(p.closed for p in log if p is not plan)
    assert [r["chosen"] for r in rows] == [False, True, False, False]
    # 8 slices per call, 2 timed calls of 1.5 ms
    assert rows[1]["slices_per_s"] == pytest.approx(8 * 2 / 3e-3)


def test_no_candidate_within_the_bar_is_an_error(monkeypatch):
    table = {(p, b): (1.0, 1e-2, 0) for p in ("fp16", "bf16") for b in (4, 8)}
    with pytest.raises(ValueError):
        _run(monkeypatch, table)
