"""Host logic of the continuous-batching server (paper_1512_01977_gb300.serve)
with the engine replaced by a counting fake: FIFO admission under the
footprint budget, ticks that end at the next completion, exact step counts,
retirement of a failing request and of an unphysical initial state, and the
one-at-a-time baseline.  No GPU."""
import types

import pytest

from paper_1512_01977_gb300 import serve


class _Err(Exception):
    def __init__(self, code, where=""):
        super().__init__(where)
        self.code = code


class _Solver:
    def __init__(self, req):
        self.req = req
        self.steps = 0
        self.fail_at = req.get("fail_at")
        self.closed = False

    def init(self, *fields, physical=False):
        assert physical  # served requests start at rest
        if self.req.get("bad_init"):
            raise _Err(-4, "init")
        return self

    def step(self, n):
        self.steps += n
        if self.fail_at is not None and self.steps >= self.fail_at:
            raise _Err(-4, "step")

    def mass(self):
        return float(self.req["id"]), 0.0

    def close(self):
        self.closed = True


class _Batch:
    log = []
    ticks_all = []

    def __init__(self, solvers):
        self.solvers = list(solvers)
        _Batch.log.append([s.req["id"] for s in self.solvers])
        self.ticks = []

    def step_async(self, k):
        self.ticks.append(k)
        _Batch.ticks_all.append(k)
        for s in self.solvers:
            s.steps += k

    def sync(self):
        return 0

    def status(self):
        return [-4 if s.fail_at is not None and s.steps >= s.fail_at else 0 for s in self.solvers]

    def autotune(self, trials=3):
        return 96, 0

    def close(self):
        pass


def _fake_lbm():
    return types.SimpleNamespace(OK=0, ERR_UNPHYSICAL=-4, LbmError=_Err, Batch=_Batch,
                                 lbm_axi_footprint=lambda nz, nr, prec: nz * nr * 100)


@pytest.fixture
def fake(monkeypatch):
    made = {}

    def make_solver(req, precision=32, stream=None):
        s = _Solver(req)
        made[req["id"]] = s
        return s, ()

    monkeypatch.setattr(serve, "lbm", _fake_lbm())
    monkeypatch.setattr(serve, "make_solver", make_solver)
    _Batch.log = []
    _Batch.ticks_all = []
    t = [0.0]

    def clock():
        t[0] += 1e-3
        return t[0]

    return made, clock


def _reqs():
    sizes = [(64, 32, 300), (128, 64, 100), (32, 32, 700), (96, 48, 250), (64, 64, 50), (40, 40, 400)]
    return [dict(id=i, t_arrive=0.004 * i, nz=nz, nr=nr, steps=st, kind="droplet", eos="cs", T_over_Tc=0.8)
            for i, (nz, nr, st) in enumerate(sizes)]


def test_every_request_runs_exactly_its_steps_in_arrival_order(fake):
    made, clock = fake
    reqs = _reqs()
    res, st = serve.serve(reqs, budget_bytes=1 << 40, max_tick_steps=120, clock=clock)
    assert st["requests"] == st["completed"] == len(reqs) and st["failed"] == 0
    by_id = {r.id: r for r in res}
    for q in reqs:
        assert made[q["id"]].steps == q["steps"] and made[q["id"]].closed
        r = by_id[q["id"]]
        assert r.t_arrive <= r.t_start <= r.t_done and r.latency >= 0
        assert r.mass_rweighted == float(q["id"])
    starts = [by_id[q["id"]].t_start for q in sorted(reqs, key=lambda q: q["t_arrive"])]
    assert starts == sorted(starts)
    # a tick never runs beyond max_tick_steps; nor past the next completion (the
    # exact step counts above would break)
    assert max(_Batch.ticks_all) <= 120 and st["ticks"] == len(_Batch.ticks_all)


def test_budget_bounds_the_resident_set(fake):
    made, clock = fake
    reqs = _reqs()
    fp = {q["id"]: q["nz"] * q["nr"] * 100 for q in reqs}
    budget = 2 * max(fp.values())
    serve.serve(reqs, budget_bytes=budget, max_tick_steps=1000, clock=clock)
    for members in _Batch.log:
        assert sum(fp[i] for i in members) <= budget or len(members) == 1


def test_failing_request_and_bad_initial_state_are_retired(fake):
    made, clock = fake
    reqs = _reqs()
    reqs[1]["fail_at"] = 30
    reqs[4]["bad_init"] = True
    res, st = serve.serve(reqs, budget_bytes=1 << 40, max_tick_steps=64, clock=clock)
    by_id = {r.id: r for r in res}
    assert by_id[1].status == -4 and by_id[4].status == -4
    assert by_id[4].t_start == by_id[4].t_done  # retired at admission, never stepped
    assert made[4].steps == 0
    assert st["failed"] == 2 and st["completed"] == len(reqs) - 2
    for q in reqs:
        if q["id"] not in (1, 4):
            assert by_id[q["id"]].status == 0 and made[q["id"]].steps == q["steps"]


def test_one_at_a_time_baseline(fake):
    made, clock = fake
    reqs = _reqs()
    reqs[2]["fail_at"] = 10
    res, st = serve.serve_sequential(reqs, clock=clock)
    assert [r.id for r in res] == [q["id"] for q in sorted(reqs, key=lambda q: q["t_arrive"])]
    assert st["failed"] == 1 and {r.id for r in res if r.status != 0} == {2}
    assert all(made[q["id"]].closed for q in reqs)
