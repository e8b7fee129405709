"""CPU tests of the continuous-batching scheduler of ``serve.ShotServer``.

The device calls (context, session footprint, resident sessions) are replaced
by stand-ins that account memory and finish after a set time, so that the host
logic alone is checked: requests are admitted in arrival order while a stream
slot is free and their footprint fits the budget left, a request that waits
for memory is materialised once, several requests are resident at a time, the
budget is never exceeded, every request returns its own result, and a request
larger than the whole budget is refused.  The batched form (one batched
advance of every resident request per tick) keeps the same admission rules,
advances only requests with steps left, and retires each request once its
steps have run.
"""

import time
import types

import numpy as np
import pytest

from paper_1608_08658_gb300 import serve, wave


class FakeContext:
    def __init__(self, budget):
        self.budget = budget
        self.used = 0
        self.peak = 0

    def budget_free(self):
        return self.budget - self.used

    def workspace_bytes(self):
        return self.used


class FakeSession:
    live = []

    def __init__(self, ctx, geom, m, src, q, rec, dt, nt, so, stream=None, graph_chunk=32):
        assert geom.fp <= ctx.budget_free(), "admitted beyond the budget"
        self.ctx, self.geom, self.nt = ctx, geom, nt
        self.steps_left = nt - 1
        ctx.used += geom.fp
        ctx.peak = max(ctx.peak, ctx.used)
        self.t_end = None
        self.stream = stream
        FakeSession.live.append(self)

    def advance(self, steps):
        assert steps == self.nt
        self.t_end = time.perf_counter() + self.geom.duration
        self.steps_left = 0
        return 0

    def done(self):
        return self.t_end is not None and time.perf_counter() >= self.t_end

    def read(self):
        return np.full((self.nt, 2), float(self.geom.req_id), dtype=np.float32)

    def close(self):
        self.ctx.used -= self.geom.fp
        FakeSession.live.remove(self)


def _server(budget, slots, batched=False, tick_steps=3, batch_max_points=0, max_batch=64):
    s = serve.ShotServer.__new__(serve.ShotServer)
    s.device = "cpu"
    s.ctx = FakeContext(budget)
    s.budget = budget
    s.max_resident = slots
    s.batched = batched
    s.tick_steps = tick_steps
    s.batch_max_points = batch_max_points
    s.max_batch = max_batch
    s.streams = [types.SimpleNamespace(cuda_stream=1000 + i) for i in range(slots)]
    s.batch_stream = types.SimpleNamespace(cuda_stream=2000)
    s.setup_stream = types.SimpleNamespace(cuda_stream=2001)
    idle = types.SimpleNamespace(synchronize=lambda: None)
    event = lambda: types.SimpleNamespace(record=lambda stream: None, query=lambda: True)  # noqa: E731
    s.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(current_stream=lambda device: idle, Event=event))
    s.graph_chunk = 32
    return s


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(wave, "Session", FakeSession)
    monkeypatch.setattr(wave, "wave_session_footprint", lambda ctx, geom, src, rec, nt, so: geom.fp)
    FakeSession.live = []
    calls = []

    def problem(req, device):
        calls.append(req["id"])
        geom = types.SimpleNamespace(fp=req["fp"], duration=req["dur"], req_id=req["id"])
        return geom, None, None, None, None, 1.0
    return problem, calls


def _requests(n, seed=5):
    r = np.random.default_rng(seed)
    return [dict(id=i, nt=int(r.integers(3, 9)), so=8, fp=int(r.integers(1, 6)) * 100,
                 dur=float(r.uniform(0.002, 0.012)), ndim=2 if i % 2 == 0 else 3, N=100, nbl=10)
            for i in range(n)]


def test_admission_by_slot_and_footprint(fakes):
    problem, calls = fakes
    reqs = _requests(40)
    arrivals = np.cumsum(np.random.default_rng(6).exponential(0.002, size=len(reqs)))
    srv = _server(budget=1000, slots=4)
    stats = srv.run(reqs, arrivals, problem=problem)
    # every request served once, with its own result
    assert sorted(stats.results) == list(range(len(reqs)))
    for rid, res in stats.results.items():
        assert res.data.shape == (reqs[rid]["nt"], 2) and np.all(res.data == rid)
        assert res.arrival <= res.admitted <= res.finished
    # admitted in arrival order, each materialised once
    order = sorted(stats.results.values(), key=lambda r: r.admitted)
    assert [r.req_id for r in order] == sorted(stats.results, key=lambda i: arrivals[i])
    assert sorted(calls) == list(range(len(reqs)))
    # resident work overlaps, within the slots and the budget
    assert 1 < stats.max_resident <= 4
    assert srv.ctx.peak <= 1000 and srv.ctx.used == 0 and not FakeSession.live


def test_request_waits_for_memory_without_rematerialising(fakes):
    problem, calls = fakes
    reqs = [dict(id=0, nt=4, so=8, fp=700, dur=0.03), dict(id=1, nt=4, so=8, fp=600, dur=0.001)]
    srv = _server(budget=1000, slots=4)
    stats = srv.run(reqs, np.array([0.0, 0.001]), problem=problem)
    assert calls == [0, 1]
    assert stats.results[1].admitted >= stats.results[0].finished - 1e-3
    assert stats.max_resident == 1


def test_request_beyond_the_whole_budget_is_refused(fakes):
    problem, _ = fakes
    srv = _server(budget=500, slots=2)
    with pytest.raises(RuntimeError, match="more than the whole budget"):
        srv.run([dict(id=0, nt=4, so=8, fp=600, dur=0.001)], np.array([0.0]), problem=problem)


def test_batched_ticks(fakes, monkeypatch):
    """Small requests (2D here) advance together by batched ticks, larger ones
    (3D) on stream slots; every request is served once, in arrival order."""
    problem, calls = fakes
    ticks = []
    batched_ids = set()

    def advance(sessions, steps, stream):
        assert sessions and all(x.steps_left > 0 for x in sessions)
        assert len(sessions) <= 3 and stream.value == 2000
        ticks.append(len(sessions))
        for x in sessions:
            batched_ids.add(x.geom.req_id)
            x.steps_left = max(0, x.steps_left - steps)
            if x.steps_left == 0:
                x.t_end = time.perf_counter() + x.geom.duration
    monkeypatch.setattr(wave, "wave_sessions_advance", advance)
    reqs = _requests(30, seed=8)
    arrivals = np.cumsum(np.random.default_rng(9).exponential(0.0003, size=len(reqs)))
    srv = _server(budget=1500, slots=2, batched=True, tick_steps=3, batch_max_points=120 ** 2, max_batch=3)
    stats = srv.run(reqs, arrivals, problem=problem)
    assert sorted(stats.results) == list(range(len(reqs)))
    for rid, res in stats.results.items():
        assert np.all(res.data == rid) and res.arrival <= res.admitted <= res.finished
    order = sorted(stats.results.values(), key=lambda r: r.admitted)
    assert [r.req_id for r in order] == sorted(stats.results, key=lambda i: arrivals[i])
    assert sorted(calls) == list(range(len(reqs)))
    assert batched_ids == {r["id"] for r in reqs if r["ndim"] == 2}   # only the small requests are batched
    assert max(ticks) > 1                                                 # several per batched advance
    assert 1 < stats.max_resident <= 5
    assert srv.ctx.peak <= 1500 and srv.ctx.used == 0 and not FakeSession.live
