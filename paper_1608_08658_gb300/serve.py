"""Continuous-batching server for shot-modelling requests.

Requests (forward modelling of one shot: geometry, layered model, space
order, nt) arrive over time.  A single host scheduler thread:

  * admits waiting requests in arrival order while a stream slot is free and
    the request's device footprint (wave_session_footprint) fits the HBM
    budget left in the context (wave_context_budget_free);
  * creates a resident session on the slot's CUDA stream and enqueues all of
    its time steps at once -- whole chunks as replays of the session's
    captured CUDA graph -- so that the GPU interleaves the kernels of every
    resident request;
  * polls completion, copies the receiver data back, destroys the session
    (freeing its memory for the next admissions) and records the latency.

With ``batched=True`` the small requests (at most ``batch_max_points``
computational points, whose steps take a few microseconds and are bound by
launch overhead) go through wave_sessions_advance instead: every scheduler
tick enqueues ``tick_steps`` steps of every resident small request on one
stream, one stencil launch per step for all of them of the same space order,
dimension and spacing variant, and one injection and one receiver launch per
step; small requests join and leave between ticks.  Larger requests keep
their own stream and graph replays, so their work still overlaps that of the
batch.  Batched sessions are set up on a stream of their own, so an admission
does not wait for the ticks in flight.

Every step of every request runs in the CUDA library; this module only
schedules.  Results are identical to running each request alone.
"""

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs, wave


@dataclass
class Result:
    req_id: int
    data: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class ServeStats:
    results: dict = field(default_factory=dict)
    wall: float = 0.0
    max_resident: int = 0
    peak_bytes: int = 0

    def summary(self):
        lat = np.array([r.latency for r in self.results.values()])
        n = len(lat)
        return {"requests": n, "shots_per_s": n / self.wall if self.wall > 0 else None,
                "p50_latency_s": float(np.percentile(lat, 50)) if n else None,
                "p99_latency_s": float(np.percentile(lat, 99)) if n else None,
                "mean_latency_s": float(lat.mean()) if n else None, "wall_s": self.wall,
                "max_resident": self.max_resident, "peak_workspace_bytes": self.peak_bytes}


def request_problem(req, device):
    """Materialise a request from ``inputs.serving_requests``: geometry, model
    (broadcast on the device from its 1D profile), points, Ricker traces, dt."""
    import torch
    N, h, nd = req["N"], req["h"], req["ndim"]
    shape = (N,) * nd
    geom = wave.Geometry(shape=shape, spacing=(h,) * nd, nbl=req["nbl"], sponge_vref=4.5)
    v = inputs.layered_profile(N, h, req["n_layers"], seed=req["model_seed"])
    m1 = torch.from_numpy((1.0 / v ** 2).astype(np.float32)).to(device)
    m = m1.view((N,) + (1,) * (nd - 1)).expand((N,) * nd).contiguous()
    vmax = float(v.max())
    dt = 0.4 * wave.wave_dt_max((h,) * nd, req["so"], vmax)
    src, rec = inputs.request_points(req)
    q = wave.wave_ricker(req["nt"], dt, req["f0"]).reshape(-1, 1)
    return geom, m, src, q, rec, dt


class ShotServer:
    def __init__(self, device=0, hbm_budget_bytes=0, max_resident=32, graph_chunk=32, batched=False,
                 tick_steps=32, batch_max_points=2_000_000, max_batch=64):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.ctx = wave.Context(device, hbm_budget_bytes)
        self.budget = int(hbm_budget_bytes)
        self.max_resident = max_resident
        self.batched = batched
        self.tick_steps = tick_steps
        self.batch_max_points = batch_max_points
        self.max_batch = max_batch
        if batched:
            # the small, latency-bound requests of the batch go first when the
            # GPU also runs the large ones
            self.batch_stream = torch.cuda.Stream(self.device, priority=-1)
            self.setup_stream = torch.cuda.Stream(self.device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_resident)]
        self.graph_chunk = graph_chunk

    def close(self):
        self.ctx.close()

    def run(self, requests, arrivals, problem=request_problem):
        """Serve ``requests`` arriving at ``arrivals`` (seconds from start)."""
        if self.batched:
            return self._run_batched(requests, arrivals, problem)
        order = np.argsort(arrivals, kind="stable")
        pending = collections.deque((requests[i], float(arrivals[i])) for i in order)
        waiting = collections.deque()
        free_slots = list(range(len(self.streams)))
        active = []
        stats = ServeStats()
        head = None  # (request id, materialised problem, footprint) of the first waiting request
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0][1] <= now:
                waiting.append(pending.popleft())
            progressed = False
            # admission in arrival order by slot and footprint; a request that
            # waits for memory is materialised once, not at every poll
            while waiting and free_slots:
                req, arr = waiting[0]
                if head is None or head[0] != req["id"]:
                    prob = problem(req, self.device)
                    geom, src, rec = prob[0], prob[2], prob[4]
                    head = (req["id"], prob, wave.wave_session_footprint(self.ctx, geom, src, rec, req["nt"],
                                                                         req["so"]))
                _, (geom, m, src, q, rec, dt), fp = head
                if self.budget and fp > self.ctx.budget_free():
                    if not active:
                        raise RuntimeError("request %d needs %d bytes, more than the whole budget" % (req["id"], fp))
                    break
                waiting.popleft()
                head = None
                slot = free_slots.pop()
                stream = self.streams[slot]
                sess = wave.Session(self.ctx, geom, m, src, q, rec, dt, req["nt"], req["so"],
                                    stream=wave.ctypes.c_void_p(stream.cuda_stream), graph_chunk=self.graph_chunk)
                sess.advance(req["nt"])
                active.append((req, arr, time.perf_counter() - t0, sess, slot))
                stats.max_resident = max(stats.max_resident, len(active))
                stats.peak_bytes = max(stats.peak_bytes, self.ctx.workspace_bytes())
                progressed = True
            # completion
            still = []
            for req, arr, adm, sess, slot in active:
                if sess.done():
                    data = sess.read()
                    sess.close()
                    free_slots.append(slot)
                    stats.results[req["id"]] = Result(req["id"], data, arr, adm, time.perf_counter() - t0)
                    progressed = True
                else:
                    still.append((req, arr, adm, sess, slot))
            active = still
            if not progressed:
                nxt = pending[0][1] - (time.perf_counter() - t0) if pending and not waiting and not active else 0
                time.sleep(min(max(nxt, 0.0), 0.01) if nxt > 0 else 0.0002)
        stats.wall = time.perf_counter() - t0
        return stats


    def _admit(self, waiting, head, problem, n_active):
        """Materialise the first waiting request (once) and return
        (head, request, arrival, problem, fits) for it."""
        req, arr = waiting[0]
        if head is None or head[0] != req["id"]:
            prob = problem(req, self.device)
            geom, src, rec = prob[0], prob[2], prob[4]
            head = (req["id"], prob, wave.wave_session_footprint(self.ctx, geom, src, rec, req["nt"], req["so"]))
        fp = head[2]
        fits = not self.budget or fp <= self.ctx.budget_free()
        if not fits and n_active == 0:
            raise RuntimeError("request %d needs %d bytes, more than the whole budget" % (req["id"], fp))
        return head, req, arr, head[1], fits

    def _run_batched(self, requests, arrivals, problem):
        """Continuous batching by ticks for the small requests (one batched
        advance of all of them per tick) beside stream slots with graph
        replays for the larger ones; admission in arrival order by slot or
        batch place and by footprint."""
        order = np.argsort(arrivals, kind="stable")
        pending = collections.deque((requests[i], float(arrivals[i])) for i in order)
        waiting = collections.deque()
        free_slots = list(range(len(self.streams)))
        active = []  # (request, arrival, admitted, session, slot or None when batched)
        stats = ServeStats()
        head = None
        bs = wave.ctypes.c_void_p(self.batch_stream.cuda_stream)
        ss = wave.ctypes.c_void_p(self.setup_stream.cuda_stream)
        ticks = collections.deque()  # completion events of the ticks in flight
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0][1] <= now:
                waiting.append(pending.popleft())
            progressed = False
            while waiting:
                req, _ = waiting[0]
                small = request_points(req) <= self.batch_max_points
                n_batch = sum(1 for a in active if a[4] is None)
                if (small and n_batch >= self.max_batch) or (not small and not free_slots):
                    break
                head, req, arr, (geom, m, src, q, rec, dt), fits = self._admit(waiting, head, problem, len(active))
                if not fits:
                    break
                waiting.popleft()
                head = None
                if small:
                    self.torch.cuda.current_stream(self.device).synchronize()  # the problem's tensors are ready
                    sess = wave.Session(self.ctx, geom, m, src, q, rec, dt, req["nt"], req["so"], stream=ss,
                                        graph_chunk=0)
                    slot = None
                else:
                    slot = free_slots.pop()
                    stream = self.streams[slot]
                    sess = wave.Session(self.ctx, geom, m, src, q, rec, dt, req["nt"], req["so"],
                                        stream=wave.ctypes.c_void_p(stream.cuda_stream),
                                        graph_chunk=self.graph_chunk)
                    sess.advance(req["nt"])
                active.append((req, arr, time.perf_counter() - t0, sess, slot))
                stats.max_resident = max(stats.max_resident, len(active))
                stats.peak_bytes = max(stats.peak_bytes, self.ctx.workspace_bytes())
                progressed = True
            # a new tick is enqueued while at most one earlier tick is in flight,
            # so the scheduler never waits for the GPU
            while ticks and ticks[0].query():
                ticks.popleft()
            running = [a[3] for a in active if a[4] is None and a[3].steps_left > 0]
            if running and len(ticks) < 2:
                wave.wave_sessions_advance(running, self.tick_steps, bs)
                ev = self.torch.cuda.Event()
                ev.record(self.batch_stream)
                ticks.append(ev)
                progressed = True
            still = []
            for req, arr, adm, sess, slot in active:
                if sess.steps_left == 0 and sess.done():
                    data = sess.read()
                    sess.close()
                    if slot is not None:
                        free_slots.append(slot)
                    stats.results[req["id"]] = Result(req["id"], data, arr, adm, time.perf_counter() - t0)
                    progressed = True
                else:
                    still.append((req, arr, adm, sess, slot))
            active = still
            if not progressed:
                nxt = pending[0][1] - (time.perf_counter() - t0) if pending and not waiting and not active else 0
                time.sleep(min(max(nxt, 0.0), 0.01) if nxt > 0 else 0.0002)
        stats.wall = time.perf_counter() - t0
        return stats


def request_points(req):
    """Computational points of a request (physical grid plus the layer)."""
    return (req["N"] + 2 * req["nbl"]) ** req["ndim"]


def poisson_arrivals(n, rate, seed=99):
    """Arrival times of a Poisson process of the given rate (requests/s)."""
    r = inputs.rng(seed + 7)
    return np.cumsum(r.exponential(1.0 / rate, size=n)) - 0.0
