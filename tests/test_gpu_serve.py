"""GPU tests of resident sessions and the continuous-batching server.

* A session (graph replays of 32 steps plus a ragged tail, or plain launches)
  returns exactly what wave_forward returns for the same request.
* Requests served in a mix -- staggered arrivals, a slot limit and an HBM
  budget that forces admissions to wait for memory -- return exactly what each
  returns alone, and the workspace never exceeds the budget.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import inputs, wave  # noqa: E402
from paper_1608_08658_gb300.serve import ShotServer, request_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _small_requests(n, seed=3):
    r = inputs.rng(seed)
    reqs = []
    for i in range(n):
        nd = 2 if i % 2 == 0 else 3
        reqs.append(dict(id=i, ndim=nd, N=int(r.integers(100, 220)) if nd == 2 else int(r.integers(36, 70)),
                         h=10.0, nbl=10 if nd == 2 else 8, so=int(r.choice([4, 8, 16])),
                         nt=int(r.integers(90, 260)), n_layers=int(r.integers(3, 9)),
                         n_rec=int(r.integers(20, 120)), model_seed=1000 + i, f0=0.015))
    return reqs


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = wave.Context(0)
    yield c
    c.close()


def _alone(ctx, req):
    geom, m, src, q, rec, dt = request_problem(req, torch.device("cuda", 0))
    return wave.wave_forward(ctx, geom, m, src, q, rec, dt, req["nt"], req["so"]).cpu().numpy()


@pytest.mark.parametrize("chunk", [32, 0])
def test_session_equals_forward(ctx, chunk):
    for req in _small_requests(4, seed=11):
        geom, m, src, q, rec, dt = request_problem(req, torch.device("cuda", 0))
        s = wave.Session(ctx, geom, m, src, q, rec, dt, req["nt"], req["so"], graph_chunk=chunk)
        while s.advance(40) > 0:
            pass
        torch.cuda.synchronize()
        got = s.read()
        assert s.done()
        s.close()
        np.testing.assert_array_equal(got, _alone(ctx, req))


@pytest.mark.parametrize("batched", [False, True])
def test_results_alone_equal_results_in_the_mix(ctx, batched):
    """batched: the 2D requests (up to 60 000 points here) advance together by
    batched launches, the 3D ones on stream slots."""
    reqs = _small_requests(12)
    geoms = [request_problem(r, torch.device("cuda", 0)) for r in reqs]
    fps = [wave.wave_session_footprint(ctx, g[0], g[2], g[4], r["nt"], r["so"]) for g, r in zip(geoms, reqs)]
    budget = int(2.5 * max(fps)) + (64 << 20)
    server = ShotServer(device=0, hbm_budget_bytes=budget, max_resident=5, batched=batched, tick_steps=16,
                        batch_max_points=60_000)
    try:
        # arrivals within 20 ms: requests overlap whatever the kernels' speed
        arrivals = np.sort(inputs.rng(4).uniform(0.0, 0.02, size=len(reqs)))
        stats = server.run(reqs, arrivals)
    finally:
        server.close()
    assert len(stats.results) == len(reqs)
    assert stats.peak_bytes <= budget
    assert stats.max_resident >= 2          # work overlapped on the device
    for r in reqs:
        np.testing.assert_array_equal(stats.results[r["id"]].data, _alone(ctx, r))
    s = stats.summary()
    print("served %d requests%s: %.1f shots/s, p50 %.3f s, p99 %.3f s, max resident %d"
          % (s["requests"], " (small ones batched)" if batched else "", s["shots_per_s"], s["p50_latency_s"],
             s["p99_latency_s"], s["max_resident"]))


def test_batched_advance_equals_forward(ctx):
    """Sessions of mixed dimension and order advanced together by batched
    launches (three of them join after the first call; 23 steps per call, not
    a divisor of any nt) return what wave_forward returns for each alone, bit
    for bit, with far fewer launches than advancing them one by one."""
    reqs = _small_requests(8, seed=21)
    dev = torch.device("cuda", 0)
    batch_stream, setup_stream = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    bs = wave.ctypes.c_void_p(batch_stream.cuda_stream)
    ss = wave.ctypes.c_void_p(setup_stream.cuda_stream)
    sess = []
    for r in reqs:
        geom, m, src, q, rec, dt = request_problem(r, dev)
        torch.cuda.synchronize()
        sess.append(wave.Session(ctx, geom, m, src, q, rec, dt, r["nt"], r["so"], stream=ss, graph_chunk=0))
    ctx.reset_stats()
    wave.wave_sessions_advance(sess[:5], 23, bs)
    while any(s.steps_left > 0 for s in sess):
        wave.wave_sessions_advance([s for s in sess if s.steps_left > 0], 23, bs)
    launches = ctx.kernel_stats(-1)[0]
    batch_stream.synchronize()
    for s, r in zip(sess, reqs):
        assert s.done()
        got = s.read()
        s.close()
        np.testing.assert_array_equal(got, _alone(ctx, r))
    one_by_one = sum(3 * (r["nt"] - 1) for r in reqs)
    print("batched advance: %d launches for %d requests (%d one by one)" % (launches, len(reqs), one_by_one))
    assert launches < one_by_one / 2


def test_batched_advance_rejects_foreign_sessions(ctx):
    reqs = _small_requests(2, seed=5)
    dev = torch.device("cuda", 0)
    with wave.Context(0) as other:
        g0, m0, s0, q0, r0, dt0 = request_problem(reqs[0], dev)
        g1, m1, s1, q1, r1, dt1 = request_problem(reqs[1], dev)
        a = wave.Session(ctx, g0, m0, s0, q0, r0, dt0, reqs[0]["nt"], reqs[0]["so"], graph_chunk=0)
        b = wave.Session(other, g1, m1, s1, q1, r1, dt1, reqs[1]["nt"], reqs[1]["so"], graph_chunk=0)
        with pytest.raises(wave.WaveError) as e:
            wave.wave_sessions_advance([a, b], 5)
        assert e.value.code == wave.WAVE_ERR_INVALID_ARG
        a.close()
        b.close()


def test_concurrent_sessions_enqueued_in_full(ctx):
    """Two resident 3D sessions of different grids and orders on their own
    streams, both enqueued in full (captured chunks and the ragged tail) before
    either is read, the shorter one finishing while the longer one's launches
    are still queued: nothing one session's launches read is written by the
    other's, and each result equals wave_forward alone, bit for bit."""
    dev = torch.device("cuda", 0)
    reqs = [dict(id=0, ndim=3, N=66, h=10.0, nbl=8, so=8, nt=250, n_layers=5, n_rec=80, model_seed=7, f0=0.015),
            dict(id=1, ndim=3, N=41, h=10.0, nbl=8, so=16, nt=60, n_layers=4, n_rec=50, model_seed=8, f0=0.015)]
    streams = [torch.cuda.Stream(dev) for _ in reqs]
    sess = []
    for r, st in zip(reqs, streams):
        geom, m, src, q, rec, dt = request_problem(r, dev)
        assert (r["nt"] - 1) % 32 != 0  # a ragged tail after the captured chunks
        torch.cuda.synchronize()
        sess.append(wave.Session(ctx, geom, m, src, q, rec, dt, r["nt"], r["so"],
                                 stream=wave.ctypes.c_void_p(st.cuda_stream), graph_chunk=32))
    for s, r in zip(sess, reqs):
        s.advance(r["nt"])
    torch.cuda.synchronize()
    for s, r in zip(sess, reqs):
        got = s.read()
        s.close()
        np.testing.assert_array_equal(got, _alone(ctx, r))
