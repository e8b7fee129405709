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


def test_results_alone_equal_results_in_the_mix(ctx):
    reqs = _small_requests(12)
    geoms = [request_problem(r, torch.device("cuda", 0)) for r in reqs]
    fps = [wave.wave_session_footprint(ctx, g[0], g[2], g[4], r["nt"], r["so"]) for g, r in zip(geoms, reqs)]
    budget = int(2.5 * max(fps)) + (64 << 20)
    server = ShotServer(device=0, hbm_budget_bytes=budget, max_resident=5)
    try:
        arrivals = np.sort(inputs.rng(4).uniform(0.0, 0.3, size=len(reqs)))
        stats = server.run(reqs, arrivals)
    finally:
        server.close()
    assert len(stats.results) == len(reqs)
    assert stats.peak_bytes <= budget
    assert stats.max_resident >= 2          # work overlapped on the device
    for r in reqs:
        np.testing.assert_array_equal(stats.results[r["id"]].data, _alone(ctx, r))
    s = stats.summary()
    print("served %d requests: %.1f shots/s, p50 %.3f s, p99 %.3f s, max resident %d"
          % (s["requests"], s["shots_per_s"], s["p50_latency_s"], s["p99_latency_s"], s["max_resident"]))
