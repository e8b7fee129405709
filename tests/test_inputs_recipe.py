"""CPU checks that the seeded input generators follow the stated workload
recipe: layer velocities and interfaces, the size, mean and correlation length
of the smoothed random perturbation, receiver jitter bounds, the served-request
mix, the FWI anomalies and the salt body.  Generators are deterministic in
their seed."""

import numpy as np
import pytest

from paper_1608_08658_gb300 import inputs


def test_two_layer_model_with_correlated_perturbation():
    shape, h = (64, 64, 64), (10.0, 10.0, 10.0)
    v0 = inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.0)
    z = np.arange(64) * 10.0
    top = z < 0.5 * 63 * 10.0
    assert np.all(v0[top] == 1.5) and np.all(v0[~top] == 2.5)
    v = inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.05, corr_len=50.0, seed=7)
    g = (v / v0 - 1.0) / 0.05
    assert abs(g.mean()) < 1e-6 and abs(g.std() - 1.0) < 1e-6
    # Gaussian smoothing of white noise with a kernel of std s points gives the
    # autocorrelation exp(-lag^2 / (4 s^2)); s = 50 m / 10 m = 5 points
    for lag in (2, 5, 10):
        rho = np.mean(g * np.roll(g, lag, axis=2))
        assert abs(rho - np.exp(-lag ** 2 / 100.0)) < 0.06, (lag, rho)
    np.testing.assert_array_equal(v, inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.05, seed=7))


def test_jittered_line_receivers():
    rec = inputs.line_receivers_jittered(101, 0.0, 10.0, 20.0, 10.0, (1000.0, 1000.0), seed=1234)
    nominal = np.stack([10.0 * np.arange(101), np.full(101, 20.0)], axis=1)
    d = rec.astype(np.float64) - nominal
    assert np.all(d >= -5.0 - 1e-4) and np.all(d < 5.0 + 1e-4)
    assert np.all(rec >= 0.0) and np.all(rec <= 1000.0)
    assert np.abs(d).max() > 4.0          # the jitter is not degenerate


def test_layered_profile():
    for seed in range(20):
        n_layers = 3 + seed % 6
        v = inputs.layered_profile(300, 10.0, n_layers, 1.5, 4.5, seed=seed)
        # the top layer starts at v_min; every layer is then scaled by 1 +- 5 % and clipped
        assert v.min() >= 1.5 and v.max() <= 4.5 and 1.5 <= v[0] <= 1.5 * 1.05
        assert len(np.unique(v)) <= n_layers
        steps = np.flatnonzero(np.diff(v))
        assert np.all((steps * 10.0 >= 0.05 * 2990.0 - 10.0) & (steps * 10.0 <= 0.95 * 2990.0))


def test_served_request_mix():
    reqs = inputs.serving_requests(2000, seed=99)
    nd = np.array([r["ndim"] for r in reqs])
    assert 0.45 < np.mean(nd == 2) < 0.55
    for r in reqs:
        lo, hi = (201, 1001) if r["ndim"] == 2 else (128, 320)
        assert lo <= r["N"] <= hi and r["so"] in (4, 8, 16) and 500 <= r["nt"] <= 2000
        assert 3 <= r["n_layers"] <= 8 and 100 <= r["n_rec"] <= 1000
        assert r["nbl"] == (20 if r["ndim"] == 2 else 40) and r["f0"] == 0.010
        src, rec = inputs.request_points(r)
        ext = (r["N"] - 1) * r["h"]
        assert len(rec) >= r["n_rec"] and np.all(rec[:, :-1] <= ext) and np.all(rec[:, -1] == 20.0)
        assert src.shape == (1, r["ndim"])
    assert set(r["so"] for r in reqs) == {4, 8, 16}


def test_fwi_models():
    shape, h = (48, 40, 64), (12.5, 12.5, 12.5)
    v0, vt = inputs.gradient_models(shape, h, seed=11)
    z = np.arange(64) * 12.5
    np.testing.assert_allclose(v0[:, 0, 0], 1.5 + 0.6 * z / 1000.0)
    dv = vt - v0
    # three blobs of +-0.2 km/s; where two of one sign overlap their sum is larger
    assert 0.1 < np.abs(dv).max() <= 3 * 0.2


def test_salt_body_volume():
    shape, h = (200, 160, 120), (25.0, 25.0, 25.0)
    v = inputs.layered_salt_velocity(shape, h, semi_axes_m=(1500.0, 1000.0, 600.0))
    salt = np.count_nonzero(v == np.float32(4.5)) * 25.0 ** 3
    # the ellipsoid 4/3 pi a b c; layers may also reach 4.5 km/s only at the bottom
    vol = 4.0 / 3.0 * np.pi * 1500.0 * 1000.0 * 600.0
    assert 0.9 * vol < salt < 1.25 * vol


@pytest.mark.parametrize("seed", [0, 3])
def test_generators_are_deterministic(seed):
    a = inputs.random_points(10, (30, 20, 10), (10.0, 10.0, 10.0), seed)
    b = inputs.random_points(10, (30, 20, 10), (10.0, 10.0, 10.0), seed)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(inputs.random_traces(5, 3, seed), inputs.random_traces(5, 3, seed))


def test_large_starting_model_is_the_smoothed_layers_without_salt():
    shape, h = (40, 30, 600), (10.0, 10.0, 10.0)
    vt = inputs.layered_salt_velocity(shape, h)
    v0 = inputs.layered_starting_velocity(shape, h)
    prof = inputs.layered_profile(600, 10.0, 8, 1.5, 4.5, seed=5)
    assert v0.shape == vt.shape and v0.dtype == np.float32
    assert np.all(v0 == v0[:, :1, :1])                    # flat layers only: no salt body
    assert np.any(vt == 4.5) and not np.any(v0 > prof.max() + 1e-6)
    # far (> 4 sigma) from every interface the smoothing leaves the layer value
    cuts = np.nonzero(np.diff(prof))[0] + 1
    far = np.array([np.all(np.abs(k - cuts) > 61) for k in range(600)])
    np.testing.assert_allclose(v0[far, 0, 0], prof[far], rtol=1e-6)
    # at an interface the starting model lies strictly between the two layers, and it is monotone
    for k in cuts:
        lo, hi = sorted((prof[k - 1], prof[k]))
        assert lo < v0[k, 0, 0] < hi
