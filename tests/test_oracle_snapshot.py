"""Pins of the oracle's 16-bit snapshot storage (``oracle.snapshot``) and of the
gradient that reads it, against things other than the oracle itself: NumPy's
IEEE half conversion and torch's bfloat16 conversion (both round to nearest,
ties to even), the scale's defining interval, slab boundaries, idempotence,
the rounding error bound, and the plumbing of the rounded levels into Eq. 3."""

import numpy as np
import pytest

import oracle
from oracle import snapshot


def _values(seed, n=200000):
    r = np.random.default_rng(seed)
    mag = np.ldexp(r.uniform(1.0, 2.0, n), r.integers(-30, 16, n))
    return np.where(r.uniform(size=n) < 0.5, -mag, mag)


def test_fp16_rounding_equals_numpy_half():
    x = _values(1)
    x = x[np.abs(x) < 65504.0]
    # exact ties between two half values, and the subnormal range
    ties = (np.arange(1, 2048) + 0.5) * 2.0 ** -10
    sub = np.arange(0, 2048) * 2.0 ** -25
    for v in (x, ties, -ties, sub):
        np.testing.assert_array_equal(snapshot.round_to_format(v, "fp16"), v.astype(np.float16).astype(np.float64))


def test_bf16_rounding_equals_torch_bfloat16():
    torch = pytest.importorskip("torch")
    x = _values(2).astype(np.float32)
    ties = ((np.arange(1, 256) + 0.5) * 2.0 ** -7).astype(np.float32)    # exact ties of 8-bit significands
    for v in (x, ties, -ties):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(snapshot.round_to_format(v.astype(np.float64), "bf16"), ref)


@pytest.mark.parametrize("fmt,p", [("bf16", 8), ("fp16", 11)])
def test_rounding_error_bound(fmt, p):
    x = _values(3)
    x = x[(np.abs(x) >= 2.0 ** -14) & (np.abs(x) < 32768.0)]       # normal range of both formats
    err = np.abs(snapshot.round_to_format(x, fmt) - x)
    assert np.all(err <= 2.0 ** -p * np.abs(x))
    assert err.max() > 0.4 * 2.0 ** -p * np.abs(x[np.argmax(err / np.abs(x))])   # the bound is reached


def test_slab_scales_definition():
    r = np.random.default_rng(4)
    level = r.standard_normal((3, 7, 150)) * np.ldexp(1.0, r.integers(-20, 20, (3, 1, 1)))
    level[1, 2:4, 64:128] = 0.0                       # one all-zero slab (plane 1, slab (1, 1))
    s = snapshot.slab_scales(level)
    assert s.shape == (3, 4, 3)                        # ceil(7/2) slabs along axis 1, ceil(150/64) along x
    assert s[1, 1, 1] == 1.0
    for z in range(3):
        for sy in range(4):
            for sx in range(3):
                blk = level[z, 2 * sy:2 * sy + 2, 64 * sx:64 * sx + 64]
                amax = np.abs(blk).max()
                if amax == 0:
                    continue
                m, _ = np.frexp(s[z, sy, sx])
                assert m == 0.5                        # a power of two
                assert 2.0 ** 14 <= amax / s[z, sy, sx] < 2.0 ** 15
    # a value changes only its own slab's scale
    bumped = level.copy()
    bumped[2, 5, 130] = 1e6
    changed = np.argwhere(snapshot.slab_scales(bumped) != s)
    assert changed.tolist() == [[2, 2, 2]]


def test_slabs_of_a_2d_level_run_along_depth():
    level = np.zeros((5, 70))                          # [nz][nx]: axis 1 of the slabs is depth
    level[3, 66] = 1.0
    s = snapshot.slab_scales(level)
    assert s.shape == (1, 3, 2)
    assert s[0, 1, 1] == 2.0 ** -14 and np.count_nonzero(s != 1.0) == 1


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_round_level_idempotent_and_close(fmt):
    r = np.random.default_rng(5)
    level = r.standard_normal((4, 9, 131)) * np.exp(r.uniform(-8, 8, (4, 9, 1)))
    once = snapshot.round_level(level, fmt)
    np.testing.assert_array_equal(snapshot.round_level(once, fmt), once)
    p = snapshot.FORMATS[fmt][0]
    s_pt = np.repeat(np.repeat(snapshot.slab_scales(level), 2, axis=1), 64, axis=2)[:, :9, :131]
    # error at most half a quantum of the value's binade, and never above half a quantum at 2^15 s
    assert np.all(np.abs(once - level) <= np.maximum(2.0 ** -p * np.abs(level), 2.0 ** (-14 - p) * s_pt))
    assert np.all(np.abs(once - level) <= 2.0 ** (15 - p) * s_pt)
    # an all-zero level stays zero
    assert not np.any(snapshot.round_level(np.zeros((2, 3, 5)), fmt))


def _small_case():
    og = oracle.model.Geometry(shape=(14, 11), spacing=(10.0, 10.0), nbl=3, sponge_vref=2.0)
    r = np.random.default_rng(6)
    m = (1.0 / (1.5 + 0.5 * r.uniform(size=og.phys_array_shape)) ** 2)
    dt = 0.4 * oracle.model.dt_max(4, og.spacing, 2.0)
    nt = 25
    q = oracle.model.ricker(nt, dt, 0.02)[:, None]
    src = np.array([[60.0, 40.0]])
    rec = np.array([[20.0, 10.0], [100.0, 90.0], [35.0, 55.0]])
    d_obs = oracle.wave.forward(og, m * 1.03, dt, nt, 4, q, src, rec).d
    return og, m, dt, nt, q, src, rec, d_obs


def test_gradient_reads_every_stored_level_through_the_rounding(monkeypatch):
    og, m, dt, nt, q, src, rec, d_obs = _small_case()
    plain, phi = oracle.wave.gradient(og, m, dt, nt, 4, q, src, rec, d_obs)
    seen = []

    def identity(u, fmt):
        seen.append(fmt)
        return u
    monkeypatch.setattr(oracle.wave, "round_level", identity)
    g_id, phi_id = oracle.wave.gradient(og, m, dt, nt, 4, q, src, rec, d_obs, snapshot_rounding="bf16")
    assert seen == ["bf16"] * (nt - 1)                  # levels u^1 .. u^{nt-1}
    np.testing.assert_array_equal(g_id, plain)
    assert phi_id == phi
    monkeypatch.setattr(oracle.wave, "round_level", lambda u, fmt: np.zeros_like(u))
    g0, _ = oracle.wave.gradient(og, m, dt, nt, 4, q, src, rec, d_obs, snapshot_rounding="fp16")
    assert not np.any(g0)


def test_gradient_with_rounded_levels_moves_by_the_format_precision():
    og, m, dt, nt, q, src, rec, d_obs = _small_case()
    plain, _ = oracle.wave.gradient(og, m, dt, nt, 4, q, src, rec, d_obs)
    for fmt, lo, hi in (("fp16", 1e-6, 1e-3), ("bf16", 1e-4, 1e-2)):
        g, _ = oracle.wave.gradient(og, m, dt, nt, 4, q, src, rec, d_obs, snapshot_rounding=fmt)
        e = np.linalg.norm(g - plain) / np.linalg.norm(plain)
        assert lo < e < hi, (fmt, e)
