"""CPU tests of the gradient's storage planner (``wave_storage_plan_for``, the
same rule ``wave_gradient`` applies with the device's free memory).

The plan keeps a buffer of F snapshot levels (the last F levels of the forward
sweep) and covers the earlier T0 = nt - F levels with segments of k*F levels,
each starting at an exact checkpoint of two FP32 fields.  Checked here against
that specification: what it stores fits the memory given, the segments cover
every level, k is the smallest power of two (<= 64) for which any buffer fits
and F the largest buffer that fits for that k; full storage and a fixed
interval are taken as asked, and a memory too small for anything is refused.
"""

import numpy as np
import pytest

from paper_1608_08658_gb300 import build as libbuild
from paper_1608_08658_gb300 import wave


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return wave.lib()


def _fits(nt, F, k, lb, fb, avail):
    T0 = nt - F
    nseg = -(-T0 // (k * F))
    return F * lb + nseg * 2 * fb <= avail


def _spec(nt, lb, fb, avail):
    """Smallest k in 1, 2, 4 .. 64 for which some buffer fits, and the largest
    such buffer (None when nothing fits)."""
    k = 1
    while k <= 64:
        for F in range(min(avail // lb, nt - 1), 0, -1):
            if _fits(nt, F, k, lb, fb, avail):
                return F, k
        k *= 2
    return None


def test_full_storage_keeps_every_level():
    assert wave.wave_storage_plan_for(1000, 100, 100, 10, checkpoint=False) == (999, 1, 0)


def test_everything_fits_means_no_checkpoint():
    # 999 levels and the conservative two-field allowance of one segment fit
    F, k, nseg = wave.wave_storage_plan_for(1000, 100, 100, 999 * 100 + 200)
    assert (F, k, nseg) == (999, 1, 0)


@pytest.mark.parametrize("seed", range(6))
def test_plan_matches_specification(seed):
    r = np.random.default_rng(seed)
    for _ in range(400):
        nt = int(r.integers(2, 2500))
        fb = int(r.integers(1, 5000))
        lb = fb if r.uniform() < 0.5 else fb // 2 + int(r.integers(1, 10))
        avail = int(r.integers(0, nt * lb * 2 + 10))
        want = _spec(nt, lb, fb, avail)
        if want is None:
            with pytest.raises(wave.WaveError) as e:
                wave.wave_storage_plan_for(nt, lb, fb, avail)
            assert e.value.code == wave.WAVE_ERR_OUT_OF_MEMORY
            continue
        F, k, nseg = wave.wave_storage_plan_for(nt, lb, fb, avail)
        assert (F, k) == want
        T0 = nt - F
        assert F * lb + nseg * 2 * fb <= avail
        # segments of k*F levels cover the levels before the buffer
        assert nseg == (-(-T0 // (k * F)) if T0 > 1 else 0)
        assert nseg * k * F >= T0 - 1


def test_fixed_interval():
    assert wave.wave_storage_plan_for(1000, 100, 100, 0, checkpoint_interval=50) == (50, 1, 19)
    assert wave.wave_storage_plan_for(30, 100, 100, 0, checkpoint_interval=50) == (29, 1, 0)


def test_benchmark_shape():
    """592^3 FP32 levels (0.83 GB) with 250 GB: about 300 stored levels, the
    other ~700 rebuilt from single-part segments."""
    lb = fb = 592 * 592 * 592 * 4
    F, k, nseg = wave.wave_storage_plan_for(1000, lb, fb, 250 * 10 ** 9)
    assert k == 1 and 250 <= F <= 300
    assert nseg == -(-(1000 - F) // F)


def test_bad_arguments():
    for args in [(1, 100, 100, 10 ** 6), (100, 0, 100, 10 ** 6)]:
        with pytest.raises(wave.WaveError) as e:
            wave.wave_storage_plan_for(*args)
        assert e.value.code == wave.WAVE_ERR_INVALID_ARG
    with pytest.raises(wave.WaveError):
        wave.wave_storage_plan_for(100, 100, 100, 10 ** 6, checkpoint_interval=-1)
