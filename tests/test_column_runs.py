"""Host-only checks of the column-segment planner of the plain 3D step
(`wave_column_runs_for`, no GPU needed): the runs cover the tile-major plane
sequence exactly once, in order, one per CTA at most per resident slot; their
costs (planes plus one queue fill of 4 + R plane times per column segment)
are balanced, so runs that cross a column are shorter; large grids keep the
z chunks unless forced; bad arguments are rejected."""

import numpy as np
import pytest

from paper_1608_08658_gb300 import wave


def _segments(runs, nz):
    """Column segments of each run."""
    out = []
    for a, b in zip(runs[:-1], runs[1:]):
        out.append(int((b - 1) // nz - a // nz + 1))
    return np.array(out)


def _costs(runs, nz, R):
    return np.diff(runs) + (4 + R) * _segments(runs, nz)


def _check_cover(runs, total, slots):
    assert runs[0] == 0 and runs[-1] == total
    assert np.all(np.diff(runs) >= 1)
    assert len(runs) - 1 <= slots


def test_paper_demo_shape_runs_are_balanced():
    # 281 x 281 x 150 at order 14: 5 x 21 columns of 64 x 14 points, 150 planes, 4 z chunks
    columns, nz, R, slots = 105, 150, 7, 304
    runs = wave.wave_column_runs_for(columns, nz, 4, 14, slots)
    assert runs is not None
    _check_cover(runs, columns * nz, slots)
    cost = _costs(runs, nz, R)
    seg = _segments(runs, nz)
    # an equal split of the planes would cost W + 2 fills where a run crosses a column
    W = -(-columns * nz // slots)
    assert cost.max() < W + 2 * (4 + R)
    assert cost.max() - cost.min() <= 4 + R
    # runs that cross a column boundary carry a second fill and are shorter
    assert np.diff(runs)[seg > 1].max() < np.diff(runs)[seg == 1].max()


def test_large_grid_keeps_z_chunks_unless_forced():
    # 592^3 at order 8: 10 x 37 columns, 9 chunks of 66 planes, 11 waves
    assert wave.wave_column_runs_for(370, 592, 9, 8, 304) is None
    runs = wave.wave_column_runs_for(370, 592, 9, 8, 304, force=True)
    _check_cover(runs, 370 * 592, 304)
    # runs longer than a column cross several columns
    assert _segments(runs, 592).max() >= 2


@pytest.mark.parametrize("columns,nz,so", [(1, 9, 4), (4, 50, 8), (380, 18, 8), (30, 38, 16), (7, 1000, 2)])
def test_forced_runs_cover_every_plane_once(columns, nz, so):
    runs = wave.wave_column_runs_for(columns, nz, 1, so, 304, force=True)
    total = columns * nz
    _check_cover(runs, total, 304)
    # at most one run per max(16, 2R) planes (a single run when the grid is smaller)
    assert len(runs) - 1 <= max(1, total // max(16, so))


def test_bad_arguments_are_rejected():
    for args in ((0, 10, 1, 8, 304), (10, 0, 1, 8, 304), (10, 10, 0, 8, 304), (10, 10, 1, 7, 304),
                 (10, 10, 1, 18, 304), (10, 10, 1, 8, 0)):
        with pytest.raises(wave.WaveError) as e:
            wave.wave_column_runs_for(*args)
        assert e.value.code == wave.WAVE_ERR_INVALID_ARG


@pytest.mark.parametrize("columns,nz,so,want", [
    (370, 592, 8, 9),     # 592^3 at order 8: 10 x 37 columns of 64 x 16, measured best of 1..9 chunks
    (430, 592, 16, 7),    # 592^3 at order 16 (equal spacing): 10 x 43 columns of 64 x 14
    (105, 150, 14, 4),    # the paper's demo shape: 8 waves out of reach, the most chunks of >= 32 planes
    (6, 20, 8, 1),        # fewer planes than one chunk's minimum: one chunk
])
def test_z_chunks_follow_the_wave_rule(columns, nz, so, want):
    """The z-chunk count of the plain 3D step on 152 SMs x 2 resident CTAs: at
    least 8 waves where chunks of max(32, 4R) planes allow it, then the count
    up to 16 waves whose last wave is fullest."""
    assert wave.wave_z_chunks_for(columns, nz, so, 304) == want


def test_z_chunks_properties():
    slots = 304
    for so in (2, 8, 16):
        R = so // 2
        for columns in (1, 7, 50, 144, 370, 1200):
            for nz in (10, 64, 150, 592, 1000):
                c = wave.wave_z_chunks_for(columns, nz, so, slots)
                cmax = max(1, nz // max(32, 4 * R))
                assert 1 <= c <= cmax
                if columns * cmax < 8 * slots:
                    assert c == cmax                        # short of 8 waves: as many chunks as allowed
                else:
                    lo = -(-8 * slots // columns)           # fewest chunks giving 8 waves
                    assert lo <= c <= min(cmax, 2 * lo)


def test_z_chunks_bad_arguments():
    for args in ((0, 10, 8, 304), (10, 0, 8, 304), (10, 10, 7, 304), (10, 10, 8, 0)):
        with pytest.raises(wave.WaveError):
            wave.wave_z_chunks_for(*args)
