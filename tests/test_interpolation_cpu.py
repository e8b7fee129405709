"""CPU check of the library's sparse-point interpolation structures (Sec. IV)
against the oracle's restriction operator: ``wave_interpolation_operator``
reads back the structure the CUDA path injects through (one row per unique
grid cell, no atomics), so this pins its host-side construction -- cell
indices with the padded layout, corner weights, the last-node rule, points on
nodes and tile edges, unequal spacing, offsets and absorbing layers -- without
a GPU.  Weights agree to FP32 rounding of the FP64 products."""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1608_08658_gb300 import build as libbuild
from paper_1608_08658_gb300 import wave


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return wave.lib()


def _geoms(og):
    return og, wave.Geometry(shape=og.shape, spacing=og.spacing, origin=og.origin, nbl=og.nbl,
                             sponge_vref=og.sponge_vref)


def _points(og, n, seed):
    r = np.random.default_rng(seed)
    lo = np.array(og.origin)
    hi = lo + (np.array(og.shape) - 1) * np.array(og.spacing)
    c = lo + r.uniform(size=(n, og.ndim)) * (hi - lo)
    c[0], c[1] = lo, hi                                        # first and last physical nodes
    c[2] = lo + np.round(r.uniform(size=og.ndim) * (np.array(og.shape) - 1)) * np.array(og.spacing)  # a node
    c[3, 0] = lo[0] + (64 - og.nbl) * og.spacing[0] if og.shape[0] > 64 - og.nbl >= 0 else c[3, 0]  # tile edge
    c[4] = np.minimum(c[4], hi)
    c[4, -1] = hi[-1]                                          # on the last depth node
    return c.astype(np.float32)


CASES = [
    ((83, 21, 40), (10.0, 12.0, 9.0), (3.0, -7.0, 0.0), 5),
    ((70, 33, 17), (12.5, 12.5, 12.5), (0.0, 0.0, 0.0), 0),
    ((150, 77), (7.5, 10.0), (0.0, 0.0), 9),
    ((41, 37), (10.0, 10.0), (-100.0, 5.0), 0),
]


@pytest.mark.parametrize("shape,spacing,origin,nbl", CASES)
def test_operator_matches_oracle(shape, spacing, origin, nbl):
    og = oracle.model.Geometry(shape=shape, spacing=spacing, origin=origin, nbl=nbl, sponge_vref=2.0)
    og, g = _geoms(og)
    coords = _points(og, 300, seed=len(shape) * 10 + nbl)
    idx, w = wave.wave_interpolation_operator(g, coords)
    n, C = idx.shape
    assert C == 2 ** og.ndim and n == len(coords)
    ncell = int(np.prod(og.comp_shape))
    assert idx.min() >= 0 and idx.max() < ncell
    ours = sp.coo_matrix((w.ravel().astype(np.float64), (np.repeat(np.arange(n), C), idx.ravel())),
                         shape=(n, ncell)).tocsr()
    ref = oracle.interp.interpolation_matrix(og, coords.astype(np.float64))
    assert abs(ours - ref).max() <= 1e-6
    # every point's weights form a partition of unity over distinct cells
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-6)
    assert all(len(set(row)) == C for row in idx)


def test_point_outside_is_rejected():
    og = oracle.model.Geometry(shape=(20, 10), spacing=(10.0, 10.0), nbl=4, sponge_vref=2.0)
    _, g = _geoms(og)
    with pytest.raises(wave.WaveError) as e:
        wave.wave_interpolation_operator(g, np.array([[50.0, 95.0]], dtype=np.float32))
    assert e.value.code == wave.WAVE_ERR_POINT_OUTSIDE


def test_empty_point_set():
    og = oracle.model.Geometry(shape=(20, 10, 8), spacing=(10.0, 10.0, 10.0), nbl=2, sponge_vref=2.0)
    _, g = _geoms(og)
    idx, w = wave.wave_interpolation_operator(g, np.zeros((0, 3), dtype=np.float32))
    assert idx.shape == (0, 8) and w.shape == (0, 8)


@pytest.mark.parametrize("shape,nbl", [((20, 20, 20), (1 << 20) + 1),                 # layer beyond 2^20 points
                                       ((1 << 20, 1 << 20, 1 << 20), 0),               # 2^60 points
                                       ((1 << 14, 1 << 14, 1 << 12), 40)])             # just above 2^40
def test_geometry_beyond_the_size_bounds_is_rejected(shape, nbl):
    """Geometry checks of the host-side set-up: the absorbing layer and the
    computational grid's point count are bounded before any size is formed, so
    no element count can overflow."""
    geom = wave.Geometry(shape=shape, spacing=(10.0, 10.0, 10.0), nbl=nbl, sponge_vref=2.0)
    with pytest.raises(wave.WaveError) as e:
        wave.wave_interpolation_operator(geom, np.array([[15.0, 15.0, 15.0]], np.float32))
    assert e.value.code == wave.WAVE_ERR_INVALID_ARG


def test_large_but_bounded_geometry_is_accepted():
    # 2^13 x 2^13 x 2^13 physical points (+ 2 x 40): below the 2^40 bound; nothing is allocated
    geom = wave.Geometry(shape=(1 << 13,) * 3, spacing=(10.0, 10.0, 10.0), nbl=40, sponge_vref=2.0)
    idx, wts = wave.wave_interpolation_operator(geom, np.array([[15.0, 15.0, 15.0]], np.float32))
    assert idx.shape == (1, 8) and abs(float(wts.sum()) - 1.0) < 1e-6


def test_point_count_bound_is_exclusive():
    """2^28 points would give 2^31 corner entries in 3D, one past the 32-bit
    row pointers of the injection structure: rejected before the coordinates
    are read (the call gets a one-point buffer that it never touches)."""
    import ctypes
    geom = wave.Geometry(shape=(20, 20, 20), spacing=(10.0, 10.0, 10.0), nbl=4, sponge_vref=2.0)
    g = geom.to_c()
    one = np.zeros(3, np.float32)
    idx = np.zeros(8, np.int64)
    wts = np.zeros(8, np.float32)
    for n, want in (((1 << 28), wave.WAVE_ERR_INVALID_ARG), ((1 << 28) + 5, wave.WAVE_ERR_INVALID_ARG),
                    (1, wave.WAVE_OK)):
        pts = wave.c_points(n, one.ctypes.data)
        rc = wave.lib().wave_interpolation_operator(ctypes.byref(g), ctypes.byref(pts), idx.ctypes.data,
                                                    wts.ctypes.data)
        assert rc == want, (n, rc)
