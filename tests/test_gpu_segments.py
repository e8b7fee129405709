"""GPU parity of the segmented plain step (column segments of equal length per
CTA; the step injects its source row and samples its receiver row itself).

* Bit for bit against the z-chunk decomposition (receiver traces, final
  fields): small grids with ragged tiles, runs that cross from one column into
  the next (several columns per run on a wide, shallow grid), many sources
  sharing cells, receivers on tile edges, receiver rows streamed to pinned host
  memory in blocks of time steps, every order from 2 to 16.
* Against the FP64 oracle (Listing 1 / Eq. 1 with the injection and
  interpolation of Sec. III-C) on a case whose runs cross columns.
* At the paper's 3D demonstration shape (Sec. V-D: 201 x 201 x 70 + 40-point
  layer = 281 x 281 x 150 points, order 14, the decomposition the benchmark
  uses): sampled outputs of two steps from a random state against the oracle
  on windows, receiver rows equal to the interpolation of the levels they
  sample, and equality with the z-chunk decomposition.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from gpu_cases import f32, geometries, rel_l2, small3d

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import inputs, wave  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = wave.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _both(ctx, geom, m, src, q, rec, dt, nt, so, **kw):
    """Forward modelling with z chunks (mode 0) and with column segments (mode 2)."""
    out = []
    for mode in (0, 2):
        ctx.set_column_segments(mode)
        try:
            r = wave.wave_forward(ctx, geom, m, src, q, rec, dt, nt, so, return_final=True, **kw)
        finally:
            ctx.set_column_segments(1)
        out.append([x.cpu().numpy() if torch.is_tensor(x) else np.array(x) for x in r])
    return out


def _many_sources(og, n, seed):
    """n sources: random points, pairs inside one cell, and points on tile
    edges (x = 64 points from the corner), so that cells and CTAs share them."""
    r = inputs.rng(seed)
    lo = np.array(og.origin, dtype=np.float64)
    hi = lo + (np.array(og.shape) - 1) * np.array(og.spacing)
    pts = lo + r.uniform(0.05, 0.95, size=(n, 3)) * (hi - lo)
    pts[1] = pts[0] + 0.1 * np.array(og.spacing)          # same cell as source 0
    pts[2, 0] = lo[0] + (64 - og.nbl) * og.spacing[0]     # on an x tile edge
    pts[3, 0] = lo[0] + (63.5 - og.nbl) * og.spacing[0]   # straddles it
    return pts.astype(np.float32)


@pytest.mark.parametrize("so,iso", [(2, False), (4, False), (8, False), (8, True), (12, False), (14, True),
                                    (16, False), (16, True)])
def test_segments_equal_chunks_small(ctx, so, iso):
    og, m, dt, nt, so, src, q, rec = small3d(so, spacing=(10.0, 10.0, 10.0) if iso else (10.0, 12.0, 9.0),
                                              nsrc=6, nrec=60)
    src = _many_sources(og, 6, seed=so)
    _, geom = geometries(og)
    (d0, fp0, fl0), (d2, fp2, fl2) = _both(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, so)
    assert np.array_equal(d0, d2) and np.array_equal(fp0, fp2) and np.array_equal(fl0, fl2)


def test_segments_cross_several_columns(ctx):
    """A wide, shallow grid: 380 columns of 18 planes for 304 resident CTAs, so
    every run covers parts of two or three columns."""
    so = 8
    og, m, dt, nt, so, src, q, rec = small3d(so, shape=(600, 600, 10), nbl=4, nt=25, nsrc=12, nrec=300,
                                              spacing=(10.0, 10.0, 10.0))
    src = _many_sources(og, 12, seed=3)
    rec = _many_sources(og, 300, seed=4)
    _, geom = geometries(og)
    (d0, fp0, fl0), (d2, fp2, fl2) = _both(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, so)
    assert np.array_equal(d0, d2) and np.array_equal(fp0, fp2) and np.array_equal(fl0, fl2)


def test_segments_match_oracle_across_columns(ctx):
    """Runs that cross columns (forced segments on a grid of 30 columns of 38
    planes) against the oracle."""
    so = 8
    og, m, dt, nt, so, src, q, rec = small3d(so, shape=(170, 40, 30), nbl=4, nt=40, nsrc=5, nrec=40)
    src = _many_sources(og, 5, seed=9)
    _, geom = geometries(og)
    ctx.set_column_segments(2)
    try:
        d, fp, fl = wave.wave_forward(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, so, return_final=True)
    finally:
        ctx.set_column_segments(1)
    ref = oracle.wave.forward(og, m, dt, nt, so, q, src, rec)
    e_d = rel_l2(d.cpu().numpy(), ref.d)
    e_u = np.abs(fl.cpu().numpy() - ref.u_last).max() / np.abs(ref.u_last).max()
    print("segmented step vs oracle: receivers rel-L2 %.2e, field %.2e" % (e_d, e_u))
    assert e_d <= 1e-4 and e_u <= 1e-4


def test_segments_streamed_rows(ctx):
    """Receiver rows copied to pinned host memory in blocks of 128 steps while
    the sweep runs: each block ends with its own sampling of the last row."""
    so = 4
    og, m, dt, nt, so, src, q, rec = small3d(so, nt=300, nsrc=2, nrec=30)
    _, geom = geometries(og)
    outs = []
    for mode in (0, 2):
        ctx.set_column_segments(mode)
        try:
            d = torch.empty((nt, len(rec)), dtype=torch.float32).pin_memory()
            wave.wave_forward(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, so, d_out=d)
            torch.cuda.synchronize()
            outs.append(d.numpy().copy())
        finally:
            ctx.set_column_segments(1)
    assert np.array_equal(outs[0], outs[1])
    assert np.abs(outs[1]).max() > 0


def test_column_segment_mode_is_checked(ctx):
    for bad in (-1, 3):
        with pytest.raises(wave.WaveError) as e:
            ctx.set_column_segments(bad)
        assert e.value.code == wave.WAVE_ERR_INVALID_ARG


# ---------------------------------------------------------------- demonstration shape

DEMO_SHAPE, DEMO_H, DEMO_NBL, DEMO_SO = (201, 201, 70), (15.0, 15.0, 15.0), 40, 14


@pytest.fixture(scope="module")
def demo(ctx):
    prof = inputs.layered_profile(DEMO_SHAPE[2], DEMO_H[2], 5, v_min=1.5, v_max=3.5, seed=21)
    v = np.broadcast_to(prof[:, None, None], DEMO_SHAPE[::-1]).astype(np.float32).copy()
    m = inputs.slowness2(v)
    vmax = float(v.max())
    og = oracle.model.Geometry(shape=DEMO_SHAPE, spacing=DEMO_H, nbl=DEMO_NBL, sponge_vref=vmax)
    _, geom = geometries(og)
    dt = f32(0.4 * oracle.model.dt_max(DEMO_SO, DEMO_H, vmax))
    return og, geom, m, dt


def _window_operator(P_full, comp_shape_zyx, window):
    """Restriction of a (points x cells) operator to the cells of a window."""
    P = P_full.tocoo()
    z, rem = np.divmod(P.col, comp_shape_zyx[1] * comp_shape_zyx[2])
    y, x = np.divmod(rem, comp_shape_zyx[2])
    (z0, z1), (y0, y1), (x0, x1) = window
    keep = (z >= z0) & (z < z1) & (y >= y0) & (y < y1) & (x >= x0) & (x < x1)
    wy, wx = y1 - y0, x1 - x0
    col = ((z[keep] - z0) * wy + (y[keep] - y0)) * wx + (x[keep] - x0)
    return sp.csr_matrix((P.data[keep], (P.row[keep], col)), shape=(P.shape[0], (z1 - z0) * wy * wx))


def test_demo_shape_sampled_two_steps(ctx, demo):
    og, geom, m, dt = demo
    nz, ny, nx = og.array_shape
    R = DEMO_SO // 2
    g = torch.Generator(device="cuda").manual_seed(99)
    u0 = torch.randn((nz, ny, nx), generator=g, device="cuda")
    u1 = torch.randn((nz, ny, nx), generator=g, device="cuda")
    src = np.array([[1500.0, 1500.0, 30.0], [1502.0, 1497.0, 31.0]], dtype=np.float32)
    q = np.array([[3.0, 1.0], [-2.0, 0.5], [0.0, 0.0]], dtype=np.float32)
    rec = inputs.surface_grid_receivers(DEMO_SHAPE[0], DEMO_SHAPE[1], DEMO_H[:2], 30.0)
    d, fp, fl = wave.wave_forward(ctx, geom, _dev(m), src, _dev(q), rec, dt, 3, DEMO_SO, u_init_prev=u0, u_init=u1,
                                  return_final=True)
    torch.cuda.synchronize()
    # receiver rows are the interpolation of the levels they sample (rows 1, 2)
    Pr = oracle.interp.interpolation_matrix(og, rec)
    for row, level in ((1, fp), (2, fl)):
        want = Pr @ level.cpu().numpy().astype(np.float64).ravel()
        got = d[row].cpu().numpy()
        assert np.abs(got - want).max() <= 2e-6 * np.abs(want).max(), row
    # sampled points: tile and segment edges, the source cells, the sponge, random points
    rng = np.random.default_rng(8)
    z_src = int(round(30.0 / DEMO_H[2])) + DEMO_NBL
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (DEMO_NBL, DEMO_NBL, DEMO_NBL), (z_src, 140, 140),
           (z_src + 1, 140, 141), (51, 13, 63), (52, 14, 64), (104, 27, 127), (nz // 2, ny // 2, nx - 1)]
    pts += [tuple(int(rng.integers(0, s)) for s in (nz, ny, nx)) for _ in range(12)]
    Ps_full = oracle.interp.interpolation_matrix(og, src)
    hw = 2 * R + 1
    worst = 0.0
    for (z, y, x) in pts:
        win = [(max(c - hw, 0), min(c + hw + 1, n)) for c, n in zip((z, y, x), (nz, ny, nx))]
        sl = tuple(slice(a, b) for a, b in win)
        mw = oracle.model.pad_model(og, m, window=win)
        ew = oracle.model.damping(og, window=win)
        Ps = _window_operator(Ps_full, (nz, ny, nx), win)
        ref = oracle.wave.forward_op(mw, ew, og.spacing, dt, 3, DEMO_SO, q, Ps, sp.csr_matrix((0, mw.size)),
                                     u_init_prev=u0[sl].cpu().numpy(), u_init=u1[sl].cpu().numpy())
        c = (z - win[0][0], y - win[1][0], x - win[2][0])
        scale = np.abs(ref.u_last).max()
        for got, want in ((fp[z, y, x].item(), ref.u_prev[c]), (fl[z, y, x].item(), ref.u_last[c])):
            err = abs(got - want) / scale
            worst = max(worst, err)
            assert err <= 1e-5, ((z, y, x), got, want)
    print("demo shape sampled two-step parity: worst error %.2e of local scale" % worst)


def test_demo_shape_segments_equal_chunks(ctx, demo):
    og, geom, m, dt = demo
    nt = 40
    src = np.array([[1500.0, 1500.0, 30.0]], dtype=np.float32)
    rec = inputs.surface_grid_receivers(DEMO_SHAPE[0], DEMO_SHAPE[1], DEMO_H[:2], 30.0)
    q = wave.wave_ricker(nt, dt, 0.010).reshape(nt, 1)
    (d0, fp0, fl0), (d2, fp2, fl2) = _both(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, DEMO_SO)
    assert np.array_equal(d0, d2) and np.array_equal(fp0, fp2) and np.array_equal(fl0, fl2)
    assert np.abs(d2).max() > 0
