"""GPU edge cases through the C ABI, each against the FP64 oracle: the shortest
time axis (nt = 2), empty point sets, no absorbing layer, grids smaller than one
CTA tile and than the stencil radius, and a grid one launch cannot cover."""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from gpu_cases import f32, geometries, rel_l2

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import wave  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = wave.Context(0)
    yield c
    c.close()


def _case(shape, spacing, nbl, so, seed=3, nrec=7):
    og = oracle.model.Geometry(shape=shape, spacing=spacing, nbl=nbl, sponge_vref=2.5)
    r = np.random.default_rng(seed)
    m = (1.0 / (1.5 + r.uniform(size=og.phys_array_shape)) ** 2).astype(np.float32)
    dt = f32(0.4 * oracle.model.dt_max(so, spacing, 2.5))
    lo = np.array(og.origin)
    hi = lo + (np.array(shape) - 1) * np.array(spacing)
    src = (lo + 0.5 * (hi - lo)).reshape(1, -1).astype(np.float32)
    rec = (lo + r.uniform(size=(nrec, len(shape))) * (hi - lo)).astype(np.float32)
    return og, m, dt, src, rec, r


def _random_state(og, r):
    return [r.standard_normal(og.array_shape).astype(np.float32) for _ in range(2)]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _oracle_from_state(og, m, dt, nt, so, q, Ps, Pr, u0, u1):
    return oracle.wave.forward_op(oracle.model.pad_model(og, m), oracle.model.damping(og), og.spacing, dt, nt, so,
                                  q, Ps, Pr, u_init_prev=u0, u_init=u1)


@pytest.mark.parametrize("ndim", [2, 3])
def test_two_time_levels(ctx, ndim):
    """nt = 2: d^0 = P_r u^0 and one step to d^1."""
    shape, h = ((40, 23), (10.0, 10.0)) if ndim == 2 else ((30, 20, 25), (10.0, 10.0, 10.0))
    so = 8
    og, m, dt, src, rec, r = _case(shape, h, 4, so)
    _, geom = geometries(og)
    u0, u1 = _random_state(og, r)
    q = r.standard_normal((2, 1)).astype(np.float32)
    d, fp, fl = wave.wave_forward(ctx, geom, _dev(m), src, _dev(q), rec, dt, 2, so, u_init_prev=_dev(u0),
                                  u_init=_dev(u1), return_final=True)
    Ps, Pr = oracle.wave.operators(og, src, rec)
    ref = _oracle_from_state(og, m, dt, 2, so, q, Ps, Pr, u0, u1)
    assert rel_l2(d.cpu().numpy(), ref.d) <= 1e-5
    np.testing.assert_array_equal(fp.cpu().numpy(), u1)           # u^{nt-2} is the given u^0
    assert np.abs(fl.cpu().numpy() - ref.u_last).max() <= 1e-5 * np.abs(ref.u_last).max()


def test_no_sources_no_receivers(ctx):
    """Empty point sets: the field evolves from its initial state alone."""
    so, nt = 6, 9
    og, m, dt, _, _, r = _case((37, 19, 21), (10.0, 12.0, 9.0), 3, so)
    _, geom = geometries(og)
    u0, u1 = _random_state(og, r)
    d, _, fl = wave.wave_forward(ctx, geom, _dev(m), None, None, None, dt, nt, so, u_init_prev=_dev(u0),
                                 u_init=_dev(u1), return_final=True)
    assert d.shape == (nt, 0)
    n = int(np.prod(og.array_shape))
    ref = _oracle_from_state(og, m, dt, nt, so, np.zeros((nt, 1)), sp.csr_matrix((1, n)), sp.csr_matrix((0, n)),
                             u0, u1)
    err = np.abs(fl.cpu().numpy() - ref.u_last).max() / np.abs(ref.u_last).max()
    print("no points, 3D so%d nt%d: max field error %.2e" % (so, nt, err))
    assert err <= 1e-5


@pytest.mark.parametrize("so", [4, 16])
def test_no_absorbing_layer(ctx, so):
    """nbl = 0: eta = 0 everywhere (the undamped update only); forward and gradient."""
    nt = 40
    og, m, dt, src, rec, r = _case((45, 30, 28), (10.0, 10.0, 10.0), 0, so, nrec=15)
    _, geom = geometries(og)
    q = (r.standard_normal((nt, 1)) * 1e2).astype(np.float32)
    d = wave.wave_forward(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, so).cpu().numpy()
    ref = oracle.wave.forward(og, m, dt, nt, so, q, src, rec)
    assert rel_l2(d, ref.d) <= 1e-4
    d_obs = oracle.wave.forward(og, m * 1.03, dt, nt, so, q, src, rec).d.astype(np.float32)
    g, phi = wave.wave_gradient(ctx, geom, _dev(m), src, _dev(q), rec, _dev(d_obs), dt, nt, so,
                                snap_mode="full_fp32")
    g_ref, phi_ref = oracle.wave.gradient(og, m, dt, nt, so, q, src, rec, d_obs)
    e_g = rel_l2(g.cpu().numpy(), g_ref)
    print("nbl 0, so%d: receivers rel-L2 %.2e, gradient %.2e" % (so, rel_l2(d, ref.d), e_g))
    assert e_g <= 5e-4 and abs(phi - phi_ref) <= 1e-4 * phi_ref


@pytest.mark.parametrize("shape,so", [((9, 5, 4), 8), ((6, 3, 2), 16), ((7, 5), 16), ((3, 2), 2)])
def test_grid_smaller_than_a_tile(ctx, shape, so):
    """Grids narrower than one 64 x 16 tile and, in places, than the stencil radius."""
    nt = 6
    h = (10.0,) * len(shape)
    og, m, dt, src, rec, r = _case(shape, h, 2, so, nrec=3)
    _, geom = geometries(og)
    u0, u1 = _random_state(og, r)
    q = r.standard_normal((nt, 1)).astype(np.float32)
    d, _, fl = wave.wave_forward(ctx, geom, _dev(m), src, _dev(q), rec, dt, nt, so, u_init_prev=_dev(u0),
                                 u_init=_dev(u1), return_final=True)
    Ps, Pr = oracle.wave.operators(og, src, rec)
    ref = _oracle_from_state(og, m, dt, nt, so, q, Ps, Pr, u0, u1)
    assert rel_l2(d.cpu().numpy(), ref.d) <= 1e-5
    assert np.abs(fl.cpu().numpy() - ref.u_last).max() <= 1e-5 * np.abs(ref.u_last).max()


def test_grid_beyond_one_launch_is_rejected(ctx):
    """More than 65535 tiles along axis 1 cannot be one launch: a clean error
    before any work, and the context keeps working."""
    shape, h = (4, 1 << 20), (10.0, 10.0)       # the largest axis; + 2 x 40 sponge points = 65541 tiles
    geom = wave.Geometry(shape=shape, spacing=h, nbl=40, sponge_vref=2.0)
    m = np.full((shape[1], shape[0]), 1.0 / 4.0, dtype=np.float32)
    dt = f32(0.4 * wave.wave_dt_max(h, 4, 2.0))
    with pytest.raises(wave.WaveError) as e:
        wave.wave_forward(ctx, geom, m, None, None, None, dt, 3, 4)
    assert e.value.code == wave.WAVE_ERR_NOT_SUPPORTED
    og, m2, dt2, src, rec, _ = _case((20, 12), (10.0, 10.0), 2, 4)
    _, g2 = geometries(og)
    q = np.ones((5, 1), np.float32)
    d = wave.wave_forward(ctx, g2, m2, src, q, rec, dt2, 5, 4)
    ref = oracle.wave.forward(og, m2, dt2, 5, 4, q, src, rec).d
    assert rel_l2(d, ref) <= 1e-4


def test_bounded_wait_runs_out_and_context_recovers():
    """Failure detection without a fault: one step launch issues none of its
    tile loads (a barrier phase that nothing completes), so with the wait
    limit at 2 ms its consumers' waits run out; each CTA records the timeout
    and returns, and the call reports WAVE_ERR_TIMEOUT.  The same context, with
    the default limit restored, then runs a normal forward that matches the
    oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so, nt = 8, 12
    og, m, dt, src, rec, r = _case((83, 37, 40), (10.0, 10.0, 10.0), 4, so, nrec=11)
    _, geom = geometries(og)
    q = (r.standard_normal((nt, 1)) * 1e2).astype(np.float32)
    with wave.Context(0) as c:
        md, qd = _dev(m), _dev(q)
        c.set_wait_limit_ns(2_000_000)
        c.withhold_next_loads()
        with pytest.raises(wave.WaveError) as e:
            wave.wave_forward(c, geom, md, src, qd, rec, dt, nt, so)
        assert e.value.code == wave.WAVE_ERR_TIMEOUT
        assert "bounded wait" in str(e.value)
        # only the one launch withholds its loads: the next call succeeds
        c.set_wait_limit_ns(0)
        d = wave.wave_forward(c, geom, md, src, qd, rec, dt, nt, so).cpu().numpy()
    ref = oracle.wave.forward(og, m, dt, nt, so, q, src, rec).d
    assert rel_l2(d, ref) <= 1e-4
