"""Parity at the full benchmark size (512^3 + 40-point sponge = 592^3 points,
order 8, the benchmark's model generator and launch configuration).

* Sampled outputs: from a seeded random state the library advances two steps;
  at sampled points (domain corners, sponge edges, tile edges, the source cell,
  random interior points) the oracle recomputes the same two steps on a window
  of half-width 2R+1 around the point (the window edge cannot influence the
  centre in two steps) and the values must agree within 1e-5 of the local scale.
* Properties that hold at any size: the dot-product test of Eq. 5-6 with all
  262 144 surface receivers, and checkpointed recomputation reproducing the
  stored-snapshot gradient bit for bit.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from gpu_cases import f32

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import inputs, wave  # noqa: E402

pytestmark = pytest.mark.gpu

N, NBL, SO = 512, 40, 8


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    shape, h = (N, N, N), (10.0, 10.0, 10.0)
    v = inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.05, corr_len=50.0, seed=7)
    m = inputs.slowness2(v)
    vmax = float(v.max())
    og = oracle.model.Geometry(shape=shape, spacing=h, nbl=NBL, sponge_vref=vmax)
    geom = wave.Geometry(shape=shape, spacing=h, nbl=NBL, sponge_vref=vmax)
    dt = f32(0.4 * oracle.model.dt_max(SO, h, vmax))
    ctx = wave.Context(0)
    yield og, geom, m, dt, ctx
    ctx.close()


def _window_operator(P_full, comp_shape_zyx, window):
    """Restriction of a (points x cells) operator to the cells of a window."""
    P = P_full.tocoo()
    z, rem = np.divmod(P.col, comp_shape_zyx[1] * comp_shape_zyx[2])
    y, x = np.divmod(rem, comp_shape_zyx[2])
    (z0, z1), (y0, y1), (x0, x1) = window
    keep = (z >= z0) & (z < z1) & (y >= y0) & (y < y1) & (x >= x0) & (x < x1)
    wy, wx = y1 - y0, x1 - x0
    col = ((z[keep] - z0) * wy + (y[keep] - y0)) * wx + (x[keep] - x0)
    ncell = (z1 - z0) * wy * wx
    return sp.csr_matrix((P.data[keep], (P.row[keep], col)), shape=(P.shape[0], ncell))


def test_sampled_two_steps_full_size(setup):
    og, geom, m, dt, ctx = setup
    nz, ny, nx = og.array_shape
    R = SO // 2
    g = torch.Generator(device="cuda").manual_seed(1234)
    u0 = torch.randn((nz, ny, nx), generator=g, device="cuda")
    u1 = torch.randn((nz, ny, nx), generator=g, device="cuda")
    src = np.array([[2555.0, 2555.0, 20.0]], dtype=np.float32)
    q = np.array([[3.0], [-2.0], [0.0]], dtype=np.float32)
    _, fp, fl = wave.wave_forward(ctx, geom, torch.from_numpy(m).cuda(), src, torch.from_numpy(q).cuda(), None,
                                  dt, 3, SO, u_init_prev=u0, u_init=u1, return_final=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (NBL, NBL, NBL), (NBL - 1, 300, 63), (300, 15, 64),
           (300, 16, 127), (nz // 2, ny // 2, 591), (42, 295, 295), (42, 296, 296), (2, 296, 295)]
    pts += [tuple(int(rng.integers(0, s)) for s in (nz, ny, nx)) for _ in range(14)]
    Ps_full = oracle.interp.interpolation_matrix(og, src)
    hw = 2 * R + 1
    worst = 0.0
    for (z, y, x) in pts:
        win = [(max(c - hw, 0), min(c + hw + 1, n)) for c, n in zip((z, y, x), (nz, ny, nx))]
        sl = tuple(slice(a, b) for a, b in win)
        mw = oracle.model.pad_model(og, m, window=win)
        ew = oracle.model.damping(og, window=win)
        Ps = _window_operator(Ps_full, (nz, ny, nx), win)
        Pr = sp.csr_matrix((0, mw.size))
        ref = oracle.wave.forward_op(mw, ew, og.spacing, dt, 3, SO, q, Ps, Pr,
                                     u_init_prev=u0[sl].cpu().numpy(), u_init=u1[sl].cpu().numpy())
        c = (z - win[0][0], y - win[1][0], x - win[2][0])
        for got, want in ((fp[z, y, x].item(), ref.u_prev[c]), (fl[z, y, x].item(), ref.u_last[c])):
            scale = np.abs(ref.u_last).max()
            err = abs(got - want) / scale
            worst = max(worst, err)
            assert err <= 1e-5, ((z, y, x), got, want)
    print("full-size sampled two-step parity: worst error %.2e of local scale" % worst)


def test_dot_product_full_size(setup):
    og, geom, m, dt, ctx = setup
    nt = 60
    src = np.array([[2555.0, 2555.0, 20.0]], dtype=np.float32)
    rec = torch.from_numpy(inputs.surface_grid_receivers(N, N, (10.0, 10.0), 20.0)).cuda()
    md = torch.from_numpy(m).cuda()
    g = torch.Generator(device="cuda").manual_seed(7)
    q = torch.randn((nt, 1), generator=g, device="cuda")
    y = torch.randn((nt, rec.shape[0]), generator=g, device="cuda")
    d = wave.wave_forward(ctx, geom, md, src, q, rec, dt, nt, SO)
    qa = wave.wave_adjoint(ctx, geom, md, src, rec, y, dt, nt, SO)
    lhs = float((d.double() * y.double()).sum())
    rhs = float((q.double() * qa.double()).sum())
    print("full-size dot test: %.9e vs %.9e (rel %.2e)" % (lhs, rhs, abs(lhs - rhs) / abs(lhs)))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))


def test_checkpointed_equals_stored_full_size(setup):
    og, geom, m, dt, ctx = setup
    nt = 40
    src = np.array([[2555.0, 2555.0, 20.0]], dtype=np.float32)
    rec = torch.from_numpy(inputs.surface_grid_receivers(N, N, (10.0, 10.0), 20.0)).cuda()
    md = torch.from_numpy(m).cuda()
    q = torch.from_numpy(wave.wave_ricker(nt, dt, 0.015).reshape(nt, 1)).cuda()
    d_obs = 0.9 * wave.wave_forward(ctx, geom, md * 1.01, src, q, rec, dt, nt, SO)
    g_full, phi_full = wave.wave_gradient(ctx, geom, md, src, q, rec, d_obs, dt, nt, SO, snap_mode="full_fp32")
    g_full = g_full.clone()
    ctx.set_checkpoint_interval(7)
    g_ck, phi_ck = wave.wave_gradient(ctx, geom, md, src, q, rec, d_obs, dt, nt, SO, snap_mode="checkpoint_fp32")
    ctx.set_checkpoint_interval(0)
    assert phi_full == phi_ck
    assert torch.equal(g_full, g_ck)
    ctx.trim()
