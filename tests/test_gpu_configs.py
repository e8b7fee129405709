"""GPU checks of the FWI-gradient and large-model workloads at their full sizes.

FWI gradient workload (256^3 + 40-point sponge = 336^3, h = 12.5 m, order 8,
nt = 1500, v(z) = 1.5 + 0.6 z with three Gaussian anomalies as the true model,
128 x 128 receivers): the gradient with snapshots stored every step in FP16 /
BF16, with checkpointed recomputation and with the automatic storage plan are
compared with each other (recomputation bit for bit, reduced precision within
the gradient tolerance), and with the autograd.Function backward pass; the
Taylor test of Eq. 7-8 runs on the GPU on the 64^3 version.

Large workload (1000 x 1000 x 600 + 40 = 1080 x 1080 x 680, order 16, layered
model with a salt body): sampled two-step parity against the oracle on local
windows, as for the throughput workload.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from gpu_cases import f32

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import inputs, wave  # noqa: E402
from paper_1608_08658_gb300.autograd import WaveOperator, forward_model  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = wave.Context(0)
    yield c
    c.close()


def _fwi_case(n, nt, so=8):
    h = (12.5, 12.5, 12.5)
    shape = (n, n, n)
    v0, vt = inputs.gradient_models(shape, h)
    vmax = float(vt.max())
    geom = wave.Geometry(shape=shape, spacing=h, nbl=40, sponge_vref=vmax)
    dt = f32(0.4 * wave.wave_dt_max(h, so, vmax))
    ext = (n - 1) * h[0]
    src = np.array([[0.5 * ext, 0.5 * ext, 25.0]], dtype=np.float32)
    k = max(2, n // 2)
    rec = inputs.surface_grid_receivers(k, k, (2 * h[0], 2 * h[1]), 25.0)
    q = wave.wave_ricker(nt, dt, 0.010).reshape(nt, 1)
    return geom, inputs.slowness2(v0), inputs.slowness2(vt), src, rec, q, dt


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


def test_fwi_gradient_storage_modes_full_size(ctx):
    nt, so = 1500, 8
    geom, m0, mt, src, rec, q, dt = _fwi_case(256, nt, so)
    m0d, qd = torch.from_numpy(m0).cuda(), torch.from_numpy(q).cuda()
    d_obs = wave.wave_forward(ctx, geom, torch.from_numpy(mt).cuda(), src, qd, rec, dt, nt, so)
    g = {}
    for mode in ("auto", "checkpoint_fp32", "full_fp16", "full_bf16"):
        ctx.set_checkpoint_interval(100 if mode == "checkpoint_fp32" else 0)
        gm, phi = wave.wave_gradient(ctx, geom, m0d, src, qd, rec, d_obs, dt, nt, so, snap_mode=mode)
        g[mode] = (gm.clone(), phi)
    ctx.set_checkpoint_interval(0)
    assert torch.equal(g["auto"][0], g["checkpoint_fp32"][0])
    assert g["auto"][1] == g["checkpoint_fp32"][1]
    e16 = _rel(g["full_fp16"][0], g["auto"][0])
    ebf = _rel(g["full_bf16"][0], g["auto"][0])
    print("336^3 nt1500 gradient: FP16 snapshots rel-L2 %.2e, BF16 %.2e vs FP32" % (e16, ebf))
    # measured on this workload: 2.4e-4 (FP16) and 1.9e-3 (BF16); gates at about twice that
    assert e16 <= 5e-4
    assert ebf <= 4e-3
    # the autograd.Function backward is the same adjoint-state computation
    op = WaveOperator(ctx, geom, src, rec, dt, nt, so, snap_mode="auto")
    mt_ = m0d.clone().requires_grad_(True)
    d = forward_model(mt_, qd, op)
    loss = 0.5 * ((d.double() - d_obs.double()) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - g["auto"][1]) <= 1e-9 * g["auto"][1]
    assert _rel(mt_.grad, g["auto"][0]) <= 1e-6
    ctx.trim()


def test_taylor_gpu_64cube(ctx):
    nt, so = 400, 8
    geom, m0, mt, src, rec, q, dt = _fwi_case(64, nt, so)
    m0d, qd = torch.from_numpy(m0).cuda(), torch.from_numpy(q).cuda()
    d_obs = wave.wave_forward(ctx, geom, torch.from_numpy(mt).cuda(), src, qd, rec, dt, nt, so)
    g, phi0 = wave.wave_gradient(ctx, geom, m0d, src, qd, rec, d_obs, dt, nt, so, snap_mode="full_fp32")
    dm = torch.from_numpy((0.05 * m0 * inputs.smooth_perturbation(geom.shape, geom.spacing, seed=3)).astype(
        np.float32)).cuda()
    gdm = float((g.double() * dm.double()).sum())
    # FP32 modelling: below h ~ 0.05 the second-order remainder (~1e-5 of phi)
    # meets the FP32 rounding of phi, so slope 2 is checked where it is resolved
    hs = np.array([0.2, 0.1, 0.05, 0.025])
    e1, e2 = [], []
    for h in hs:
        d = wave.wave_forward(ctx, geom, m0d + h * dm, src, qd, rec, dt, nt, so)
        phi = 0.5 * float(((d.double() - d_obs.double()) ** 2).sum())
        e1.append(abs(phi - phi0))
        e2.append(abs(phi - phi0 - h * gdm))
    s1 = np.diff(np.log(e1)) / np.diff(np.log(hs))
    s2 = np.diff(np.log(e2)) / np.diff(np.log(hs))
    print("GPU Taylor test slopes: first order", np.round(s1, 3), "second order", np.round(s2, 3))
    assert np.all(np.abs(s1 - 1.0) < 0.1)
    assert np.all(np.abs(s2[:2] - 2.0) < 0.3)


def _window_operator(P_full, comp_shape_zyx, window):
    P = P_full.tocoo()
    z, rem = np.divmod(P.col, comp_shape_zyx[1] * comp_shape_zyx[2])
    y, x = np.divmod(rem, comp_shape_zyx[2])
    (z0, z1), (y0, y1), (x0, x1) = window
    keep = (z >= z0) & (z < z1) & (y >= y0) & (y < y1) & (x >= x0) & (x < x1)
    wy, wx = y1 - y0, x1 - x0
    col = ((z[keep] - z0) * wy + (y[keep] - y0)) * wx + (x[keep] - x0)
    return sp.csr_matrix((P.data[keep], (P.row[keep], col)), shape=(P.shape[0], (z1 - z0) * wy * wx))


def test_large_model_sampled_two_steps(ctx):
    so, nbl = 16, 40
    shape, h = (1000, 1000, 600), (10.0, 10.0, 10.0)
    v = inputs.layered_salt_velocity(shape, h)
    m = inputs.slowness2(v)
    og = oracle.model.Geometry(shape=shape, spacing=h, nbl=nbl, sponge_vref=4.5)
    geom = wave.Geometry(shape=shape, spacing=h, nbl=nbl, sponge_vref=4.5)
    dt = f32(0.4 * oracle.model.dt_max(so, h, 4.5))
    nz, ny, nx = og.array_shape
    g = torch.Generator(device="cuda").manual_seed(99)
    u0 = torch.randn((nz, ny, nx), generator=g, device="cuda")
    u1 = torch.randn((nz, ny, nx), generator=g, device="cuda")
    src = np.array([[4995.0, 4995.0, 20.0]], dtype=np.float32)
    q = np.array([[5.0], [1.0], [0.0]], dtype=np.float32)
    _, fp, fl = wave.wave_forward(ctx, geom, torch.from_numpy(m).cuda(), src, torch.from_numpy(q).cuda(), None,
                                  dt, 3, so, u_init_prev=u0, u_init=u1, return_final=True)
    torch.cuda.synchronize()
    R = so // 2
    hw = 2 * R + 1
    rng = np.random.default_rng(17)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nbl, 540, 63), (340, 16, 64), (42, 539, 539), (42, 540, 540),
           (679, 1079, 1079), (300, 700, 1023)]
    pts += [tuple(int(rng.integers(0, s)) for s in (nz, ny, nx)) for _ in range(10)]
    Ps_full = oracle.interp.interpolation_matrix(og, src)
    worst = 0.0
    for (z, y, x) in pts:
        win = [(max(c - hw, 0), min(c + hw + 1, n)) for c, n in zip((z, y, x), (nz, ny, nx))]
        sl = tuple(slice(a, b) for a, b in win)
        mw = oracle.model.pad_model(og, m, window=win)
        ew = oracle.model.damping(og, window=win)
        Ps = _window_operator(Ps_full, (nz, ny, nx), win)
        ref = oracle.wave.forward_op(mw, ew, og.spacing, dt, 3, so, q, Ps, sp.csr_matrix((0, mw.size)),
                                     u_init_prev=u0[sl].cpu().numpy(), u_init=u1[sl].cpu().numpy())
        c = (z - win[0][0], y - win[1][0], x - win[2][0])
        scale = np.abs(ref.u_last).max()
        for got, want in ((fp[z, y, x].item(), ref.u_prev[c]), (fl[z, y, x].item(), ref.u_last[c])):
            err = abs(got - want) / scale
            worst = max(worst, err)
            assert err <= 1e-5, ((z, y, x), got, want)
    print("large-model sampled two-step parity: worst error %.2e of local scale" % worst)
    ctx.trim()


def test_large_salt_gradient_bf16_against_fp32(ctx):
    """Large workload at its full grid (1080 x 1080 x 680 points, order 16) and a
    shorter time axis: observed data from the layered model with the salt body,
    the gradient at the depth-smoothed layers without the salt.  The objective
    is not zero (the smoothed near-surface layers change the early arrivals),
    and the gradient with BF16 checkpointed snapshots is compared with the FP32
    checkpointed one; the objective of both is the same forward sweep."""
    so, nt = 16, 1200
    shape, h = (1000, 1000, 600), (10.0, 10.0, 10.0)
    geom = wave.Geometry(shape=shape, spacing=h, nbl=40, sponge_vref=4.5)
    dt = f32(0.4 * wave.wave_dt_max(h, so, 4.5))
    src = np.array([[4995.0, 4995.0, 20.0]], dtype=np.float32)
    gx = np.linspace(0.0, 9990.0, 100)
    X, Y = np.meshgrid(gx, gx, indexing="xy")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 20.0)], axis=1).astype(np.float32)
    qd = torch.from_numpy(wave.wave_ricker(nt, dt, 0.010).reshape(nt, 1)).cuda()
    mt = torch.from_numpy(inputs.slowness2(inputs.layered_salt_velocity(shape, h))).cuda()
    d_obs = wave.wave_forward(ctx, geom, mt, src, qd, rec, dt, nt, so)
    del mt
    m0 = torch.from_numpy(inputs.slowness2(inputs.layered_starting_velocity(shape, h))).cuda()
    g32, phi32 = wave.wave_gradient(ctx, geom, m0, src, qd, rec, d_obs, dt, nt, so, snap_mode="checkpoint_fp32")
    g32 = g32.clone()
    gbf, phibf = wave.wave_gradient(ctx, geom, m0, src, qd, rec, d_obs, dt, nt, so, snap_mode="checkpoint_bf16")
    e = _rel(gbf, g32)
    print("large salt model, so16 nt%d: objective %.6e, |g| %.3e, BF16-checkpointed vs FP32 gradient rel-L2 %.2e"
          % (nt, phi32, float(g32.double().norm()), e))
    assert phi32 > 0.0 and float(g32.abs().max()) > 0.0
    assert phibf == phi32
    assert e <= 4e-3
    ctx.trim()
