"""GPU checks of the torch.autograd.Function: backward against the oracle
gradient, against finite differences of the FP32 forward, and the q-gradient
against the dot-product identity."""

import numpy as np
import pytest

import oracle
from gpu_cases import geometries, rel_l2, small2d, small3d

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import wave  # noqa: E402
from paper_1608_08658_gb300.autograd import WaveOperator, forward_model  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = wave.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case,snap", [("2d", "full_fp32"), ("3d", "checkpoint_fp32"), ("3d", "full_fp16")])
def test_backward_matches_oracle_gradient(ctx, case, snap):
    og, m, dt, nt, so, src, q, rec = small2d(4) if case == "2d" else small3d(8)
    _, geom = geometries(og)
    d_obs = oracle.wave.forward(og, m * 1.03, dt, nt, so, q, src, rec).d.astype(np.float32)
    op = WaveOperator(ctx, geom, src, rec, dt, nt, so, snap_mode=snap)
    mt = torch.from_numpy(m).cuda().requires_grad_(True)
    qt = torch.from_numpy(q).cuda()
    d = forward_model(mt, qt, op)
    loss = 0.5 * ((d.double() - torch.from_numpy(d_obs).cuda().double()) ** 2).sum()
    loss.backward()
    g_ref, phi_ref = oracle.wave.gradient(og, m, dt, nt, so, q, src, rec, d_obs)
    assert abs(loss.item() - phi_ref) <= 1e-4 * phi_ref
    assert rel_l2(mt.grad.cpu().numpy(), g_ref) <= 5e-4


def test_backward_finite_difference(ctx):
    og, m, dt, nt, so, src, q, rec = small2d(8, nt=120)
    _, geom = geometries(og)
    d_obs = oracle.wave.forward(og, m * 0.97, dt, nt, so, q, src, rec).d.astype(np.float32)
    op = WaveOperator(ctx, geom, src, rec, dt, nt, so, snap_mode="full_fp32")
    qt = torch.from_numpy(q).cuda()
    dobs = torch.from_numpy(d_obs).cuda().double()

    def loss_of(mm, grad=False):
        mt = torch.from_numpy(mm.astype(np.float32)).cuda().requires_grad_(grad)
        L = 0.5 * ((forward_model(mt, qt, op).double() - dobs) ** 2).sum()
        if grad:
            L.backward()
            return L.item(), mt.grad.cpu().numpy().astype(np.float64)
        return L.item()

    _, g = loss_of(m, grad=True)
    rng = np.random.default_rng(2)
    from paper_1608_08658_gb300 import inputs
    dm = inputs.smooth_perturbation(og.shape, og.spacing, seed=5) * 0.01 * m
    eps = 1.0
    fd = (loss_of(m + eps * dm) - loss_of(m - eps * dm)) / (2 * eps)
    an = float(np.sum(g * dm))
    print("FD directional derivative %.6e, adjoint-state %.6e" % (fd, an))
    assert abs(fd - an) <= 2e-3 * abs(an)
    del rng


def test_q_gradient_is_the_adjoint(ctx):
    og, m, dt, nt, so, src, q, rec = small2d(6)
    _, geom = geometries(og)
    op = WaveOperator(ctx, geom, src, rec, dt, nt, so)
    mt = torch.from_numpy(m).cuda()
    qt = torch.from_numpy(q).cuda().requires_grad_(True)
    rng = np.random.default_rng(8)
    y = torch.from_numpy(rng.standard_normal((nt, len(rec))).astype(np.float32)).cuda()
    d = forward_model(mt, qt, op)
    (d * y).sum().backward()
    ref = oracle.wave.adjoint(og, m, dt, nt, so, y.cpu().numpy(), src, rec)
    assert rel_l2(qt.grad.cpu().numpy(), ref) <= 1e-4
