"""torch.autograd.Function over the forward operator of the wave library.

``WaveForward.apply(m, q, op)`` returns receiver data d = F(m) q (Listing 1).
Its backward pass, for an upstream gradient ``g_d`` on d, returns
  * for m: J^T g_d, the adjoint-state vector-Jacobian product (Eq. 3 with the
    residual replaced by g_d), computed by wave_jacobian_adjoint with the
    forward wavefield stored or recomputed from checkpoints;
  * for q: F^T g_d (d is linear in q), computed by wave_adjoint.
Both run entirely in the CUDA library; nothing is differentiated by torch.
"""

from dataclasses import dataclass

import torch

from . import wave


@dataclass
class WaveOperator:
    """Everything but (m, q) that defines the forward operator."""
    ctx: wave.Context
    geom: wave.Geometry
    src: object          # (n_src, ndim) coordinates (tensor or array)
    rec: object          # (n_rec, ndim)
    dt: float
    nt: int
    space_order: int
    snap_mode: str = "auto"


class WaveForward(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m, q, op):
        m = m.detach().contiguous()
        q = q.detach().contiguous()
        d = wave.wave_forward(op.ctx, op.geom, m, op.src, q, op.rec, op.dt, op.nt, op.space_order)
        fctx.save_for_backward(m, q)
        fctx.op = op
        return d

    @staticmethod
    def backward(fctx, grad_d):
        m, q = fctx.saved_tensors
        op = fctx.op
        grad_d = grad_d.contiguous().to(torch.float32)
        gm = gq = None
        if fctx.needs_input_grad[0]:
            gm = wave.wave_jacobian_adjoint(op.ctx, op.geom, m, op.src, q, op.rec, grad_d, op.dt, op.nt,
                                            op.space_order, snap_mode=op.snap_mode)
        if fctx.needs_input_grad[1]:
            gq = wave.wave_adjoint(op.ctx, op.geom, m, op.src, op.rec, grad_d, op.dt, op.nt, op.space_order)
        return gm, gq, None


def forward_model(m, q, op):
    """Differentiable receiver data d = F(m) q."""
    return WaveForward.apply(m, q, op)
