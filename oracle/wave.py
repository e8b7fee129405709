"""Damped acoustic wave operator, its adjoint and the FWI gradient (oracle, FP64).

The PDE is Eq. 1 with the damping term of Listing 1,
``m u_tt - lap(u) + eta u_t = q``, zero initial state.  Listing 1 solves the
discrete equation for ``u.forward``; with the second-order leapfrog for ``u_tt``
and (reading) the centred difference for ``u_t`` this is, per time row k,

    a u^{k+1} - b u^k + c u^{k-1} = S^k,
    a = m/dt^2 + eta/(2 dt),  b = 2 m/dt^2 + L,  c = m/dt^2 - eta/(2 dt),

with ``L`` the Laplacian of Sec. IV-A1 (sum over axes of the centred second
derivatives of the chosen space order, zero ghost values outside the
computational grid) and ``S^k = P_s^T q^k`` the injected source.  The receiver
data of Eq. 2 are ``d^n = P_r u^n``, n = 0..nt-1, with ``u^{-1} = u^0 = 0``.

Listing 2 (adjoint: damping sign flipped, solved for the backward level, time
reversed) is the transpose of that block lower-triangular system: ``a`` and
``c`` are diagonal and ``b`` is symmetric, so for the adjoint field

    lam_{j-1} = (b lam_j - c lam_{j+1} + P_r^T y^j) / a,   j = nt-1 .. 1,
    lam_{nt-1} = lam_nt = 0,   (F^T y)^k = P_s lam_k  (k <= nt-2),  0 at nt-1.

The gradient of the objective of Eq. 2 by the adjoint-state method (Eq. 3-4),
with the index alignment and sign that the discrete system fixes, is

    grad = -(1/dt^2) sum_{j=1..nt-1} u^j (lam_{j-1} - 2 lam_j + lam_{j+1}),

computed on the computational grid and folded back onto the physical grid by the
transpose of the padding.  All arithmetic is float64, one plain step after
another, with library calls (NumPy slicing, scipy sparse products) as steps.

Test infrastructure only (see the package docstring).
"""

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .fd import fd_weights, radius
from .interp import interpolation_matrix
from .model import damping, fold_gradient, pad_model
from .snapshot import round_level


def _odd_pad(u, R):
    """Ghost values for a Dirichlet box: odd reflection about the virtual zero
    nodes at index -1 and n of every axis (test option only)."""
    out = u
    for ax in range(u.ndim):
        n = out.shape[ax]
        if n < R:
            raise ValueError("odd ghost needs at least R points per axis")
        zero = np.zeros_like(np.take(out, [0], axis=ax))
        lo = [zero] + [-np.take(out, [k - 2], axis=ax) for k in range(2, R + 1)]
        hi = [zero] + [-np.take(out, [n - k + 1], axis=ax) for k in range(2, R + 1)]
        out = np.concatenate(lo[::-1] + [out] + hi, axis=ax)
    return out


def laplacian(u, space_order, spacing, ghost="zero"):
    """Sum over axes of the centred second derivative of order ``space_order``.

    ``spacing`` is x-first; ``u`` is in array layout (axes reversed).
    ``ghost='zero'`` (the operator of the method) uses zero values outside the
    grid; ``ghost='odd'`` is the Dirichlet-box test variant.
    """
    u = np.asarray(u, dtype=np.float64)
    R = radius(space_order)
    w = fd_weights(space_order)
    nd = u.ndim
    if ghost == "zero":
        up = np.pad(u, R)
    elif ghost == "odd":
        up = _odd_pad(u, R)
    else:
        raise ValueError(ghost)
    L = np.zeros_like(u)
    for d in range(nd):
        ax = nd - 1 - d
        inv_h2 = 1.0 / float(spacing[d]) ** 2
        for j in range(-R, R + 1):
            sl = [slice(R, R + u.shape[a]) for a in range(nd)]
            sl[ax] = slice(R + j, R + j + u.shape[ax])
            L += (w[abs(j)] * inv_h2) * up[tuple(sl)]
    return L


@dataclass
class ForwardResult:
    d: np.ndarray            # (nt, n_rec) receiver data
    u_prev: np.ndarray       # u^{nt-2}
    u_last: np.ndarray       # u^{nt-1}
    history: list = None     # [u^0, ..., u^{nt-1}] when requested


def _coefficients(m, eta, dt):
    a = m / dt ** 2 + eta / (2.0 * dt)
    c = m / dt ** 2 - eta / (2.0 * dt)
    return a, c


def forward_op(m, eta, spacing, dt, nt, space_order, q, Ps, Pr,
               u_init_prev=None, u_init=None, save=False, ghost="zero"):
    """Forward leapfrog on the computational grid (``m``, ``eta`` in array layout).

    ``q`` is (nt, n_src) and enters row k as ``P_s^T q^k`` (k = 0..nt-2);
    returns receiver data ``d^n = P_r u^n`` for n = 0..nt-1.
    """
    m = np.asarray(m, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64).reshape(nt, -1)
    shape = m.shape
    a, c = _coefficients(m, eta, dt)
    u_prev = np.zeros(shape) if u_init_prev is None else np.array(u_init_prev, dtype=np.float64)
    u_cur = np.zeros(shape) if u_init is None else np.array(u_init, dtype=np.float64)
    d = np.zeros((nt, Pr.shape[0]))
    d[0] = Pr @ u_cur.ravel()
    history = [u_cur.copy()] if save else None
    for k in range(nt - 1):
        b_u = 2.0 * m / dt ** 2 * u_cur + laplacian(u_cur, space_order, spacing, ghost)
        S = (Ps.T @ q[k]).reshape(shape)
        u_next = (b_u - c * u_prev + S) / a
        d[k + 1] = Pr @ u_next.ravel()
        u_prev, u_cur = u_cur, u_next
        if save:
            history.append(u_cur.copy())
    return ForwardResult(d=d, u_prev=u_prev, u_last=u_cur, history=history)


def adjoint_op(m, eta, spacing, dt, nt, space_order, y, Ps, Pr, ghost="zero",
               u_history=None):
    """Adjoint sweep (Listing 2 read as the transpose of ``forward_op``).

    ``y`` is (nt, n_rec).  Returns ``(q_adj, grad_comp)`` where ``q_adj`` is
    (nt, n_src) = F^T y and ``grad_comp`` (only when ``u_history`` is given) is
    ``-(1/dt^2) sum_j u^j (lam_{j-1} - 2 lam_j + lam_{j+1})`` on the
    computational grid.
    """
    m = np.asarray(m, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(nt, -1)
    shape = m.shape
    a, c = _coefficients(m, eta, dt)
    lam_next = np.zeros(shape)   # lam_{j+1}
    lam_cur = np.zeros(shape)    # lam_j
    q_adj = np.zeros((nt, Ps.shape[0]))
    grad = np.zeros(shape) if u_history is not None else None
    for j in range(nt - 1, 0, -1):
        b_l = 2.0 * m / dt ** 2 * lam_cur + laplacian(lam_cur, space_order, spacing, ghost)
        rhs = (Pr.T @ y[j]).reshape(shape)
        lam_prev = (b_l - c * lam_next + rhs) / a          # lam_{j-1}
        q_adj[j - 1] = Ps @ lam_prev.ravel()
        if grad is not None:
            grad -= u_history[j] * (lam_prev - 2.0 * lam_cur + lam_next) / dt ** 2
        lam_next, lam_cur = lam_cur, lam_prev
    return q_adj, grad


# ---------------------------------------------------------------------------
# Physical-model wrappers (Listing 1 / Listing 2 call shape: model, nt, dt, h,
# space order; the geometry also carries origin, sponge width and points).
# ---------------------------------------------------------------------------

def operators(geom, src_coords, rec_coords):
    return interpolation_matrix(geom, src_coords), interpolation_matrix(geom, rec_coords)


def forward(geom, m_phys, dt, nt, space_order, q, src_coords, rec_coords, save=False):
    """Receiver data of the forward model for a physical squared-slowness model."""
    m = pad_model(geom, m_phys)
    Ps, Pr = operators(geom, src_coords, rec_coords)
    return forward_op(m, damping(geom), geom.spacing, dt, nt, space_order, q, Ps, Pr, save=save)


def adjoint(geom, m_phys, dt, nt, space_order, y, src_coords, rec_coords):
    """F^T y: adjoint source-side traces (nt, n_src) for receiver-side traces y."""
    m = pad_model(geom, m_phys)
    Ps, Pr = operators(geom, src_coords, rec_coords)
    q_adj, _ = adjoint_op(m, damping(geom), geom.spacing, dt, nt, space_order, y, Ps, Pr)
    return q_adj


def objective(geom, m_phys, dt, nt, space_order, q, src_coords, rec_coords, d_obs):
    """Eq. 2: 0.5 * || P_r A^{-1}(m) q - d_obs ||^2 over all n = 0..nt-1."""
    res = forward(geom, m_phys, dt, nt, space_order, q, src_coords, rec_coords)
    r = res.d - np.asarray(d_obs, dtype=np.float64)
    return 0.5 * float(np.sum(r * r))


def gradient(geom, m_phys, dt, nt, space_order, q, src_coords, rec_coords, d_obs, snapshot_rounding=None):
    """Eq. 3 gradient of Eq. 2 on the physical grid, and the objective value.

    ``snapshot_rounding`` ("bf16" or "fp16") evaluates the imaging condition on
    the stored forward levels u^1..u^{nt-1} as the 16-bit storage reads them
    back (``snapshot.round_level``); the forward and adjoint sweeps themselves
    are unchanged.
    """
    m = pad_model(geom, m_phys)
    eta = damping(geom)
    Ps, Pr = operators(geom, src_coords, rec_coords)
    fwd = forward_op(m, eta, geom.spacing, dt, nt, space_order, q, Ps, Pr, save=True)
    resid = fwd.d - np.asarray(d_obs, dtype=np.float64)
    phi = 0.5 * float(np.sum(resid * resid))
    history = fwd.history
    if snapshot_rounding is not None:
        history = [history[0]] + [round_level(u, snapshot_rounding) for u in history[1:]]
    _, g = adjoint_op(m, eta, geom.spacing, dt, nt, space_order, resid, Ps, Pr,
                      u_history=history)
    return fold_gradient(geom, g), phi


def identity_operator(shape):
    """Full-field restriction (every cell a point), for operator-level tests."""
    n = int(np.prod(shape))
    return sp.identity(n, format="csr", dtype=np.float64)


def born_op(m, eta, spacing, dt, nt, space_order, q, dm, Ps, Pr):
    """Linearised (Born) modelling J dm on the computational grid.

    Differentiating the rows ``a u^{k+1} - b u^k + c u^{k-1} = P_s^T q^k`` with
    respect to m in the direction dm (a, b, c depend on m through m/dt^2,
    2m/dt^2, m/dt^2) gives the scattered field
        a du^{k+1} - b du^k + c du^{k-1} = -dm (u^{k+1} - 2u^k + u^{k-1}) / dt^2
    with zero initial state, and the linearised data dd^n = P_r du^n.  The
    background u is the forward field of ``forward_op``.
    """
    m = np.asarray(m, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    dm = np.asarray(dm, dtype=np.float64)
    fwd = forward_op(m, eta, spacing, dt, nt, space_order, q, Ps, Pr, save=True)
    u = fwd.history
    shape = m.shape
    a, c = _coefficients(m, eta, dt)
    du_prev = np.zeros(shape)
    du_cur = np.zeros(shape)
    dd = np.zeros((nt, Pr.shape[0]))
    for k in range(nt - 1):
        u_prev = u[k - 1] if k >= 1 else np.zeros(shape)
        src = -dm * (u[k + 1] - 2.0 * u[k] + u_prev) / dt ** 2
        b_du = 2.0 * m / dt ** 2 * du_cur + laplacian(du_cur, space_order, spacing)
        du_next = (b_du - c * du_prev + src) / a
        dd[k + 1] = Pr @ du_next.ravel()
        du_prev, du_cur = du_cur, du_next
    return dd


def born(geom, m_phys, dm_phys, dt, nt, space_order, q, src_coords, rec_coords):
    """J dm for a physical model perturbation (padded like the model)."""
    m = pad_model(geom, m_phys)
    dm = pad_model(geom, dm_phys)
    Ps, Pr = operators(geom, src_coords, rec_coords)
    return born_op(m, damping(geom), geom.spacing, dt, nt, space_order, q, dm, Ps, Pr)
