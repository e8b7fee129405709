"""Model set-up for the oracle (FP64): geometry, padding, sponge, CFL, Ricker.

Conventions (shared with the CUDA library by specification, not by code):

* Axis ``d = 0`` is x (fastest in memory), ``d = 1`` is y in 3D or z (depth) in
  2D, ``d = 2`` is z (depth) in 3D.  NumPy arrays are stored C-order with the
  axes reversed: 3D fields have shape ``(n_z, n_y, n_x)``, 2D fields
  ``(n_z, n_x)``.
* Units: spacing in m, time in ms, velocity in km/s (= m/ms), so the squared
  slowness ``m = 1/v**2`` is in s**2/km**2 (= ms**2/m**2).
* Sec. V-D adds the absorbing layer outside the physical model on every side:
  the computational grid has ``n_d = N_d + 2*nbl`` points per axis, and its node
  0 sits at ``origin_d - nbl*h_d``.

Readings of points the paper leaves open (each is one explicit choice):

* the model inside the sponge is the edge value of the physical model
  (edge replication); the gradient is folded back by the transpose of that map;
* the damping ``eta`` of Listing 1 is a quadratic sponge summed over axes,
  ``eta = sum_d eta_max_d * (delta_d/nbl)**2`` with ``delta_d`` the number of
  points into the layer (1..nbl) and ``eta_max_d = 3 v_ref ln(1/R_c)/(2 nbl h_d)``,
  ``R_c = 1e-3``; ``v_ref`` is a fixed geometry parameter so that ``eta`` does
  not depend on ``m`` (otherwise the gradient of Eq. 3 would miss a term);
* the Ricker wavelet of Sec. V-D is the standard one with peak time ``t0``
  (default ``1/f0``).

Test infrastructure only (see the package docstring).
"""

from dataclasses import dataclass, field
from math import log

import numpy as np

from .fd import fd_weights

REFLECTION_COEFF = 1e-3


@dataclass
class Geometry:
    """Physical grid + absorbing layer; per-axis lists are x-first."""
    shape: tuple            # physical points per axis, x-first (N_x, [N_y,] N_z)
    spacing: tuple          # h per axis, m
    origin: tuple = None    # physical coordinate of node 0 per axis, m
    nbl: int = 0            # absorbing points added on every side
    sponge_vref: float = 1.5  # km/s, sets the sponge strength
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.spacing = tuple(float(h) for h in self.spacing)
        if self.origin is None:
            self.origin = (0.0,) * len(self.shape)
        self.origin = tuple(float(o) for o in self.origin)
        if len(self.shape) not in (2, 3):
            raise ValueError("ndim must be 2 or 3")
        if not (len(self.spacing) == len(self.origin) == len(self.shape)):
            raise ValueError("shape, spacing, origin must have the same length")

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def comp_shape(self):
        """Computational points per axis, x-first."""
        return tuple(n + 2 * self.nbl for n in self.shape)

    @property
    def comp_origin(self):
        return tuple(o - self.nbl * h for o, h in zip(self.origin, self.spacing))

    @property
    def array_shape(self):
        """NumPy shape of a computational field (axes reversed)."""
        return self.comp_shape[::-1]

    @property
    def phys_array_shape(self):
        return self.shape[::-1]


def pad_model(geom, m_phys, window=None):
    """Extend the physical model by ``nbl`` points on every side by edge replication.

    ``window`` (optional): per array axis ``(start, stop)`` on the computational
    grid; only that block of the padded model is formed (same values)."""
    m_phys = np.asarray(m_phys)
    if m_phys.shape != geom.phys_array_shape:
        raise ValueError("model shape %r != %r" % (m_phys.shape, geom.phys_array_shape))
    if window is None:
        return np.pad(m_phys.astype(np.float64), geom.nbl, mode="edge")
    idx = [np.clip(np.arange(a, b) - geom.nbl, 0, n - 1) for (a, b), n in zip(window, m_phys.shape)]
    return m_phys[np.ix_(*idx)].astype(np.float64)


def fold_gradient(geom, g_comp):
    """Transpose of ``pad_model``: every computational cell adds into the physical
    cell it was replicated from."""
    g = np.asarray(g_comp, dtype=np.float64)
    if g.shape != geom.array_shape:
        raise ValueError("gradient shape %r != %r" % (g.shape, geom.array_shape))
    nbl = geom.nbl
    out = g
    for ax in range(g.ndim):
        n_comp = out.shape[ax]
        n_phys = n_comp - 2 * nbl
        # computational index i was copied from physical index clip(i - nbl)
        src = np.clip(np.arange(n_comp) - nbl, 0, n_phys - 1)
        moved = np.moveaxis(out, ax, 0)
        acc = np.zeros((n_phys,) + moved.shape[1:], dtype=np.float64)
        np.add.at(acc, src, moved)
        out = np.moveaxis(acc, 0, ax)
    return out


def sponge_depth(n, nbl):
    """Points into the absorbing layer along one axis: nbl..1 on the low side,
    1..nbl on the high side, 0 inside."""
    i = np.arange(n)
    d = np.zeros(n, dtype=np.float64)
    if nbl > 0:
        lo = i < nbl
        hi = i >= n - nbl
        d[lo] = nbl - i[lo]
        d[hi] = i[hi] - (n - nbl) + 1
    return d


def damping(geom, window=None):
    """Sponge damping eta (1/ms) on the computational grid, array layout
    (optionally only the block ``window``, per array axis ``(start, stop)``)."""
    nd = geom.ndim
    if window is None:
        window = [(0, n) for n in geom.array_shape]
    eta = np.zeros(tuple(b - a for a, b in window), dtype=np.float64)
    if geom.nbl == 0:
        return eta
    for d in range(nd):
        ax = nd - 1 - d
        n = geom.comp_shape[d]
        eta_max = 3.0 * geom.sponge_vref * log(1.0 / REFLECTION_COEFF) / (2.0 * geom.nbl * geom.spacing[d])
        a, b = window[ax]
        prof = eta_max * (sponge_depth(n, geom.nbl)[a:b] / geom.nbl) ** 2
        shape = [1] * nd
        shape[ax] = b - a
        eta = eta + prof.reshape(shape)
    return eta


def dt_max(space_order, spacing, v_max):
    """Von Neumann limit of the undamped leapfrog scheme: the time step at which
    dt**2 v**2 max(-L) reaches 4, with max(-L) = sum_d (sum_j |w_j|) / h_d**2."""
    w = fd_weights(space_order)
    abs_sum = abs(w[0]) + 2.0 * np.abs(w[1:]).sum()
    lam = sum(abs_sum / float(h) ** 2 for h in spacing)
    return 2.0 / (float(v_max) * np.sqrt(lam))


def ricker(nt, dt, f0, t0=None):
    """Ricker wavelet sampled at t_n = n*dt, n = 0..nt-1 (f0 in kHz, dt in ms)."""
    if t0 is None:
        t0 = 1.0 / f0
    t = np.arange(nt, dtype=np.float64) * dt
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)
