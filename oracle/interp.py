"""Sparse-point interpolation for source injection and receiver sampling (FP64).

Sec. IV names sparse-point interpolation (source insertion, receiver sampling)
as a feature the stencil abstraction alone cannot express; Listing 3 elides the
code.  The reading taken here: multilinear interpolation on the computational
grid (bilinear in 2D, trilinear in 3D).  Per axis d, with
``t = (p_d - o_d)/h_d`` relative to computational node 0, ``i = floor(t)`` and
``f = t - i``; a point exactly on the last node uses ``i = n_d - 2, f = 1`` so
both corners exist.  The weight of corner ``(i_d + b_d)_d`` is
``prod_d (f_d if b_d else 1 - f_d)``.  Points outside the physical domain are
rejected.

The restriction operator ``P`` (rows = points, columns = flattened grid cells)
is a scipy sparse matrix: receiver sampling is ``P @ u``, source injection is
``P.T @ q``, so injection is the exact transpose of sampling by construction.

Test infrastructure only (see the package docstring).
"""

import numpy as np
import scipy.sparse as sp


def _check_inside(geom, coords):
    for d in range(geom.ndim):
        lo = geom.origin[d]
        hi = geom.origin[d] + (geom.shape[d] - 1) * geom.spacing[d]
        c = coords[:, d]
        if np.any(c < lo) or np.any(c > hi):
            raise ValueError("point outside the physical domain along axis %d" % d)


def interpolation_matrix(geom, coords):
    """Sparse (n_points x n_cells) multilinear restriction operator."""
    coords = np.asarray(coords, dtype=np.float64).reshape(-1, geom.ndim)
    _check_inside(geom, coords)
    nd = geom.ndim
    n = geom.comp_shape
    o = geom.comp_origin
    strides = [1] * nd
    for d in range(1, nd):
        strides[d] = strides[d - 1] * n[d - 1]
    npts = coords.shape[0]
    base = np.zeros(npts, dtype=np.int64)
    frac = np.zeros((npts, nd), dtype=np.float64)
    for d in range(nd):
        t = (coords[:, d] - o[d]) / geom.spacing[d]
        i = np.floor(t).astype(np.int64)
        last = i >= n[d] - 1
        i[last] = n[d] - 2
        frac[:, d] = t - i
        base += i * strides[d]
    rows, cols, vals = [], [], []
    for corner in range(2 ** nd):
        w = np.ones(npts, dtype=np.float64)
        idx = base.copy()
        for d in range(nd):
            if (corner >> d) & 1:
                w = w * frac[:, d]
                idx += strides[d]
            else:
                w = w * (1.0 - frac[:, d])
        rows.append(np.arange(npts))
        cols.append(idx)
        vals.append(w)
    ncells = int(np.prod(n))
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(npts, ncells))
    return P.tocsr()


def sample(P, u):
    """Values of the field ``u`` (array layout) at the points of ``P``."""
    return P @ np.asarray(u, dtype=np.float64).ravel()


def inject(P, values, array_shape):
    """Field ``P.T @ values`` (the transpose of ``sample``)."""
    return (P.T @ np.asarray(values, dtype=np.float64)).reshape(array_shape)
