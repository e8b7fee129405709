"""Pins for the oracle's adjoint, gradient, interpolation and model set-up (CPU).

* adjoint dot-product test of Eq. 5-6, <F q, y> = <q, F^T y>, to 1e-12 relative
  (sparse points and full-field operators, damping on, 2D and 3D);
* Taylor test of Eq. 7-8 over h in [1e-6, 1]: first-order and second-order
  decay of the remainders;
* multilinear interpolation reproduces linear fields exactly, samples nodes
  exactly, and rejects points outside the domain;
* padding/fold adjointness, sponge closed form, Ricker closed-form features.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import interp, model, wave


def _geom(ndim, nbl=4):
    if ndim == 2:
        return model.Geometry(shape=(17, 13), spacing=(10.0, 8.0), origin=(5.0, -3.0), nbl=nbl, sponge_vref=2.5)
    return model.Geometry(shape=(11, 9, 8), spacing=(10.0, 12.0, 9.0), origin=(0.0, 0.0, 0.0), nbl=nbl,
                          sponge_vref=2.5)


def _case(ndim, so, seed=0, nsrc=2, nrec=7):
    geom = _geom(ndim)
    rng = np.random.default_rng(seed)
    m = 1.0 / rng.uniform(1.5, 2.5, size=geom.phys_array_shape) ** 2
    lo = np.array(geom.origin)
    hi = lo + (np.array(geom.shape) - 1) * np.array(geom.spacing)
    src = lo + rng.uniform(size=(nsrc, ndim)) * (hi - lo)
    rec = lo + rng.uniform(size=(nrec, ndim)) * (hi - lo)
    dt = 0.5 * model.dt_max(so, geom.spacing, 2.5)
    return geom, m, src, rec, dt


@pytest.mark.parametrize("ndim,so", [(2, 2), (2, 4), (2, 16), (3, 8), (3, 4)])
def test_dot_product_sparse_points(ndim, so):
    nt = 40
    geom, m, src, rec, dt = _case(ndim, so)
    rng = np.random.default_rng(1)
    q = rng.standard_normal((nt, len(src)))
    y = rng.standard_normal((nt, len(rec)))
    d = wave.forward(geom, m, dt, nt, so, q, src, rec).d
    qa = wave.adjoint(geom, m, dt, nt, so, y, src, rec)
    lhs, rhs = np.sum(d * y), np.sum(q * qa)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("ndim,so", [(2, 6), (3, 2)])
def test_dot_product_full_field(ndim, so):
    nt = 25
    geom, m, _, _, dt = _case(ndim, so)
    mc = model.pad_model(geom, m)
    eta = model.damping(geom)
    P = wave.identity_operator(mc.shape)
    rng = np.random.default_rng(2)
    q = rng.standard_normal((nt, mc.size))
    y = rng.standard_normal((nt, mc.size))
    d = wave.forward_op(mc, eta, geom.spacing, dt, nt, so, q, P, P).d
    qa, _ = wave.adjoint_op(mc, eta, geom.spacing, dt, nt, so, y, P, P)
    lhs, rhs = np.sum(d * y), np.sum(q * qa)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("ndim,so", [(2, 4), (3, 8)])
def test_taylor(ndim, so):
    nt = 60
    geom, m0, src, rec, dt = _case(ndim, so, seed=4, nsrc=1, nrec=9)
    rng = np.random.default_rng(8)
    q = rng.standard_normal((nt, 1))
    # observed data from a perturbed "true" model
    m_true = m0 * (1.0 + 0.05 * rng.uniform(-1, 1, size=m0.shape))
    d_obs = wave.forward(geom, m_true, dt, nt, so, q, src, rec).d
    g, phi0 = wave.gradient(geom, m0, dt, nt, so, q, src, rec, d_obs)
    dm = 0.05 * m0 * rng.uniform(-1, 1, size=m0.shape)
    hs = 10.0 ** np.arange(0, -7, -1, dtype=np.float64)
    e1, e2 = [], []
    gdm = float(np.sum(g * dm))
    for h in hs:
        phi = wave.objective(geom, m0 + h * dm, dt, nt, so, q, src, rec, d_obs)
        e1.append(abs(phi - phi0))
        e2.append(abs(phi - phi0 - h * gdm))
    e1, e2 = np.array(e1), np.array(e2)
    s1 = np.diff(np.log10(e1)) / np.diff(np.log10(hs))
    s2 = np.diff(np.log10(e2)) / np.diff(np.log10(hs))
    # first-order remainder: slope 1 once h*dm is in the linear regime (h <= 1e-1)
    assert np.all(np.abs(s1[1:] - 1.0) < 0.25), s1
    assert np.all(np.abs(s1[3:] - 1.0) < 0.01), s1
    # second-order remainder: slope 2 until it meets FP64 round-off of phi
    ok = e2[1:] > 1e3 * np.finfo(float).eps * phi0
    assert ok.sum() >= 3
    assert np.all(np.abs(s2[ok] - 2.0) < 0.15), (s2, e2)


@pytest.mark.parametrize("ndim", [2, 3])
def test_interpolation_linear_exact_and_nodes(ndim):
    geom = _geom(ndim)
    rng = np.random.default_rng(3)
    lo = np.array(geom.origin)
    hi = lo + (np.array(geom.shape) - 1) * np.array(geom.spacing)
    pts = lo + rng.uniform(size=(50, ndim)) * (hi - lo)
    pts = np.vstack([pts, lo, hi])          # first and last physical nodes
    P = interp.interpolation_matrix(geom, pts)
    coef = rng.standard_normal(ndim + 1)
    axes = [geom.comp_origin[d] + np.arange(geom.comp_shape[d]) * geom.spacing[d] for d in range(ndim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    field = coef[0] + sum(coef[d + 1] * grids[d] for d in range(ndim))
    exact = coef[0] + pts @ coef[1:]
    np.testing.assert_allclose(interp.sample(P, field), exact, rtol=1e-12, atol=1e-10)
    # rows are partitions of unity
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, rtol=1e-14)
    # transpose identity
    u = rng.standard_normal(geom.array_shape)
    v = rng.standard_normal(len(pts))
    assert abs(np.dot(interp.sample(P, u), v) - np.sum(u * interp.inject(P, v, u.shape))) < 1e-11


def test_interpolation_last_node_with_no_sponge():
    geom = model.Geometry(shape=(6, 5), spacing=(2.0, 3.0), nbl=0)
    pts = np.array([[10.0, 12.0], [10.0, 0.0]])
    P = interp.interpolation_matrix(geom, pts).toarray()
    u = np.arange(30, dtype=float).reshape(5, 6)
    np.testing.assert_allclose(P @ u.ravel(), [u[4, 5], u[0, 5]])


def test_interpolation_rejects_outside():
    geom = _geom(2)
    with pytest.raises(ValueError):
        interp.interpolation_matrix(geom, np.array([[4.9, 0.0]]))
    with pytest.raises(ValueError):
        interp.interpolation_matrix(geom, np.array([[10.0, 200.0]]))


@pytest.mark.parametrize("ndim", [2, 3])
def test_pad_fold_adjoint(ndim):
    geom = _geom(ndim, nbl=3)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(geom.phys_array_shape)
    y = rng.standard_normal(geom.array_shape)
    px = model.pad_model(geom, x)
    assert abs(np.sum(px * y) - np.sum(x * model.fold_gradient(geom, y))) < 1e-10
    # edge replication: corner of the padded grid equals the physical corner
    assert px[(0,) * ndim] == x[(0,) * ndim]
    assert px[(-1,) * ndim] == x[(-1,) * ndim]


def test_sponge_closed_form():
    geom = model.Geometry(shape=(30, 20), spacing=(10.0, 5.0), nbl=10, sponge_vref=2.0)
    eta = model.damping(geom)
    inner = eta[10:-10, 10:-10]
    assert np.all(inner == 0.0)
    emx = 3 * 2.0 * np.log(1000.0) / (2 * 10 * 10.0)
    emz = 3 * 2.0 * np.log(1000.0) / (2 * 10 * 5.0)
    # outermost x point in the middle of z: delta_x = nbl
    assert abs(eta[20, 0] - emx) < 1e-14 and abs(eta[20, -1] - emx) < 1e-14
    assert abs(eta[0, 20] - emz) < 1e-14
    assert abs(eta[0, 0] - (emx + emz)) < 1e-14
    # first layer point next to the interior: delta = 1
    assert abs(eta[20, 9] - emx / 100.0) < 1e-15


def test_ricker_closed_form_features():
    f0, dt = 0.010, 0.5
    r = model.ricker(2001, dt, f0)
    t0 = 1.0 / f0
    assert abs(r[int(round(t0 / dt))] - 1.0) < 1e-15
    tz = t0 + 1.0 / (np.pi * f0 * np.sqrt(2.0))
    rz = model.ricker(1, 1.0, f0, t0=t0 - tz)      # value at t = tz
    assert abs(rz[0]) < 1e-14
    # zero mean over the real line (window centred on the peak)
    rc = model.ricker(2001, dt, f0, t0=500.0)
    assert abs(rc.sum() * dt) < 1e-9


def test_sponge_profile_shape_and_absorption():
    """Quadratic growth into the layer, additivity at corners, and a reflected
    energy far below that of the same grid with the damping switched off."""
    geom = model.Geometry(shape=(41, 41), spacing=(10.0, 10.0), nbl=30, sponge_vref=1.5)
    eta = model.damping(geom)
    row = eta[50, :30][::-1]                      # delta = 1..30 on the low-x side
    np.testing.assert_allclose(row / row[0], np.arange(1, 31) ** 2, rtol=1e-12)
    assert abs(eta[0, 0] - (eta[50, 0] + eta[0, 50])) < 1e-15
    so, nt = 4, 700
    dt = 0.5 * model.dt_max(so, geom.spacing, 1.5)
    m = model.pad_model(geom, np.full(geom.phys_array_shape, 1.0 / 1.5 ** 2))
    src = np.array([[200.0, 200.0]])
    Ps = interp.interpolation_matrix(geom, src)
    q = model.ricker(nt, dt, 0.02)[:, None]
    empty = sp.csr_matrix((0, m.size))
    inner = (slice(30, 71), slice(30, 71))
    e_damped = np.sum(wave.forward_op(m, eta, geom.spacing, dt, nt, so, q, Ps, empty).u_last[inner] ** 2)
    e_free = np.sum(wave.forward_op(m, 0 * eta, geom.spacing, dt, nt, so, q, Ps, empty).u_last[inner] ** 2)
    assert e_damped < 1e-2 * e_free, (e_damped, e_free)


@pytest.mark.parametrize("ndim", [2, 3])
def test_windowed_model_and_damping_equal_crops(ndim):
    geom = _geom(ndim, nbl=3)
    rng = np.random.default_rng(12)
    m = rng.uniform(0.1, 0.4, size=geom.phys_array_shape)
    full_m = model.pad_model(geom, m)
    full_e = model.damping(geom)
    win = [(0, 4), (2, 9), (1, 7)][:ndim]
    win = [(a, min(b, n)) for (a, b), n in zip(win, geom.array_shape)]
    sl = tuple(slice(a, b) for a, b in win)
    np.testing.assert_array_equal(model.pad_model(geom, m, window=win), full_m[sl])
    np.testing.assert_array_equal(model.damping(geom, window=win), full_e[sl])


@pytest.mark.parametrize("ndim,so", [(2, 4), (3, 8)])
def test_born_is_the_derivative_of_the_forward_map(ndim, so):
    """J dm against central differences of F (error O(eps^2)) and against the
    gradient through <J dm, y> = <dm, J^T y> (J^T y: gradient with residual y)."""
    nt = 50
    geom, m, src, rec, dt = _case(ndim, so, seed=12, nsrc=1, nrec=8)
    rng = np.random.default_rng(13)
    q = rng.standard_normal((nt, 1))
    dm = 0.1 * m * rng.uniform(-1, 1, size=m.shape)
    jd = wave.born(geom, m, dm, dt, nt, so, q, src, rec)
    errs = []
    for eps in (1e-2, 5e-3):
        fp = wave.forward(geom, m + eps * dm, dt, nt, so, q, src, rec).d
        fm = wave.forward(geom, m - eps * dm, dt, nt, so, q, src, rec).d
        errs.append(np.linalg.norm((fp - fm) / (2 * eps) - jd) / np.linalg.norm(jd))
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 3.5, errs
    y = rng.standard_normal((nt, len(rec)))
    d_pred = wave.forward(geom, m, dt, nt, so, q, src, rec).d
    jty, _ = wave.gradient(geom, m, dt, nt, so, q, src, rec, d_pred - y)
    lhs, rhs = np.sum(jd * y), np.sum(dm * jty)
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs)), (lhs, rhs)
