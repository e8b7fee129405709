"""Pins for the oracle's time stepping (CPU only).

* a discrete standing mode in a Dirichlet box evolves exactly as cos(n theta),
  with cos(theta) fixed by the leapfrog and the Laplacian symbol (round-off);
* the same mode converges to the analytic cos(omega t) with order 2 in dt and
  order ``so`` in h;
* the CFL limit of the oracle matches the closed form of the 2D order-4 case
  and separates bounded from growing runs;
* a brute-force dense space-time solve, assembled independently from Kronecker
  products of 1D difference matrices, reproduces forward and adjoint.
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fd, interp, model, wave

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mode(shape_xyz, modes):
    """phi = prod_d sin(pi k_d (i_d+1)/(n_d+1)), array layout."""
    axes = [np.sin(np.pi * k * (np.arange(n) + 1) / (n + 1)) for n, k in zip(shape_xyz, modes)]
    phi = axes[-1]
    for a in axes[-2::-1]:
        phi = np.multiply.outer(phi, a)
    return phi


def _keff2(so, shape_xyz, modes, spacing):
    w = fd.fd_weights(so)
    R = so // 2
    s = 0.0
    for n, k, h in zip(shape_xyz, modes, spacing):
        th = np.pi * k / (n + 1)
        s += (-w[0] - 2 * sum(w[j] * np.cos(j * th) for j in range(1, R + 1))) / h ** 2
    return s


@pytest.mark.parametrize("so,ndim", [(2, 2), (4, 2), (8, 3), (16, 2), (12, 3)])
def test_standing_mode_exact(so, ndim):
    shape = [23, 19, 17][:ndim]
    spacing = [10.0, 12.0, 9.0][:ndim]
    modes = [2, 3, 1][:ndim]
    v, dt, nt = 2.0, 0.8, 60
    phi = _mode(shape, modes)
    k2 = _keff2(so, shape, modes, spacing)
    cos_th = 1.0 - 0.5 * dt * dt * v * v * k2
    th = np.arccos(cos_th)
    m = np.full(phi.shape, 1.0 / v ** 2)
    P = wave.identity_operator(phi.shape)
    res = wave.forward_op(m, np.zeros_like(m), spacing, dt, nt, so, np.zeros((nt, 0)),
                          sp.csr_matrix((0, phi.size)), P,
                          u_init_prev=np.cos(th) * phi, u_init=phi, ghost="odd")
    for n in range(nt):
        np.testing.assert_allclose(res.d[n], np.cos(n * th) * phi.ravel(), rtol=0, atol=1e-11)


def _analytic_error(so, n_inner, dt, T=60.0, box=200.0, v=1.5):
    spacing = [box / (n_inner + 1)] * 2
    shape = [n_inner, n_inner]
    phi = _mode(shape, [1, 1])
    omega = v * np.pi / box * np.sqrt(2.0)
    nt = int(round(T / dt)) + 1
    m = np.full(phi.shape, 1.0 / v ** 2)
    res = wave.forward_op(m, np.zeros_like(m), spacing, dt, nt, so, np.zeros((nt, 0)),
                          sp.csr_matrix((0, phi.size)), sp.csr_matrix((0, phi.size)),
                          u_init_prev=np.cos(omega * dt) * phi, u_init=phi, ghost="odd")
    return np.abs(res.u_last - np.cos(omega * (nt - 1) * dt) * phi).max()


def test_convergence_second_order_in_time():
    # h = 5 m, so = 16, v = 1.5: dt_max ~ 1.7 ms, so both steps are stable
    e1 = _analytic_error(16, 39, 1.0)
    e2 = _analytic_error(16, 39, 0.5)
    slope = np.log2(e1 / e2)
    assert 1.8 < slope < 2.2, (e1, e2, slope)


@pytest.mark.parametrize("so", [2, 4])
def test_convergence_in_space(so):
    dt = 0.01
    e1 = _analytic_error(so, 9, dt, T=20.0)
    e2 = _analytic_error(so, 19, dt, T=20.0)
    slope = np.log(e1 / e2) / np.log(20.0 / 10.0)
    assert slope > so - 0.3, (e1, e2, slope)


def test_cfl_closed_form_2d_order4():
    vals = [float(l) for l in open(os.path.join(GOLDEN, "cfl_2d_so4.txt")) if l.strip() and l[0] != "#"]
    assert abs(model.dt_max(4, (10.0, 10.0), 1.5) - vals[0]) < 1e-12


@pytest.mark.parametrize("so", [2, 8])
def test_cfl_separates_stable_and_unstable(so):
    shape, spacing, v = [30, 30], [10.0, 10.0], 2.0
    dtm = model.dt_max(so, spacing, v)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(shape[::-1])
    m = np.full(u0.shape, 1.0 / v ** 2)
    empty = sp.csr_matrix((0, u0.size))

    def amp(dt, ghost, steps):
        r = wave.forward_op(m, np.zeros_like(m), spacing, dt, steps, so, np.zeros((steps, 0)),
                            empty, empty, u_init_prev=u0, u_init=u0, ghost=ghost)
        return np.abs(r.u_last).max()

    assert amp(0.98 * dtm, "zero", 400) < 50 * np.abs(u0).max()
    # in the Dirichlet box the highest mode sits within 0.3% of the bound,
    # so 5% above the limit it grows by ~1.8 per step
    assert amp(1.05 * dtm, "odd", 100) > 1e10 * np.abs(u0).max()


# --------------------------------------------------------------------------
# brute force: dense space-time system built from 1D matrices
# --------------------------------------------------------------------------

def _lap_matrix(comp_shape_xyz, spacing, so):
    """Laplacian with zero ghosts as a sum of Kronecker products (x fastest)."""
    w = fd.fd_weights(so)
    R = so // 2
    nd = len(comp_shape_xyz)
    L = None
    for d in range(nd):
        n = comp_shape_xyz[d]
        D = sum(sp.eye(n, k=j) * w[abs(j)] for j in range(-R, R + 1)) / spacing[d] ** 2
        mats = [sp.eye(comp_shape_xyz[e]) for e in range(nd)]
        mats[d] = D
        K = mats[nd - 1]
        for e in range(nd - 2, -1, -1):
            K = sp.kron(K, mats[e])
        L = K if L is None else L + K
    return L.toarray()


def _space_time(geom, m_phys, dt, nt, so):
    m = model.pad_model(geom, m_phys).ravel()
    eta = model.damping(geom).ravel()
    a = m / dt ** 2 + eta / (2 * dt)
    c = m / dt ** 2 - eta / (2 * dt)
    B = np.diag(2 * m / dt ** 2) + _lap_matrix(geom.comp_shape, geom.spacing, so)
    N = m.size
    T = nt - 1                       # unknowns u^1 .. u^{nt-1}
    A = np.zeros((T * N, T * N))
    for k in range(T):               # row k determines u^{k+1}
        A[k * N:(k + 1) * N, k * N:(k + 1) * N] = np.diag(a)
        if k >= 1:
            A[k * N:(k + 1) * N, (k - 1) * N:k * N] = -B
        if k >= 2:
            A[k * N:(k + 1) * N, (k - 2) * N:(k - 1) * N] = np.diag(c)
    return A, N


def _tiny_case(so=4):
    geom = model.Geometry(shape=(5, 4), spacing=(10.0, 8.0), origin=(0.0, 0.0), nbl=2, sponge_vref=2.0)
    rng = np.random.default_rng(5)
    m_phys = 1.0 / rng.uniform(1.5, 2.5, size=geom.phys_array_shape) ** 2
    src = np.array([[13.0, 9.5]])
    rec = np.array([[0.0, 0.0], [40.0, 24.0], [21.3, 11.1], [33.0, 3.0]])
    dt = 0.5 * model.dt_max(so, geom.spacing, 2.5)
    return geom, m_phys, src, rec, dt


def test_bruteforce_forward_and_adjoint():
    so, nt = 4, 9
    geom, m_phys, src, rec, dt = _tiny_case(so)
    A, N = _space_time(geom, m_phys, dt, nt, so)
    Ps = interp.interpolation_matrix(geom, src).toarray()
    Pr = interp.interpolation_matrix(geom, rec).toarray()
    rng = np.random.default_rng(9)
    q = rng.standard_normal((nt, 1))
    rhs = np.concatenate([Ps.T @ q[k] for k in range(nt - 1)])
    U = np.linalg.solve(A, rhs).reshape(nt - 1, N)
    d_dense = np.vstack([np.zeros(len(rec))] + [Pr @ U[k] for k in range(nt - 1)])
    d_orc = wave.forward(geom, m_phys, dt, nt, so, q, src, rec).d
    np.testing.assert_allclose(d_orc, d_dense, rtol=1e-11, atol=1e-13 * np.abs(d_dense).max())
    # adjoint: A^T lam = P_r^T y^j (unknown u^j is column block j-1)
    y = rng.standard_normal((nt, len(rec)))
    rhs_a = np.concatenate([Pr.T @ y[j] for j in range(1, nt)])
    lam = np.linalg.solve(A.T, rhs_a).reshape(nt - 1, N)    # block k = multiplier of row k
    q_dense = np.vstack([Ps @ lam[k] for k in range(nt - 1)] + [np.zeros(1)])
    q_orc = wave.adjoint(geom, m_phys, dt, nt, so, y, src, rec)
    np.testing.assert_allclose(q_orc, q_dense, rtol=1e-11, atol=1e-13 * np.abs(q_dense).max())


def test_bruteforce_gradient_by_finite_differences():
    so, nt = 4, 10
    geom, m_phys, src, rec, dt = _tiny_case(so)
    rng = np.random.default_rng(21)
    q = rng.standard_normal((nt, 1))
    d_obs = rng.standard_normal((nt, len(rec))) * 1e-3
    g, phi = wave.gradient(geom, m_phys, dt, nt, so, q, src, rec, d_obs)
    assert abs(phi - wave.objective(geom, m_phys, dt, nt, so, q, src, rec, d_obs)) < 1e-14 * phi
    eps = 1e-6 * m_phys.mean()
    fd_g = np.zeros_like(m_phys)
    for idx in np.ndindex(m_phys.shape):
        mp = m_phys.copy(); mp[idx] += eps
        mm = m_phys.copy(); mm[idx] -= eps
        fd_g[idx] = (wave.objective(geom, mp, dt, nt, so, q, src, rec, d_obs)
                     - wave.objective(geom, mm, dt, nt, so, q, src, rec, d_obs)) / (2 * eps)
    np.testing.assert_allclose(g, fd_g, rtol=1e-5, atol=1e-6 * np.abs(fd_g).max())
