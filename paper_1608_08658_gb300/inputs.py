"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle.

This module holds no arithmetic of the wave method itself (no stencil weights,
no time stepping, no CFL limit, no wavelet): only velocity models, point
positions and random traces, drawn from NumPy's PCG64 generator with explicit
seeds.  Coordinates are x-first per point; model arrays are C-order with the
axes reversed ((n_z, n_y, n_x) in 3D, (n_z, n_x) in 2D); velocities are km/s
and the squared slowness is ``1/v**2``.
"""

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def slowness2(v):
    """Squared slowness m = 1/v^2 (float32) from a velocity array in km/s."""
    v = np.asarray(v, dtype=np.float64)
    return (1.0 / (v * v)).astype(np.float32)


def _depth_axis(shape_xyz, spacing):
    nd = len(shape_xyz)
    nz = shape_xyz[-1]
    z = np.arange(nz, dtype=np.float64) * spacing[-1]
    return z.reshape((nz,) + (1,) * (nd - 1))


def constant_velocity(shape_xyz, v):
    return np.full(tuple(shape_xyz)[::-1], float(v), dtype=np.float64)


def smooth_gaussian_noise(shape_xyz, corr_len_points, seed):
    """Unit-variance white noise smoothed by a Gaussian kernel of standard
    deviation ``corr_len_points`` grid points, renormalised to unit std."""
    from scipy.ndimage import gaussian_filter
    g = rng(seed).standard_normal(tuple(shape_xyz)[::-1], dtype=np.float32)
    g = gaussian_filter(g, sigma=float(corr_len_points), mode="wrap")
    g -= g.mean(dtype=np.float64)
    g /= g.std(dtype=np.float64)
    return g


def two_layer_random_velocity(shape_xyz, spacing, v_top=1.5, v_bottom=2.5, interface=None,
                              sigma=0.05, corr_len=50.0, seed=7):
    """Two layers split at ``interface`` metres depth (default: mid-depth), times
    ``1 + sigma * g`` with g smoothed Gaussian noise of correlation length
    ``corr_len`` metres."""
    nz = shape_xyz[-1]
    if interface is None:
        interface = 0.5 * (nz - 1) * spacing[-1]
    z = _depth_axis(shape_xyz, spacing)
    v = np.where(z < interface, v_top, v_bottom) * np.ones(tuple(shape_xyz)[::-1])
    if sigma:
        g = smooth_gaussian_noise(shape_xyz, corr_len / spacing[0], seed)
        v = v * (1.0 + sigma * g)
    return v


def linear_gradient_velocity(shape_xyz, spacing, v0=1.5, k=0.6):
    """v(z) = v0 + k * z[km]."""
    z = _depth_axis(shape_xyz, spacing)
    return (v0 + k * z / 1000.0) * np.ones(tuple(shape_xyz)[::-1])


def gaussian_anomalies(shape_xyz, spacing, n=3, amp=0.2, sigma_m=150.0, seed=11):
    """Sum of ``n`` Gaussian blobs of amplitude +-amp km/s at seeded positions."""
    r = rng(seed)
    nd = len(shape_xyz)
    ext = [(s - 1) * h for s, h in zip(shape_xyz, spacing)]
    axes = [np.arange(s, dtype=np.float64) * h for s, h in zip(shape_xyz, spacing)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]   # x-first list of arrays
    out = np.zeros(tuple(shape_xyz)[::-1])
    for _ in range(n):
        c = [r.uniform(0.25 * e, 0.75 * e) for e in ext]
        s = amp if r.uniform() < 0.5 else -amp
        d2 = sum((grids[d] - c[d]) ** 2 for d in range(nd))
        out += s * np.exp(-d2 / (2.0 * sigma_m ** 2))
    return out


def layered_velocity(shape_xyz, spacing, n_layers, v_min=1.5, v_max=4.5, perturb=0.05, seed=0):
    """``n_layers`` flat layers with sorted velocities drawn in [v_min, v_max],
    interfaces at sorted random depths, each layer scaled by 1 + U(-perturb, perturb)."""
    r = rng(seed)
    nz = shape_xyz[-1]
    depth = (nz - 1) * spacing[-1]
    vs = np.sort(r.uniform(v_min, v_max, size=n_layers))
    vs[0] = v_min
    cuts = np.sort(r.uniform(0.05 * depth, 0.95 * depth, size=n_layers - 1))
    z = _depth_axis(shape_xyz, spacing)
    v = np.full(z.shape, vs[0])
    for i, c in enumerate(cuts):
        v = np.where(z >= c, vs[i + 1], v)
    v = v * (1.0 + r.uniform(-perturb, perturb, size=v.shape))
    v = np.clip(v, v_min, v_max)
    return v * np.ones(tuple(shape_xyz)[::-1])


def salt_body(v, shape_xyz, spacing, semi_axes_m=(1500.0, 1000.0, 600.0), v_salt=4.5, seed=5):
    """Overwrite an ellipsoid (centred mid-model, jittered by seed) with v_salt."""
    r = rng(seed)
    nd = len(shape_xyz)
    ext = [(s - 1) * h for s, h in zip(shape_xyz, spacing)]
    c = [0.5 * e + r.uniform(-0.05, 0.05) * e for e in ext]
    axes = [np.arange(s, dtype=np.float64) * h for s, h in zip(shape_xyz, spacing)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    q = sum(((grids[d] - c[d]) / semi_axes_m[d]) ** 2 for d in range(nd))
    out = np.array(v, copy=True)
    out[q <= 1.0] = v_salt
    return out


def line_receivers_jittered(n, x0, dx, depth, h, extent_xz, seed=1234):
    """2D receivers: x_i = x0 + i*dx at ``depth``; each coordinate jittered by
    U[-h/2, h/2) and clamped inside [0, extent]."""
    r = rng(seed)
    x = x0 + dx * np.arange(n, dtype=np.float64)
    z = np.full(n, float(depth))
    x = x + r.uniform(-0.5 * h, 0.5 * h, size=n)
    z = z + r.uniform(-0.5 * h, 0.5 * h, size=n)
    x = np.clip(x, 0.0, extent_xz[0])
    z = np.clip(z, 0.0, extent_xz[1])
    return np.stack([x, z], axis=1).astype(np.float32)


def surface_grid_receivers(nx, ny, spacing_xy, depth, origin_xy=(0.0, 0.0)):
    """3D receivers on an nx-by-ny grid at constant depth (x fastest)."""
    x = origin_xy[0] + spacing_xy[0] * np.arange(nx, dtype=np.float64)
    y = origin_xy[1] + spacing_xy[1] * np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y, indexing="xy")
    Z = np.full(X.shape, float(depth))
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)


def random_points(n, shape_xyz, spacing, seed, margin=0.0):
    """Uniform random off-grid points inside the physical domain."""
    r = rng(seed)
    ext = [(s - 1) * h for s, h in zip(shape_xyz, spacing)]
    cols = [r.uniform(margin, e - margin, size=n) for e in ext]
    return np.stack(cols, axis=1).astype(np.float32)


def random_traces(nt, n, seed, scale=1.0):
    return (scale * rng(seed).standard_normal((nt, n))).astype(np.float32)


def smooth_perturbation(shape_xyz, spacing, seed, corr_len=30.0):
    """A smooth, bounded model perturbation (unit max-abs) for Taylor tests."""
    g = smooth_gaussian_noise(shape_xyz, corr_len / spacing[0], seed).astype(np.float64)
    return g / np.abs(g).max()


def layered_profile(nz, dz, n_layers, v_min=1.5, v_max=4.5, perturb=0.05, seed=0):
    """1D velocity v(z) (km/s, length nz): ``n_layers`` flat layers with sorted
    velocities drawn in [v_min, v_max] (the top one v_min), interfaces at sorted
    random depths, each layer scaled by 1 + U(-perturb, perturb), clipped."""
    r = rng(seed)
    depth = (nz - 1) * dz
    vs = np.sort(r.uniform(v_min, v_max, size=n_layers))
    vs[0] = v_min
    vs = np.clip(vs * (1.0 + r.uniform(-perturb, perturb, size=n_layers)), v_min, v_max)
    cuts = np.sort(r.uniform(0.05 * depth, 0.95 * depth, size=n_layers - 1))
    z = np.arange(nz, dtype=np.float64) * dz
    v = np.full(nz, vs[0])
    for i, c in enumerate(cuts):
        v = np.where(z >= c, vs[i + 1], v)
    return v


def serving_requests(n, seed=99):
    """Seeded stream of shot-modelling requests: half 2D (N x N, N in
    [201, 1001]), half 3D (N^3, N in [128, 320]); space order in {4, 8, 16};
    nt in [500, 2000]; 3-8 velocity layers in [1.5, 4.5] km/s; one 10 Hz
    Ricker source at the surface centre; 100-1000 surface receivers;
    h = 10 m, 20-point (2D) or 40-point (3D) absorbing layer."""
    r = rng(seed)
    out = []
    for i in range(n):
        ndim = 2 if r.uniform() < 0.5 else 3
        N = int(r.integers(201, 1002)) if ndim == 2 else int(r.integers(128, 321))
        out.append(dict(id=i, ndim=ndim, N=N, h=10.0, nbl=20 if ndim == 2 else 40,
                        so=int(r.choice([4, 8, 16])), nt=int(r.integers(500, 2001)),
                        n_layers=int(r.integers(3, 9)), n_rec=int(r.integers(100, 1001)),
                        model_seed=int(seed * 100003 + i), f0=0.010))
    return out


def request_points(req):
    """Source (surface centre, 20 m deep) and receivers (surface line in 2D, a
    k x k surface grid with k*k >= n_rec in 3D, at 20 m) of a serving request."""
    N, h, nd = req["N"], req["h"], req["ndim"]
    ext = (N - 1) * h
    if nd == 2:
        src = np.array([[0.5 * ext, 20.0]], dtype=np.float32)
        x = np.linspace(0.0, ext, req["n_rec"])
        rec = np.stack([x, np.full_like(x, 20.0)], axis=1).astype(np.float32)
    else:
        src = np.array([[0.5 * ext, 0.5 * ext, 20.0]], dtype=np.float32)
        k = int(np.ceil(np.sqrt(req["n_rec"])))
        g = np.linspace(0.0, ext, k)
        X, Y = np.meshgrid(g, g, indexing="xy")
        rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 20.0)], axis=1).astype(np.float32)
    return src, rec


def gradient_models(shape_xyz, spacing, seed=11):
    """FWI gradient workload: background v(z) = 1.5 + 0.6 z[km] and the true
    model with three seeded Gaussian anomalies (+-0.2 km/s, sigma 150 m)."""
    v0 = linear_gradient_velocity(shape_xyz, spacing)
    return v0, v0 + gaussian_anomalies(shape_xyz, spacing, n=3, amp=0.2, sigma_m=150.0, seed=seed)


def layered_salt_velocity(shape_xyz, spacing, n_layers=8, v_min=1.5, v_max=4.5, v_salt=4.5,
                          semi_axes_m=(1500.0, 1000.0, 600.0), seed=5):
    """Large-model workload: ``n_layers`` flat layers (1D profile, see
    ``layered_profile``) with an ellipsoidal salt-like body of velocity v_salt
    centred mid-model (jittered by the seed), built plane by plane in float32."""
    nx, ny, nz = shape_xyz
    prof = layered_profile(nz, spacing[2], n_layers, v_min, v_max, seed=seed).astype(np.float32)
    r = rng(seed + 1)
    ext = [(s - 1) * h for s, h in zip(shape_xyz, spacing)]
    c = [0.5 * e + r.uniform(-0.05, 0.05) * e for e in ext]
    x = ((np.arange(nx) * spacing[0] - c[0]) / semi_axes_m[0]) ** 2
    y = ((np.arange(ny) * spacing[1] - c[1]) / semi_axes_m[1]) ** 2
    xy = (y[:, None] + x[None, :]).astype(np.float32)
    v = np.empty((nz, ny, nx), dtype=np.float32)
    for k in range(nz):
        zz = ((k * spacing[2] - c[2]) / semi_axes_m[2]) ** 2
        v[k] = np.where(xy + zz <= 1.0, np.float32(v_salt), prof[k])
    return v


def layered_starting_velocity(shape_xyz, spacing, n_layers=8, v_min=1.5, v_max=4.5, sigma_m=150.0, seed=5):
    """Starting model of the large-model gradient: the flat layers of
    ``layered_salt_velocity`` (same seed) smoothed along depth by a Gaussian of
    standard deviation sigma_m (edge values repeated), without the salt body;
    float32, [nz][ny][nx]."""
    nx, ny, nz = shape_xyz
    prof = layered_profile(nz, spacing[2], n_layers, v_min, v_max, seed=seed)
    k = int(np.ceil(4.0 * sigma_m / spacing[2]))
    t = np.arange(-k, k + 1) * spacing[2] / sigma_m
    w = np.exp(-0.5 * t * t)
    w /= w.sum()
    smooth = np.convolve(np.pad(prof, k, mode="edge"), w, mode="valid").astype(np.float32)
    return np.broadcast_to(smooth[:, None, None], (nz, ny, nx)).copy()
