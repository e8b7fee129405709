"""Shared seeded cases for the GPU parity tests (inputs only; expected values
always come from the oracle)."""

import numpy as np

import oracle
from paper_1608_08658_gb300 import inputs, wave


def geometries(og):
    """(oracle geometry, library geometry) pair with the same fields."""
    return og, wave.Geometry(shape=og.shape, spacing=og.spacing, origin=og.origin, nbl=og.nbl,
                             sponge_vref=og.sponge_vref)


def f32(x):
    return float(np.float32(x))


def config1():
    """2D parity workload: 101x101, h = 10 m, v = 1.5 km/s, order 4, 20-point
    sponge, dt = 0.4 of the stability limit, nt = 500, Ricker 10 Hz at the
    grid centre, 101 receivers at 20 m depth jittered by seed 1234."""
    og = oracle.model.Geometry(shape=(101, 101), spacing=(10.0, 10.0), nbl=20, sponge_vref=1.5)
    so, nt = 4, 500
    m = inputs.slowness2(inputs.constant_velocity(og.shape, 1.5))
    dt = f32(0.4 * oracle.model.dt_max(so, og.spacing, 1.5))
    src = np.array([[500.0, 500.0]], dtype=np.float32)
    rec = inputs.line_receivers_jittered(101, 0.0, 10.0, 20.0, 10.0, (1000.0, 1000.0), seed=1234)
    q = oracle.model.ricker(nt, dt, 0.010)[:, None].astype(np.float32)
    return og, m, dt, nt, so, src, q, rec


def small3d(so, shape=(83, 21, 40), nbl=5, nt=60, seed=0, nsrc=2, nrec=25, spacing=(10.0, 12.0, 9.0)):
    """Small 3D case with ragged tiles and several z chunks; sources and
    receivers off-grid, on nodes, on tile edges and on the last node.  The
    default spacing differs per axis; equal spacing selects the kernel that
    shares one coefficient per offset between the axes."""
    og = oracle.model.Geometry(shape=shape, spacing=spacing, origin=(3.0, -7.0, 0.0), nbl=nbl,
                               sponge_vref=2.5)
    r = inputs.rng(seed)
    v = 1.5 + 1.0 * r.uniform(size=og.phys_array_shape)
    m = inputs.slowness2(v)
    dt = f32(0.45 * oracle.model.dt_max(so, og.spacing, 2.5))
    lo = np.array(og.origin)
    hi = lo + (np.array(og.shape) - 1) * np.array(og.spacing)
    src = (lo + r.uniform(0.2, 0.8, size=(nsrc, 3)) * (hi - lo)).astype(np.float32)
    rec = lo + r.uniform(size=(nrec, 3)) * (hi - lo)
    rec[0] = lo                                   # first physical node
    rec[1] = hi                                   # last physical node
    hx, hy, hz = spacing
    rec[2] = lo + np.array([(64 - nbl) * hx, (16 - nbl) * hy, 4 * hz])   # tile corner node
    rec[3] = lo + np.array([(63.5 - nbl) * hx, 3.25 * hy, 17.7 * hz])   # straddles an x tile edge
    rec = rec.astype(np.float32)
    q = (r.standard_normal((nt, nsrc)) * 1e2).astype(np.float32)
    return og, m, dt, nt, so, src, q, rec


def small2d(so, shape=(150, 77), nbl=9, nt=80, seed=1, nsrc=2, nrec=19, spacing=(7.5, 10.0)):
    og = oracle.model.Geometry(shape=shape, spacing=spacing, origin=(0.0, 0.0), nbl=nbl, sponge_vref=2.0)
    r = inputs.rng(seed)
    v = 1.5 + 0.5 * r.uniform(size=og.phys_array_shape)
    m = inputs.slowness2(v)
    dt = f32(0.45 * oracle.model.dt_max(so, og.spacing, 2.0))
    lo = np.array(og.origin)
    hi = lo + (np.array(og.shape) - 1) * np.array(og.spacing)
    src = (lo + r.uniform(0.2, 0.8, size=(nsrc, 2)) * (hi - lo)).astype(np.float32)
    rec = lo + r.uniform(size=(nrec, 2)) * (hi - lo)
    rec[0] = lo
    rec[1] = hi
    rec = rec.astype(np.float32)
    q = (r.standard_normal((nt, nsrc)) * 1e2).astype(np.float32)
    return og, m, dt, nt, so, src, q, rec


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
