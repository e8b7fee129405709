"""GPU test of the allocation-free objective entry point.

wave_objective_noalloc serves callers that cannot allocate device memory when
they need the objective (a host application that owns every device allocation
through its own pool, a service that must not touch the allocator mid-run); it
keeps its scratch in a fixed device array inside the library.  The first test
calls it through the C ABI twice in a row and checks both calls against the
residual and objective that wave_gradient returns for the same data; the others
cover several scratch chunks ending in a partial one, the call without a
residual output, and the Python wrapper, against an FP64 NumPy sum.  The file
name makes pytest collect it last.
"""

import ctypes

import numpy as np
import pytest

from gpu_cases import geometries, small2d

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import wave  # noqa: E402

pytestmark = pytest.mark.gpu


def test_objective_noalloc_matches_gradient_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    og, m, dt, nt, so, src, q, rec = small2d(4)
    _, geom = geometries(og)
    rng = np.random.default_rng(31)
    with wave.Context(0) as ctx:
        md = torch.from_numpy(m).cuda()
        qd = torch.from_numpy(q).cuda()
        d_pred = wave.wave_forward(ctx, geom, md, src, qd, rec, dt, nt, so)
        d_obs = d_pred + torch.from_numpy(rng.standard_normal(tuple(d_pred.shape)).astype(np.float32)).cuda()
        _, phi_ref, r_ref = wave.wave_gradient(ctx, geom, md, src, qd, rec, d_obs, dt, nt, so,
                                               snap_mode="full_fp32", return_residual=True)
        torch.cuda.synchronize()
    n = d_pred.numel()
    lib = wave.lib()
    for call in range(2):
        r = torch.full_like(d_pred, float("nan"))
        phi = ctypes.c_double(-1.0)
        rc = lib.wave_objective_noalloc(ctypes.c_void_p(d_pred.data_ptr()), ctypes.c_void_p(d_obs.data_ptr()),
                                        ctypes.c_void_p(r.data_ptr()), n, ctypes.byref(phi), None)
        assert rc == wave.WAVE_OK, (call, rc)
        assert abs(phi.value - phi_ref) <= 1e-6 * phi_ref, (call, phi.value, phi_ref)
        np.testing.assert_allclose(r.cpu().numpy(), r_ref.cpu().numpy(), rtol=1e-6, atol=1e-6)
    # sizes beyond the scratch maximum are rejected, without touching the GPU
    big = lib.wave_objective_noalloc(ctypes.c_void_p(d_pred.data_ptr()), ctypes.c_void_p(d_obs.data_ptr()), None,
                                     (1 << 28) + 1, ctypes.byref(ctypes.c_double()), None)
    assert big == wave.WAVE_ERR_INVALID_ARG


def _reference(d, d_obs):
    """Residual in float32 (as the kernels form it) and phi = 0.5 sum r^2 in FP64."""
    r = (d - d_obs).astype(np.float32)
    return r, 0.5 * float(np.sum(r.astype(np.float64) ** 2))


@pytest.mark.parametrize("n", [3 * 8192 + 123, 8192, 1])
def test_objective_noalloc_several_chunks_and_no_residual(n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n).astype(np.float32)
    d_obs = rng.standard_normal(n).astype(np.float32)
    r_ref, phi_ref = _reference(d, d_obs)
    dd, od = torch.from_numpy(d).cuda(), torch.from_numpy(d_obs).cuda()
    lib = wave.lib()
    for call in range(2):
        r = torch.full_like(dd, float("nan"))
        phi = ctypes.c_double(-1.0)
        rc = lib.wave_objective_noalloc(ctypes.c_void_p(dd.data_ptr()), ctypes.c_void_p(od.data_ptr()),
                                        ctypes.c_void_p(r.data_ptr()), n, ctypes.byref(phi), None)
        assert rc == wave.WAVE_OK, (call, rc)
        assert abs(phi.value - phi_ref) <= 1e-12 * phi_ref, (call, phi.value, phi_ref)
        np.testing.assert_array_equal(r.cpu().numpy(), r_ref)
        phi2 = ctypes.c_double(-1.0)
        rc = lib.wave_objective_noalloc(ctypes.c_void_p(dd.data_ptr()), ctypes.c_void_p(od.data_ptr()), None, n,
                                        ctypes.byref(phi2), None)
        assert rc == wave.WAVE_OK and abs(phi2.value - phi_ref) <= 1e-12 * phi_ref, (call, phi2.value)


def test_objective_noalloc_python_wrapper():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 2 * 8192 + 4097
    rng = np.random.default_rng(5)
    d = rng.standard_normal(n).astype(np.float32)
    d_obs = rng.standard_normal(n).astype(np.float32)
    r_ref, phi_ref = _reference(d, d_obs)
    dd, od = torch.from_numpy(d).cuda(), torch.from_numpy(d_obs).cuda()
    for _ in range(2):
        r = torch.empty_like(dd)
        phi, r_back = wave.wave_objective_noalloc(dd, od, r_out=r)
        assert r_back is r
        assert abs(phi - phi_ref) <= 1e-12 * phi_ref
        np.testing.assert_array_equal(r.cpu().numpy(), r_ref)
        phi_only, none = wave.wave_objective_noalloc(dd, od)
        assert none is None and abs(phi_only - phi_ref) <= 1e-12 * phi_ref
