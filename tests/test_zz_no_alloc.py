"""GPU test of the allocation-free objective entry point.

wave_objective_noalloc serves callers that cannot allocate device memory when
they need the objective (a stream being captured into a CUDA graph, a host
application that owns every device allocation, a service that must not touch
the allocator mid-run); it keeps its scratch in a fixed device array inside the
library.  This test calls it through the C ABI twice in a row and checks both
calls against the residual and objective that wave_gradient returns for the
same data.  The file name makes pytest collect it last.
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
