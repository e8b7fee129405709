"""CPU checks of the C ABI: the library builds and loads, exports every entry
point declared in include/wave.h, and its host-side helpers (weights, CFL
limit, Ricker wavelet, error strings) agree with the oracle.  No GPU compute."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1608_08658_gb300 import build as libbuild
from paper_1608_08658_gb300 import wave

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return wave.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "wave.h")).read()
    return sorted(set(re.findall(r"WAVE_API\s+[\w\s\*]+?\b(wave_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers the same set
    assert sorted(names) == wave.exported_names()


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_fd_weights_match_oracle(lib, so):
    np.testing.assert_allclose(wave.wave_fd_weights(so), oracle.fd.fd_weights(so), rtol=2e-15, atol=1e-16)


def test_fd_weights_reject_bad_order(lib):
    for bad in (0, 3, 18):
        with pytest.raises(wave.WaveError):
            wave.wave_fd_weights(bad)


@pytest.mark.parametrize("so,spacing,v", [(4, (10.0, 10.0), 1.5), (8, (10.0, 10.0, 10.0), 2.5),
                                          (16, (12.5, 7.0, 9.0), 4.5)])
def test_dt_max_matches_oracle(lib, so, spacing, v):
    assert abs(wave.wave_dt_max(spacing, so, v) - oracle.model.dt_max(so, spacing, v)) < 1e-12


def test_ricker_matches_oracle(lib):
    nt, dt, f0 = 700, 1.633, 0.01
    r = wave.wave_ricker(nt, dt, f0)
    ref = oracle.model.ricker(nt, np.float32(dt), np.float32(f0), t0=np.float32(1.0 / f0))
    np.testing.assert_allclose(r, ref, rtol=0, atol=2e-7)


def test_error_strings(lib):
    for code in range(8):
        assert wave.wave_error_string(code)
    assert "unknown" in wave.wave_error_string(99)


def test_context_without_gpu_reports_error(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    rc = lib.wave_context_create(ctypes.byref(h), 0, 0)
    assert rc in (wave.WAVE_ERR_CUDA, wave.WAVE_ERR_NOT_SUPPORTED)
    assert not h.value
    assert lib.wave_context_destroy(None) == 0


def test_step_kernel_layout(lib):
    """Host-only layout query: the tile of every step kernel covers whole 16-byte
    quads, two CTAs fit one SM's shared memory and register file, and the
    register-queue settings are consistent (paired planes and renamed groups
    exclude each other)."""
    smem_two_ctas = 228 * 1024 // 2 - 1024
    for so in range(2, 17, 2):
        R = so // 2
        for ndim in (2, 3):
            for kernel in range(9):
                for eq in (0, 1):
                    L = wave.wave_step_kernel_layout(so, ndim, kernel, eq)
                    assert (L["radius"], L["ndim"], L["kernel"]) == (R, ndim, kernel)
                    assert L["equal_spacing_variant"] == int(bool(eq) and R >= 6)
                    assert L["bx"] % 4 == 0 and L["hx"] % 4 == 0 and L["hx"] >= min(R, 8) - 4
                    assert L["threads"] == (L["by"] // 2 + 1) * 32
                    assert L["smem_bytes"] <= smem_two_ctas
                    assert L["ctas_per_sm"] * L["threads"] <= 2048
                    if ndim == 2:
                        assert L["prefetch"] == 0 and L["planes_per_renamed_group"] == 1
                        continue
                    assert L["planes_per_move"] == 1 or L["planes_per_renamed_group"] == 1
                    assert L["planes_per_renamed_group"] >= 1
                    q = L["queue_stages"]
                    assert q == (L["prefetch"] + 1 if L["lead_plane"] else R + 1 + L["prefetch"])
    with pytest.raises(wave.WaveError):
        wave.wave_step_kernel_layout(7, 3, 0, 1)
    with pytest.raises(wave.WaveError):
        wave.wave_step_kernel_layout(8, 3, 9, 1)
    with pytest.raises(wave.WaveError):
        wave.wave_step_kernel_layout(8, 4, 0, 1)


def test_objective_noalloc_wrapper_rejects_bad_arrays_before_any_call(monkeypatch):
    """The Python wrapper of wave_objective_noalloc checks every array (type,
    dtype, contiguity, size, device) before it reaches the library: none of
    these calls launches anything."""
    torch = pytest.importorskip("torch")

    def no_call():
        raise AssertionError("the library must not be called")
    monkeypatch.setattr(wave, "lib", no_call)
    d = torch.zeros(10)
    bad = [((np.zeros(10, np.float32), d), {}, TypeError),                       # not a tensor
           ((d, torch.zeros(9)), {}, ValueError),                                 # d_obs too short
           ((d, torch.zeros(10, dtype=torch.float64)), {}, TypeError),            # d_obs not float32
           ((d, d), {"r_out": torch.zeros(9)}, ValueError),                       # r_out too short
           ((d, d), {"r_out": torch.zeros(10, dtype=torch.float64)}, TypeError),  # r_out not float32
           ((d, d), {"r_out": torch.zeros(20)[::2]}, ValueError),                # r_out not contiguous
           ((torch.zeros(20)[::2], torch.zeros(10)), {}, ValueError),             # d not contiguous
           ((d, d), {}, ValueError)]                                              # host tensors
    for args, kw, exc in bad:
        with pytest.raises(exc):
            wave.wave_objective_noalloc(*args, **kw)
