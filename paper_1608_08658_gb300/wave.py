"""ctypes binding of libwave (include/wave.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name.  Array
arguments may be NumPy arrays (host memory: the library stages them) or
torch tensors (device memory on the context's GPU, used in place; the call is
enqueued on torch's current stream).  Outputs are allocated like the inputs
when not given.  There is no fallback: if ``libwave.so`` is missing or the GPU
path fails, the call raises.
"""

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwave.so")

WAVE_OK = 0
WAVE_ERR_INVALID_ARG = 1
WAVE_ERR_POINT_OUTSIDE = 2
WAVE_ERR_UNSTABLE_DT = 3
WAVE_ERR_OUT_OF_MEMORY = 4
WAVE_ERR_CUDA = 5
WAVE_ERR_TIMEOUT = 6
WAVE_ERR_NOT_SUPPORTED = 7

SNAP_FULL_FP32 = 0
SNAP_FULL_BF16 = 1
SNAP_FULL_FP16 = 2
SNAP_CHECKPOINT_FP32 = 3
SNAP_CHECKPOINT_BF16 = 4
SNAP_CHECKPOINT_FP16 = 5
SNAP_AUTO = 6
SNAP_MODES = {
    "full_fp32": SNAP_FULL_FP32, "full_bf16": SNAP_FULL_BF16, "full_fp16": SNAP_FULL_FP16,
    "checkpoint_fp32": SNAP_CHECKPOINT_FP32, "checkpoint_bf16": SNAP_CHECKPOINT_BF16,
    "checkpoint_fp16": SNAP_CHECKPOINT_FP16, "auto": SNAP_AUTO,
}

KERNEL_STEP, KERNEL_STEP_SNAP, KERNEL_STEP_GRAD, KERNEL_SPARSE, KERNEL_OTHER = range(5)
KERNEL_NAMES = ["step", "step_snap", "step_grad", "sparse", "other"]


class WaveError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d): %s" % (_lib_error_string(code), code, msg))
        self.code = code


class c_geometry(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("nbl", ctypes.c_int32), ("shape", ctypes.c_int64 * 3),
                ("spacing", ctypes.c_double * 3), ("origin", ctypes.c_double * 3),
                ("sponge_vref", ctypes.c_double)]


class c_points(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("coords", ctypes.c_void_p)]


_P = ctypes.c_void_p
_SIGS = {
    "wave_context_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]),
    "wave_context_destroy": (ctypes.c_int, [_P]),
    "wave_context_workspace_bytes": (ctypes.c_size_t, [_P]),
    "wave_context_trim": (ctypes.c_int, [_P]),
    "wave_context_set_checkpoint_interval": (ctypes.c_int, [_P, ctypes.c_int]),
    "wave_context_set_wait_limit_ns": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "wave_context_withhold_next_loads": (ctypes.c_int, [_P]),
    "wave_context_set_time_blocking": (ctypes.c_int, [_P, ctypes.c_int]),
    "wave_context_set_column_segments": (ctypes.c_int, [_P, ctypes.c_int]),
    "wave_column_runs_for": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "wave_z_chunks_for": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                         ctypes.POINTER(ctypes.c_int)]),
    "wave_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "wave_last_error": (ctypes.c_char_p, [_P]),
    "wave_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, ctypes.c_int, _P]),
    "wave_forward_ex": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                       _P, _P, _P, _P, _P]),
    "wave_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, ctypes.c_int, _P]),
    "wave_gradient": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_int, ctypes.c_int, _P]),
    "wave_jacobian_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_float,
                                             ctypes.c_int, ctypes.c_int, _P]),
    "wave_gradient_shots": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int, _P]),
    "wave_born": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, ctypes.c_int, _P]),
    "wave_fd_weights": (ctypes.c_int, [ctypes.c_int, _P]),
    "wave_interpolation_operator": (ctypes.c_int, [_P, _P, _P, _P]),
    "wave_dt_max": (ctypes.c_double, [ctypes.c_int, _P, ctypes.c_int, ctypes.c_double]),
    "wave_ricker": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "wave_context_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "wave_context_kernel_stats": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_double)]),
    "wave_context_reset_stats": (ctypes.c_int, [_P]),
    "wave_step_kernel_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]),
    "wave_objective_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), _P]),
    "wave_session_footprint": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "wave_session_create": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p), _P, _P, _P, _P, _P, ctypes.c_float,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "wave_session_advance": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "wave_session_query": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "wave_sessions_advance": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, _P]),
    "wave_session_read": (ctypes.c_int, [_P, _P]),
    "wave_session_destroy": (ctypes.c_int, [_P]),
    "wave_context_budget_free": (ctypes.c_size_t, [_P]),
    "wave_context_storage_plan": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_int)]),
    "wave_storage_plan_for": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
}

_lib = None


def lib():
    """Load libwave.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libwave.so is not built (run `python -m paper_1608_08658_gb300.build`)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return sorted(_SIGS)


def _lib_error_string(code):
    try:
        return lib().wave_error_string(code).decode()
    except Exception:  # noqa: BLE001 - only used to format an error message
        return "status"


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Raw pointer of a contiguous float32/float64 array (NumPy or torch)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be a C-contiguous numpy array or a torch tensor")
    return x.ctypes.data


def _f32(x):
    if x is None:
        return None
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32:
            raise TypeError("tensor must be float32")
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=np.float32)


def _numel(x):
    return int(x.numel()) if _is_torch(x) else int(x.size)


def _sized(name, x, shape):
    """An input array as contiguous float32 holding exactly prod(shape)
    elements (the library reads that many): checked before any call, so a
    short array raises instead of being read past its end."""
    x = _f32(x)
    n = int(np.prod(shape))
    if _numel(x) != n:
        raise ValueError("%s has %d elements, expected %d %s" % (name, _numel(x), n, tuple(shape)))
    return x


def _out(name, x, shape, ref):
    """A caller-supplied output buffer (float32, contiguous, exactly
    prod(shape) elements: the library writes that many), or a new one of the
    kind of `ref` when x is None."""
    if x is None:
        return _empty_like_kind(ref, shape)
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32:
            raise TypeError("%s must be float32, got %s" % (name, x.dtype))
        if not x.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    elif not isinstance(x, np.ndarray) or x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
        raise TypeError("%s must be a C-contiguous float32 numpy array or torch tensor" % name)
    n = int(np.prod(shape))
    if _numel(x) != n:
        raise ValueError("%s has %d elements, expected %d %s" % (name, _numel(x), n, tuple(shape)))
    return x


def _empty_like_kind(ref, shape):
    if ref is not None and _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=torch.float32, device=ref.device)
    return np.empty(shape, dtype=np.float32)


def _stream_for(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None


@dataclass
class Geometry:
    """Physical grid (x-first per-axis values) plus absorbing layer."""
    shape: tuple
    spacing: tuple
    origin: tuple = None
    nbl: int = 0
    sponge_vref: float = 1.5
    _c: object = field(default=None, repr=False, compare=False)

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.spacing = tuple(float(h) for h in self.spacing)
        if self.origin is None:
            self.origin = (0.0,) * len(self.shape)
        self.origin = tuple(float(o) for o in self.origin)

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def phys_array_shape(self):
        return self.shape[::-1]

    @property
    def comp_array_shape(self):
        return tuple(n + 2 * self.nbl for n in self.shape)[::-1]

    def to_c(self):
        g = c_geometry()
        g.ndim = self.ndim
        g.nbl = int(self.nbl)
        for d in range(3):
            g.shape[d] = self.shape[d] if d < self.ndim else 1
            g.spacing[d] = self.spacing[d] if d < self.ndim else 1.0
            g.origin[d] = self.origin[d] if d < self.ndim else 0.0
        g.sponge_vref = float(self.sponge_vref)
        self._c = g
        return g


def _points(coords, ndim):
    if coords is None:
        return c_points(0, None), None
    c = _f32(coords)
    n = int(c.shape[0]) if c.ndim == 2 else int(c.size // ndim)
    if n and (c.ndim != 2 or c.shape[1] != ndim):
        raise ValueError("point coordinates must be (n, %d)" % ndim)
    return c_points(n, _ptr(c) if n else None), c


def _check(ctx, rc):
    if rc != WAVE_OK:
        raise WaveError(rc, lib().wave_last_error(ctx.handle).decode())


class Context:
    """Owns a wave_context (device workspace reused across calls)."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        h = ctypes.c_void_p()
        rc = lib().wave_context_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if rc != WAVE_OK:
            raise WaveError(rc, "wave_context_create failed on device %d" % device)
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            lib().wave_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def workspace_bytes(self):
        return int(lib().wave_context_workspace_bytes(self.handle))

    def trim(self):
        _check(self, lib().wave_context_trim(self.handle))

    def set_checkpoint_interval(self, steps):
        _check(self, lib().wave_context_set_checkpoint_interval(self.handle, int(steps)))

    def set_wait_limit_ns(self, ns):
        """Limit of each bounded wait of the step kernels (0 = the default 10 s)."""
        _check(self, lib().wave_context_set_wait_limit_ns(self.handle, int(ns)))

    def set_time_blocking(self, levels):
        """Time levels per pass of source-free forward modelling (1 or 2)."""
        _check(self, lib().wave_context_set_time_blocking(self.handle, int(levels)))

    def set_column_segments(self, mode):
        """Decomposition of plain 3D forward steps: 0 z chunks, 1 automatic, 2 column segments."""
        _check(self, lib().wave_context_set_column_segments(self.handle, int(mode)))

    def withhold_next_loads(self):
        """Test hook: the next step launch issues no tile loads (its waits run out)."""
        _check(self, lib().wave_context_withhold_next_loads(self.handle))

    def set_profiling(self, enable):
        _check(self, lib().wave_context_set_profiling(self.handle, int(bool(enable))))

    def kernel_stats(self, kind=-1):
        n = ctypes.c_int64()
        t = ctypes.c_double()
        _check(self, lib().wave_context_kernel_stats(self.handle, int(kind), ctypes.byref(n), ctypes.byref(t)))
        return int(n.value), float(t.value)

    def reset_stats(self):
        _check(self, lib().wave_context_reset_stats(self.handle))

    def budget_free(self):
        return int(lib().wave_context_budget_free(self.handle))

    def storage_plan(self):
        """(buffer levels, parts per segment, segments) of the last gradient call."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self, lib().wave_context_storage_plan(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


class Session:
    """A resident forward-modelling request (wave_session_*): created on a
    stream, advanced asynchronously, polled, read, destroyed."""

    def __init__(self, ctx, geom, m, src, q, rec, dt, nt, space_order, stream=None, graph_chunk=32):
        self.ctx = ctx
        self.nt = int(nt)
        g = geom.to_c()
        ps, self._src = _points(src, geom.ndim)
        pr, self._rec = _points(rec, geom.ndim)
        self.n_rec = int(pr.n)
        m = _sized("m", m, geom.phys_array_shape)
        q = _sized("q", q, (self.nt, ps.n)) if ps.n else None
        h = ctypes.c_void_p()
        st = stream if stream is not None else _stream_for(m, q)
        rc = lib().wave_session_create(ctx.handle, ctypes.byref(h), ctypes.byref(g), _ptr(m), ctypes.byref(ps),
                                       _ptr(q), ctypes.byref(pr), ctypes.c_float(dt), self.nt, int(space_order),
                                       int(graph_chunk), st)
        _check(ctx, rc)
        self.handle = h
        self.steps_left = self.nt - 1

    def advance(self, steps):
        left = ctypes.c_int()
        _check(self.ctx, lib().wave_session_advance(self.handle, int(steps), ctypes.byref(left)))
        self.steps_left = left.value
        return self.steps_left

    def done(self):
        d = ctypes.c_int()
        _check(self.ctx, lib().wave_session_query(self.handle, ctypes.byref(d)))
        return bool(d.value)

    def read(self, out=None):
        if out is None:
            out = np.empty((self.nt, self.n_rec), dtype=np.float32)
        out = _out("out", out, (self.nt, self.n_rec), None)
        _check(self.ctx, lib().wave_session_read(self.handle, _ptr(out) if self.n_rec else None))
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().wave_session_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def wave_sessions_advance(sessions, steps, stream=None):
    """Enqueue up to ``steps`` more steps of every session in ``sessions`` with
    batched launches (one stencil launch per step per space order, dimension and
    spacing variant; one injection and one receiver launch per step) on
    ``stream`` (a ctypes c_void_p or None)."""
    sessions = list(sessions)
    if not sessions:
        return
    arr = (ctypes.c_void_p * len(sessions))(*[sess.handle for sess in sessions])
    rc = lib().wave_sessions_advance(arr, len(sessions), int(steps), stream)
    if rc != WAVE_OK:
        raise WaveError(rc, lib().wave_last_error(sessions[0].ctx.handle).decode())
    for sess in sessions:
        sess.steps_left = max(0, sess.steps_left - int(steps))


def wave_session_footprint(ctx, geom, src, rec, nt, space_order):
    g = geom.to_c()
    ps, _s = _points(src, geom.ndim)
    pr, _r = _points(rec, geom.ndim)
    b = ctypes.c_size_t()
    _check(ctx, lib().wave_session_footprint(ctx.handle, ctypes.byref(g), ctypes.byref(ps), ctypes.byref(pr),
                                             int(nt), int(space_order), ctypes.byref(b)))
    return int(b.value)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def wave_forward(ctx, geom, m, src, q, rec, dt, nt, space_order, d_out=None, stream=None,
                 u_init_prev=None, u_init=None, return_final=False):
    """Receiver data [nt][n_rec] of the forward model (Listing 1).  With
    ``return_final`` also returns (u^{nt-2}, u^{nt-1}) on the computational grid."""
    m = _sized("m", m, geom.phys_array_shape)
    g = geom.to_c()
    ps, src_c = _points(src, geom.ndim)
    pr, rec_c = _points(rec, geom.ndim)
    q = _sized("q", q, (nt, ps.n)) if ps.n else None
    d_out = _out("d_out", d_out, (nt, pr.n), m)
    ui_p = None if u_init_prev is None else _sized("u_init_prev", u_init_prev, geom.comp_array_shape)
    ui = None if u_init is None else _sized("u_init", u_init, geom.comp_array_shape)
    fin_p = fin = None
    if return_final:
        fin_p = _empty_like_kind(m, geom.comp_array_shape)
        fin = _empty_like_kind(m, geom.comp_array_shape)
    st = stream if stream is not None else _stream_for(m, q, d_out)
    rc = lib().wave_forward_ex(ctx.handle, ctypes.byref(g), _ptr(m), ctypes.byref(ps), _ptr(q), ctypes.byref(pr),
                               _ptr(d_out) if pr.n else None, ctypes.c_float(dt), int(nt), int(space_order),
                               _ptr(ui_p), _ptr(ui), _ptr(fin_p), _ptr(fin), st)
    _check(ctx, rc)
    return (d_out, fin_p, fin) if return_final else d_out


def wave_adjoint(ctx, geom, m, src, rec, y, dt, nt, space_order, q_out=None, stream=None):
    """Source-side traces F^T y [nt][n_src] (Listing 2 as the transpose)."""
    m = _sized("m", m, geom.phys_array_shape)
    g = geom.to_c()
    ps, src_c = _points(src, geom.ndim)
    pr, rec_c = _points(rec, geom.ndim)
    y = _sized("y", y, (nt, pr.n)) if pr.n else None
    q_out = _out("q_out", q_out, (nt, ps.n), m)
    st = stream if stream is not None else _stream_for(m, y, q_out)
    rc = lib().wave_adjoint(ctx.handle, ctypes.byref(g), _ptr(m), ctypes.byref(ps), ctypes.byref(pr), _ptr(y),
                            _ptr(q_out) if ps.n else None, ctypes.c_float(dt), int(nt), int(space_order), st)
    _check(ctx, rc)
    return q_out


def wave_gradient(ctx, geom, m, src, q, rec, d_obs, dt, nt, space_order, snap_mode="auto",
                  grad_out=None, return_residual=False, stream=None):
    """(grad, phi[, residual]) of the objective of Eq. 2 by Eq. 3."""
    mode = SNAP_MODES[snap_mode] if isinstance(snap_mode, str) else int(snap_mode)
    m = _sized("m", m, geom.phys_array_shape)
    g = geom.to_c()
    ps, src_c = _points(src, geom.ndim)
    pr, rec_c = _points(rec, geom.ndim)
    q = _sized("q", q, (nt, ps.n)) if ps.n else None
    d_obs = _sized("d_obs", d_obs, (nt, pr.n)) if pr.n else None
    grad_out = _out("grad_out", grad_out, geom.phys_array_shape, m)
    resid = _empty_like_kind(m, (nt, pr.n)) if return_residual else None
    phi = ctypes.c_double()
    st = stream if stream is not None else _stream_for(m, q, d_obs, grad_out)
    rc = lib().wave_gradient(ctx.handle, ctypes.byref(g), _ptr(m), ctypes.byref(ps), _ptr(q), ctypes.byref(pr),
                             _ptr(d_obs), _ptr(grad_out), ctypes.byref(phi), _ptr(resid) if pr.n else None,
                             int(mode), ctypes.c_float(dt), int(nt), int(space_order), st)
    _check(ctx, rc)
    if return_residual:
        return grad_out, phi.value, resid
    return grad_out, phi.value


def wave_jacobian_adjoint(ctx, geom, m, src, q, rec, y, dt, nt, space_order, snap_mode="auto",
                          grad_out=None, d_out=None, stream=None):
    """J^T y for the map m -> receiver data (the residual replaced by y)."""
    mode = SNAP_MODES[snap_mode] if isinstance(snap_mode, str) else int(snap_mode)
    m = _sized("m", m, geom.phys_array_shape)
    g = geom.to_c()
    ps, src_c = _points(src, geom.ndim)
    pr, rec_c = _points(rec, geom.ndim)
    q = _sized("q", q, (nt, ps.n)) if ps.n else None
    y = _sized("y", y, (nt, pr.n)) if pr.n else None
    grad_out = _out("grad_out", grad_out, geom.phys_array_shape, m)
    if d_out is not None:
        d_out = _out("d_out", d_out, (nt, pr.n), m)
    st = stream if stream is not None else _stream_for(m, q, y, grad_out)
    rc = lib().wave_jacobian_adjoint(ctx.handle, ctypes.byref(g), _ptr(m), ctypes.byref(ps), _ptr(q),
                                     ctypes.byref(pr), _ptr(y), _ptr(grad_out), _ptr(d_out) if pr.n else None,
                                     int(mode), ctypes.c_float(dt), int(nt), int(space_order), st)
    _check(ctx, rc)
    return grad_out


def wave_gradient_shots(ctx, geom, m, shots, dt, nt, space_order, snap_mode="auto", grad_out=None, stream=None):
    """(sum of gradients, sum of objectives) over ``shots`` = [(src, q, rec, d_obs), ...]."""
    mode = SNAP_MODES[snap_mode] if isinstance(snap_mode, str) else int(snap_mode)
    m = _sized("m", m, geom.phys_array_shape)
    g = geom.to_c()
    n = len(shots)
    srcs = (c_points * n)()
    recs = (c_points * n)()
    qs = (ctypes.c_void_p * n)()
    obs = (ctypes.c_void_p * n)()
    keep = []
    for i, (src, q, rec, d_obs) in enumerate(shots):
        ps, sc = _points(src, geom.ndim)
        pr, rc_ = _points(rec, geom.ndim)
        qf = _sized("q of shot %d" % i, q, (nt, ps.n)) if ps.n else None
        df = _sized("d_obs of shot %d" % i, d_obs, (nt, pr.n)) if pr.n else None
        keep += [sc, rc_, qf, df]
        srcs[i], recs[i] = ps, pr
        qs[i], obs[i] = _ptr(qf), _ptr(df)
    grad_out = _out("grad_out", grad_out, geom.phys_array_shape, m)
    phi = ctypes.c_double()
    st = stream if stream is not None else _stream_for(m, grad_out)
    rc = lib().wave_gradient_shots(ctx.handle, ctypes.byref(g), _ptr(m), n, srcs, qs, recs, obs, _ptr(grad_out),
                                   ctypes.byref(phi), int(mode), ctypes.c_float(dt), int(nt), int(space_order), st)
    _check(ctx, rc)
    del keep
    return grad_out, phi.value


def wave_born(ctx, geom, m, dm, src, q, rec, dt, nt, space_order, d_out=None, stream=None):
    """Linearised data J dm [nt][n_rec] (derivative of wave_forward's data in m)."""
    m = _sized("m", m, geom.phys_array_shape)
    dm = _sized("dm", dm, geom.phys_array_shape)
    g = geom.to_c()
    ps, src_c = _points(src, geom.ndim)
    pr, rec_c = _points(rec, geom.ndim)
    q = _sized("q", q, (nt, ps.n)) if ps.n else None
    d_out = _out("d_out", d_out, (nt, pr.n), m)
    st = stream if stream is not None else _stream_for(m, dm, q, d_out)
    rc = lib().wave_born(ctx.handle, ctypes.byref(g), _ptr(m), _ptr(dm), ctypes.byref(ps), _ptr(q),
                         ctypes.byref(pr), _ptr(d_out) if pr.n else None, ctypes.c_float(dt), int(nt),
                         int(space_order), st)
    _check(ctx, rc)
    return d_out


def wave_fd_weights(space_order):
    w = np.zeros(space_order // 2 + 1 if space_order > 0 else 1, dtype=np.float64)
    rc = lib().wave_fd_weights(int(space_order), w.ctypes.data)
    if rc != WAVE_OK:
        raise WaveError(rc, "bad space order %r" % (space_order,))
    return w


def wave_interpolation_operator(geom, coords):
    """Sparse-point interpolation operator of a point set as the library builds
    it: (index, weight), each (n, 2^ndim), with dense computational-grid
    indices (x fastest); host-only."""
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.float32).reshape(-1, geom.ndim))
    n, C = c.shape[0], 1 << geom.ndim
    idx = np.zeros((n, C), dtype=np.int64)
    wts = np.zeros((n, C), dtype=np.float32)
    g = geom.to_c()
    pts = c_points(n, c.ctypes.data if n else None)
    rc = lib().wave_interpolation_operator(ctypes.byref(g), ctypes.byref(pts), idx.ctypes.data if n else None,
                                           wts.ctypes.data if n else None)
    if rc != WAVE_OK:
        raise WaveError(rc, wave_error_string(rc))
    return idx, wts


def wave_dt_max(spacing, space_order, v_max):
    h = np.ascontiguousarray(spacing, dtype=np.float64)
    v = lib().wave_dt_max(len(h), h.ctypes.data, int(space_order), float(v_max))
    if v < 0:
        raise WaveError(WAVE_ERR_INVALID_ARG, "bad arguments to wave_dt_max")
    return v


def wave_storage_plan_for(nt, level_bytes, field_bytes, avail_bytes, checkpoint=True, checkpoint_interval=0):
    """(buffer levels, parts per segment, checkpointed segments) that the
    gradient's storage planner chooses for these sizes; host-only."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = lib().wave_storage_plan_for(int(nt), int(level_bytes), int(field_bytes), int(avail_bytes),
                                     int(bool(checkpoint)), int(checkpoint_interval), ctypes.byref(a),
                                     ctypes.byref(b), ctypes.byref(c))
    if rc != WAVE_OK:
        raise WaveError(rc, wave_error_string(rc))
    return a.value, b.value, c.value


STEP_KERNELS = {"plain": 0, "snap_fp32": 1, "snap_bf16": 2, "snap_fp16": 3, "grad_fp32": 4, "grad_bf16": 5,
                "grad_fp16": 6, "born_background": 7, "scattered": 8}
STEP_LAYOUT_FIELDS = ("radius", "ndim", "kernel", "equal_spacing_variant", "bx", "by", "hx", "threads",
                      "ctas_per_sm", "lead_plane", "prefetch", "queue_stages", "point_stages", "planes_per_move",
                      "planes_per_renamed_group", "smem_bytes")


def wave_step_kernel_layout(space_order, ndim, kernel, equal_spacing):
    """Compile-time configuration (dict) of the step kernel launched for these
    arguments; host-only (no GPU needed).  `kernel` is a STEP_KERNELS name or code."""
    k = STEP_KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    buf = (ctypes.c_int * 32)()
    n = ctypes.c_int()
    rc = lib().wave_step_kernel_layout(int(space_order), int(ndim), k, int(bool(equal_spacing)), buf, 32,
                                       ctypes.byref(n))
    if rc != WAVE_OK:
        raise WaveError(rc, "bad arguments to wave_step_kernel_layout")
    return dict(zip(STEP_LAYOUT_FIELDS, list(buf)[:n.value]))


def wave_column_runs_for(columns, nz, chunks, space_order, slots=304, force=False):
    """Host-only: run starts of the segmented plain step for a grid of
    `columns` columns of nz planes (numpy int64 array of runs + 1 entries), or
    None where the z chunks are kept."""
    cap = int(min(slots, columns * nz)) + 1
    buf = (ctypes.c_longlong * cap)()
    n = ctypes.c_int()
    rc = lib().wave_column_runs_for(int(columns), int(nz), int(chunks), int(space_order), int(slots),
                                    int(bool(force)), buf, cap, ctypes.byref(n))
    if rc != WAVE_OK:
        raise WaveError(rc, "bad arguments to wave_column_runs_for")
    return np.array(buf[:n.value + 1], dtype=np.int64) if n.value else None


def wave_z_chunks_for(columns, nz, space_order, slots=304):
    """Host-only: chunks per column of the z-chunk grid of the plain 3D step."""
    c = ctypes.c_int()
    rc = lib().wave_z_chunks_for(int(columns), int(nz), int(space_order), int(slots), ctypes.byref(c))
    if rc != WAVE_OK:
        raise WaveError(rc, "bad arguments to wave_z_chunks_for")
    return int(c.value)


def wave_ricker(nt, dt, f0, t0=None, out=None):
    if t0 is None:
        t0 = 1.0 / f0
    out = _out("out", out, (int(nt),), None)
    rc = lib().wave_ricker(_ptr(out), int(nt), ctypes.c_float(dt), ctypes.c_float(f0), ctypes.c_float(t0))
    if rc != WAVE_OK:
        raise WaveError(rc, "bad arguments to wave_ricker")
    return out


def _noalloc_array(name, x, n=None):
    """Checks one array argument of wave_objective_noalloc without touching
    the GPU: a contiguous float32 torch tensor (of n elements when n is given)."""
    if not _is_torch(x):
        raise TypeError("%s must be a torch tensor on a CUDA device" % name)
    import torch
    if x.dtype != torch.float32:
        raise TypeError("%s must be float32, got %s" % (name, x.dtype))
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and x.numel() != n:
        raise ValueError("%s has %d elements, expected %d" % (name, x.numel(), n))


def wave_objective_noalloc(d, d_obs, r_out=None, stream=None):
    """(phi, r_out) of Eq. 2 for CUDA tensors d, d_obs without any allocation in
    the library; r = d - d_obs is written into ``r_out`` when given.  Every array
    is checked (type, size, device) before the call, so a mismatch raises
    instead of reaching the GPU."""
    _noalloc_array("d", d)
    n = int(d.numel())
    _noalloc_array("d_obs", d_obs, n)
    if r_out is not None:
        _noalloc_array("r_out", r_out, n)
    arrays = [d, d_obs] + ([r_out] if r_out is not None else [])
    if not all(a.is_cuda for a in arrays):
        raise ValueError("d, d_obs and r_out must be CUDA tensors")
    if len({a.device for a in arrays}) != 1:
        raise ValueError("d, d_obs and r_out must be on the same device")
    import torch
    if torch.cuda.current_device() != d.device.index:
        raise ValueError("the current CUDA device (%d) is not the tensors' device (%s)"
                         % (torch.cuda.current_device(), d.device))
    phi = ctypes.c_double()
    st = stream if stream is not None else _stream_for(d)
    rc = lib().wave_objective_noalloc(_ptr(d), _ptr(d_obs), _ptr(r_out), n, ctypes.byref(phi), st)
    if rc != WAVE_OK:
        raise WaveError(rc, "wave_objective_noalloc failed")
    return phi.value, r_out


def wave_error_string(code):
    return lib().wave_error_string(int(code)).decode()
