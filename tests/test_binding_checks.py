"""Argument checks of the Python binding (no GPU, no library call): every array
handed to the C ABI must hold exactly the elements the header documents for it
(the library reads or writes that many through a raw pointer), and every
caller-supplied output must be contiguous float32.  A mismatch raises before
the library is reached; a correct call goes through to it."""

import numpy as np
import pytest
import torch

from paper_1608_08658_gb300 import wave


class _Reached(Exception):
    pass


class _StubLib:
    """Stands in for libwave.so: any entry point raises _Reached."""

    def __getattr__(self, name):
        def call(*args, **kwargs):
            raise _Reached(name)
        return call


class _Ctx:
    handle = None


@pytest.fixture(autouse=True)
def stub_lib(monkeypatch):
    monkeypatch.setattr(wave, "lib", lambda: _StubLib())


NT = 7
GEOM3 = wave.Geometry(shape=(12, 10, 8), spacing=(10.0, 10.0, 10.0), nbl=3, sponge_vref=2.0)
SRC = np.array([[40.0, 50.0, 30.0]], np.float32)
REC = np.array([[20.0, 30.0, 10.0], [60.0, 40.0, 10.0]], np.float32)


def _m(shape=None):
    return np.full(shape or GEOM3.phys_array_shape, 0.25, np.float32)


def _q(rows=NT, cols=1):
    return np.ones((rows, cols), np.float32)


def _d(rows=NT, cols=2, dtype=np.float32):
    return np.zeros((rows, cols), dtype)


def test_valid_arguments_reach_the_library():
    with pytest.raises(_Reached, match="wave_forward_ex"):
        wave.wave_forward(_Ctx(), GEOM3, _m(), SRC, _q(), REC, 1.0, NT, 4)
    with pytest.raises(_Reached, match="wave_gradient"):
        wave.wave_gradient(_Ctx(), GEOM3, torch.from_numpy(_m()), SRC, _q(), REC, _d(), 1.0, NT, 4,
                           grad_out=torch.empty(GEOM3.phys_array_shape))
    with pytest.raises(_Reached, match="wave_forward_ex"):
        comp = np.zeros(GEOM3.comp_array_shape, np.float32)
        wave.wave_forward(_Ctx(), GEOM3, _m(), None, None, REC, 1.0, NT, 4, u_init_prev=comp, u_init=comp)


@pytest.mark.parametrize("what", ["m", "q", "u_init", "u_init_prev"])
def test_forward_inputs_of_the_wrong_size(what):
    args = dict(m=_m(), q=_q())
    kw = {}
    if what == "m":
        args["m"] = _m((8, 10, 11))                       # one x column short
    elif what == "q":
        args["q"] = _q(rows=NT - 1)                       # one time row short
    else:
        kw[what] = np.zeros(GEOM3.phys_array_shape, np.float32)   # physical instead of computational grid
    with pytest.raises(ValueError, match="^%s has" % what):
        wave.wave_forward(_Ctx(), GEOM3, args["m"], SRC, args["q"], REC, 1.0, NT, 4, **kw)


def test_forward_output_checks():
    with pytest.raises(ValueError, match="^d_out (has|must)"):
        wave.wave_forward(_Ctx(), GEOM3, _m(), SRC, _q(), REC, 1.0, NT, 4, d_out=_d(rows=NT - 1))
    with pytest.raises(TypeError, match="^d_out (has|must)"):
        wave.wave_forward(_Ctx(), GEOM3, _m(), SRC, _q(), REC, 1.0, NT, 4, d_out=_d(dtype=np.float64))
    with pytest.raises(TypeError, match="^d_out (has|must)"):
        wave.wave_forward(_Ctx(), GEOM3, _m(), SRC, _q(), REC, 1.0, NT, 4,
                          d_out=torch.zeros((NT, 2), dtype=torch.float64))
    with pytest.raises(ValueError, match="^d_out (has|must)"):
        wave.wave_forward(_Ctx(), GEOM3, _m(), SRC, _q(), REC, 1.0, NT, 4, d_out=torch.zeros((2, NT)).t())


def test_adjoint_checks():
    with pytest.raises(ValueError, match="^y (has|must)"):
        wave.wave_adjoint(_Ctx(), GEOM3, _m(), SRC, REC, _d(cols=3), 1.0, NT, 4)
    with pytest.raises(ValueError, match="^q_out (has|must)"):
        wave.wave_adjoint(_Ctx(), GEOM3, _m(), SRC, REC, _d(), 1.0, NT, 4, q_out=_q(cols=2))


def test_gradient_checks():
    with pytest.raises(ValueError, match="^d_obs (has|must)"):
        wave.wave_gradient(_Ctx(), GEOM3, _m(), SRC, _q(), REC, _d(rows=NT + 1), 1.0, NT, 4)
    with pytest.raises(ValueError, match="^grad_out (has|must)"):
        wave.wave_gradient(_Ctx(), GEOM3, _m(), SRC, _q(), REC, _d(), 1.0, NT, 4,
                           grad_out=np.zeros(GEOM3.comp_array_shape, np.float32))
    with pytest.raises(TypeError, match="^grad_out (has|must)"):
        wave.wave_gradient(_Ctx(), GEOM3, _m(), SRC, _q(), REC, _d(), 1.0, NT, 4,
                           grad_out=np.zeros(GEOM3.phys_array_shape, np.float64))
    with pytest.raises(ValueError, match="^y (has|must)"):
        wave.wave_jacobian_adjoint(_Ctx(), GEOM3, _m(), SRC, _q(), REC, _d(rows=1), 1.0, NT, 4)
    with pytest.raises(ValueError, match="^d_out (has|must)"):
        wave.wave_jacobian_adjoint(_Ctx(), GEOM3, _m(), SRC, _q(), REC, _d(), 1.0, NT, 4, d_out=_d(cols=1))


def test_multi_shot_checks_name_the_shot():
    shots = [(SRC, _q(), REC, _d()), (SRC, _q(), REC, _d(rows=NT - 2))]
    with pytest.raises(ValueError, match="d_obs of shot 1"):
        wave.wave_gradient_shots(_Ctx(), GEOM3, _m(), shots, 1.0, NT, 4)
    shots = [(SRC, _q(cols=2), REC, _d())]
    with pytest.raises(ValueError, match="q of shot 0"):
        wave.wave_gradient_shots(_Ctx(), GEOM3, _m(), shots, 1.0, NT, 4)


def test_born_and_session_checks():
    with pytest.raises(ValueError, match="^dm (has|must)"):
        wave.wave_born(_Ctx(), GEOM3, _m(), _m((1, 10, 8)), SRC, _q(), REC, 1.0, NT, 4)
    with pytest.raises(ValueError, match="^q (has|must)"):
        wave.Session(_Ctx(), GEOM3, _m(), SRC, _q(rows=NT + 3), REC, 1.0, NT, 4)


def test_ricker_output_checks():
    with pytest.raises(ValueError, match="^out (has|must)"):
        wave.wave_ricker(10, 1.0, 0.01, out=np.zeros(9, np.float32))
    with pytest.raises(TypeError, match="^out (has|must)"):
        wave.wave_ricker(10, 1.0, 0.01, out=np.zeros(10, np.float64))
