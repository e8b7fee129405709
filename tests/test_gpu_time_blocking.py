"""GPU parity of the two-level pass (temporal blocking; Sec. VI lists time
tiling as future work): source-free 3D forward modelling at space order 8 from
a random initial state, with two leapfrog levels of Listing 1 / Eq. 1 per pass,
against the FP64 oracle and against the single-level path of the library.
Grids with ragged x and axis-1 tiles, several z chunks, odd and even numbers
of levels (an odd last level takes the single-level step), and no sponge."""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from gpu_cases import f32, geometries, rel_l2

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import wave  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [((83, 37, 40), (10.0, 12.0, 9.0), 4, 9),     # one z chunk, odd number of levels after the first
         ((70, 30, 120), (10.0, 10.0, 10.0), 4, 12),  # four z chunks, even
         ((130, 21, 70), (9.0, 11.0, 10.0), 0, 7),    # no sponge, three x tiles
         ((17, 5, 9), (10.0, 10.0, 10.0), 2, 6)]      # grid smaller than one tile


@pytest.mark.parametrize("shape,spacing,nbl,nt", CASES)
def test_two_level_forward_matches_oracle(shape, spacing, nbl, nt):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so = 8
    og = oracle.model.Geometry(shape=shape, spacing=spacing, nbl=nbl, sponge_vref=2.5)
    _, geom = geometries(og)
    r = np.random.default_rng(sum(shape) + nt)
    m = (1.0 / (1.5 + r.uniform(size=og.phys_array_shape)) ** 2).astype(np.float32)
    dt = f32(0.4 * oracle.model.dt_max(so, spacing, 2.5))
    lo = np.array(og.origin)
    hi = lo + (np.array(shape) - 1) * np.array(spacing)
    rec = (lo + r.uniform(size=(13, 3)) * (hi - lo)).astype(np.float32)
    u0 = r.standard_normal(og.array_shape).astype(np.float32)
    u1 = r.standard_normal(og.array_shape).astype(np.float32)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    out = {}
    with wave.Context(0) as c:
        for levels in (2, 1):
            c.set_time_blocking(levels)
            d, fp, fl = wave.wave_forward(c, geom, dev(m), None, None, rec, dt, nt, so, u_init_prev=dev(u0),
                                          u_init=dev(u1), return_final=True)
            out[levels] = (d.cpu().numpy(), fp.cpu().numpy(), fl.cpu().numpy())
    n = int(np.prod(og.array_shape))
    Pr = oracle.interp.interpolation_matrix(og, rec)
    ref = oracle.wave.forward_op(oracle.model.pad_model(og, m), oracle.model.damping(og), og.spacing, dt, nt, so,
                                 np.zeros((nt, 1)), sp.csr_matrix((1, n)), Pr, u_init_prev=u0, u_init=u1)
    d2, fp2, fl2 = out[2]
    scale = np.abs(ref.u_last).max()
    e_d = rel_l2(d2, ref.d)
    e_f = max(np.abs(fl2 - ref.u_last).max(), np.abs(fp2 - ref.u_prev).max()) / scale
    e_1 = max(np.abs(fl2 - out[1][2]).max(), np.abs(fp2 - out[1][1]).max()) / scale
    print("two-level pass %s nt%d: receivers rel-L2 %.2e, field %.2e vs oracle, %.2e vs single levels"
          % ("x".join(map(str, shape)), nt, e_d, e_f, e_1))
    assert e_d <= 1e-5 and e_f <= 1e-5 and e_1 <= 1e-5


def test_time_blocking_setting_is_checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with wave.Context(0) as c:
        for bad in (0, 3, -1):
            with pytest.raises(wave.WaveError) as e:
                c.set_time_blocking(bad)
            assert e.value.code == wave.WAVE_ERR_INVALID_ARG
