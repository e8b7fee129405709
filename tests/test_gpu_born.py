"""GPU checks of linearised (Born) modelling: J dm against the oracle, and the
adjoint pair <J dm, y> = <dm, J^T y> with J^T from wave_jacobian_adjoint."""

import numpy as np
import pytest

import oracle
from gpu_cases import geometries, rel_l2, small2d, small3d

torch = pytest.importorskip("torch")
from paper_1608_08658_gb300 import wave  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = wave.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("case", ["3d2", "3d4", "3d6", "3d8", "3d10", "2d4", "3d12", "3d14", "3d16", "3d8iso",
                                  "3d14iso", "3d16iso"])
def test_born_matches_oracle(ctx, case):
    so = int(case[2:].replace("iso", ""))
    h = (10.0, 10.0, 10.0) if case.endswith("iso") else (10.0, 12.0, 9.0)
    og, m, dt, nt, so, src, q, rec = small3d(so, spacing=h) if case.startswith("3d") else small2d(so)
    _, geom = geometries(og)
    rng = np.random.default_rng(41)
    dm = (0.05 * m * rng.uniform(-1, 1, size=m.shape)).astype(np.float32)
    jd = wave.wave_born(ctx, geom, _dev(m), _dev(dm), src, _dev(q), rec, dt, nt, so).cpu().numpy()
    ref = oracle.wave.born(og, m, dm, dt, nt, so, q, src, rec)
    err = rel_l2(jd, ref)
    print("%s Born: rel-L2 vs oracle %.3e" % (case, err))
    assert err <= 1e-4


@pytest.mark.parametrize("case", ["3d8", "2d6"])
def test_born_adjoint_pair(ctx, case):
    og, m, dt, nt, so, src, q, rec = small3d(8) if case == "3d8" else small2d(6)
    _, geom = geometries(og)
    rng = np.random.default_rng(42)
    dm = (0.05 * m * rng.uniform(-1, 1, size=m.shape)).astype(np.float32)
    y = rng.standard_normal((nt, len(rec))).astype(np.float32)
    jd = wave.wave_born(ctx, geom, _dev(m), _dev(dm), src, _dev(q), rec, dt, nt, so)
    jty = wave.wave_jacobian_adjoint(ctx, geom, _dev(m), src, _dev(q), rec, _dev(y), dt, nt, so,
                                     snap_mode="full_fp32")
    lhs = float((jd.double() * _dev(y).double()).sum())
    rhs = float((_dev(dm).double() * jty.double()).sum())
    print("%s <J dm, y> = %.9e, <dm, J^T y> = %.9e (rel %.2e)" % (case, lhs, rhs, abs(lhs - rhs) / abs(lhs)))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))
