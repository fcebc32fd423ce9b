"""FP32 deviation storage against the FP64 path over the channel grid of
Pe in {1, 10, 100} (rest fraction: J0 up to 0.98 at Pe = 100), Da in
{0.1, 1, 10} and walls tilted 0 / 30 / 45 degrees (reduced channels of the
256x128x128 case, same Re = 1 and c_in = 1, c_eq = 0.5).  The FP64 path is
first matched against the oracle on every point of the grid; the FP32
populations must then stay within relative L2 1e-5 of it in c and u after
2000 steps."""
import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import lbrbc, workloads

pytestmark = pytest.mark.gpu
GRID = [(t, pe, da) for t in (0.0, 30.0, 45.0) for pe in (1.0, 10.0, 100.0) for da in (0.1, 1.0, 10.0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()
    oracle.build()


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("theta,pe,da", GRID)
def test_fp64_matches_oracle_on_the_channel_grid(theta, pe, da):
    p, mask, extra = workloads.case_channel(nx=40, ny=28, nz=28, h=9.0, theta_deg=theta, Pe=pe, Da=da)
    g = lbrbc.Sim(dict(p, precision="fp64"), mask, **extra)
    o = oracle.OracleSim(p, mask, **extra)
    g.step(25)
    o.step(25)
    g.check()
    for a, b in zip(g.fields(), o.fields()):
        assert np.abs(a - b).max() < 1e-11
    assert g.ledger()["reacted"] == pytest.approx(o.ledger()["reacted"], rel=1e-9)
    g.close()


@pytest.mark.parametrize("theta,pe,da", GRID)
def test_fp32_within_1e5_of_fp64_after_2000_steps(theta, pe, da):
    p, mask, extra = workloads.case_channel(nx=96, ny=48, nz=48, h=12.0, theta_deg=theta, Pe=pe, Da=da)
    s64 = lbrbc.Sim(dict(p, precision="fp64"), mask, **extra)
    s32 = lbrbc.Sim(dict(p, precision="fp32"), mask, **extra)
    s64.step(2000)
    s32.step(2000)
    s32.check()
    u64, _, c64, _ = s64.fields()
    u32, _, c32, _ = s32.fields()
    ec, eu = rel_l2(c32, c64), rel_l2(u32, u64)
    assert ec <= 1e-5 and eu <= 1e-5, (ec, eu, p["rest_fraction"])
    s64.close()
    s32.close()
