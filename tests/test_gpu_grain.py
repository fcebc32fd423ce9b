"""Grain growth during precipitation (Sec. 3.2) on the GPU: a star-shaped
seed (four lobes) in the centre of a 300 x 300 circle of fixed concentration,
k_r = 0.0014, C_eq = 0, pure diffusion, seeds aligned with the grid and
turned clockwise by 19 degrees, 300 000 steps.  The paper shows the grains
as figures; what they show is checked through the grain's largest radius in
5-degree sectors:

* the new scheme grows the grain along the seed's lobes, whatever the
  seed's orientation: the two grains nearly identical once turned back, the
  lobes of the turned run within 10 degrees of the seed's (they drift by
  about 8 degrees towards the grid axes while the grain triples its radius),
  where S.P.J.'s lie on the grid diagonals;
* the scheme with the wall normal in the denominator (S.P.J.) grows fastest
  on diagonal walls: its lobes lie on the grid diagonals for both seeds,
  and the grain is strongly anisotropic;
* the scheme without gamma (S.V.) grows less (its effective rate is
  k_r / gamma);
* sum C + sum phi / V_m - (Dirichlet inflow) stays constant through the
  phase changes: to 1e-9 with FP64 populations; the FP32 runs drift by the
  accumulated rounding of 2.7e10 cell updates (below 2e-3)."""
import math

import numpy as np
import pytest

from paper_2306_10794_gb300 import lbrbc, workloads

pytestmark = pytest.mark.gpu
STEPS = 300_000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()


def grow(scheme, angle, precision="fp32", steps=STEPS):
    p, mask, init, geom = workloads.case_grain_2d(angle, scheme, precision=precision)
    s = lbrbc.Sim(p, mask, **init)
    inv = lambda L: L["solute"] + L["solid_over_vm"] + L["unpaid"] - L["dirichlet_in"]
    I0 = inv(s.ledger())
    s.step(steps)
    s.check()
    I1 = inv(s.ledger())
    grain = (s.classes()[0] != 0) & geom["inside"][0]
    s.close()
    return grain, (I0, I1)


def sector_radii(m):
    n = m.shape[0]
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.hypot(xx - c, yy - c)[m]
    th = np.degrees(np.arctan2((yy - c)[m], (xx - c)[m])) % 360.0
    rmax = np.zeros(72)
    np.maximum.at(rmax, (th // 5).astype(int) % 72, r)
    return rmax


def lobe_angle(rmax):
    # orientation (mod 90 degrees) of a four-lobed shape from its sector radii
    th = np.radians(np.arange(72) * 5.0 + 2.5)
    z = (rmax * np.exp(4j * th)).sum()
    return math.degrees(np.angle(z)) / 4.0 % 90.0


def turned_back(m, angle):
    n = m.shape[0]
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    a = math.radians(-angle)
    xs = c + (xx - c) * math.cos(a) - (yy - c) * math.sin(a)
    ys = c + (xx - c) * math.sin(a) + (yy - c) * math.cos(a)
    return m[np.clip(np.rint(ys).astype(int), 0, n - 1), np.clip(np.rint(xs).astype(int), 0, n - 1)]


def iou(a, b):
    return float((a & b).sum()) / float((a | b).sum())


def adiff(a, b):
    # distance of two angles mod 90 degrees
    d = (a - b) % 90.0
    return min(d, 90.0 - d)


@pytest.fixture(scope="module")
def grains():
    return {(s, a): grow(s, a) for s, a in (("new", 0.0), ("new", 19.0), ("patel_ju", 0.0), ("patel_ju", 19.0),
                                            ("verhaeghe", 0.0))}


def test_new_scheme_follows_the_seed(grains):
    g0, g19 = grains["new", 0.0][0], grains["new", 19.0][0]
    a0, a19 = lobe_angle(sector_radii(g0)), lobe_angle(sector_radii(g19))
    assert adiff(a0, 0.0) < 5.0, a0
    assert adiff(a19, -19.0) < 10.0, a19
    a19_pj = lobe_angle(sector_radii(grains["patel_ju", 19.0][0]))
    assert adiff(a19_pj, -19.0) > adiff(a19, -19.0) + 10.0, (a19_pj, a19)
    assert iou(g0, turned_back(g19, 19.0)) > 0.9
    r = sector_radii(g0)
    assert r.max() / r.min() < 1.25


def test_patel_ju_grows_along_grid_diagonals(grains):
    for angle in (0.0, 19.0):
        r = sector_radii(grains["patel_ju", angle][0])
        assert adiff(lobe_angle(r), 45.0) < 5.0, (angle, lobe_angle(r))
        assert r.max() / r.min() > 1.3
    rot_pj = iou(grains["patel_ju", 0.0][0], turned_back(grains["patel_ju", 19.0][0], 19.0))
    rot_new = iou(grains["new", 0.0][0], turned_back(grains["new", 19.0][0], 19.0))
    assert rot_pj < rot_new - 0.1


def test_verhaeghe_grows_less(grains):
    assert grains["verhaeghe", 0.0][0].sum() < 0.7 * grains["new", 0.0][0].sum()


def test_mass_invariant_through_phase_change(grains):
    grain, (I0, I1) = grow("new", 19.0, precision="fp64", steps=100_000)
    assert grain.sum() > 4000  # the seed (2880 cells) has grown
    assert abs(I1 - I0) < 1e-9 * abs(I0), (I0, I1)
    for key, (_, (J0, J1)) in grains.items():
        assert abs(J1 - J0) < 2e-3 * abs(J0), (key, J0, J1)
