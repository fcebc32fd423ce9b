"""Wall-orientation behaviour of the oracle's reactive boundary schemes
(Sec. 3.1.2, Sec. 3.2): on a staircase circle every wall orientation occurs.

* The total reaction rate of a reactive disk inside a Dirichlet circle is
  compared with the closed form of steady radial diffusion; the new scheme
  (Eq. k_i_S_New) matches it, the scheme without gamma (Eq. k_i_S_Ve) reacts
  too slowly and the scheme with the normal in the denominator (Eq. k_i_S2)
  too fast, in the order Table 2 (case 4) reports.
* The flux through diagonal wall sectors relative to axis-aligned ones is
  near 1 for the new scheme and clearly above 1 for Eq. k_i_S2, which the
  paper attributes to faster reactions on diagonal walls (Sec. 3.2).
* The isotropic-gradient normal is exact on flat and 45-degree walls.
Tolerances are proposed here (the paper gives these results as figures).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_2306_10794_gb300 import workloads

N, R, R2, TAU = 72, 12.0, 32.0, 1.0


def _run(scheme):
    mask, c = workloads.annulus(N, R, R2, 0.3)
    D = (TAU - 0.5) / 3.0
    k_r = D / R  # PeDa = 1 on the disk radius
    p = dict(dim=2, nx=N, ny=N, flow_q=0, solute_q=5, bc=("wall", "wall", "periodic"), tau_solute=TAU, k_r=k_r,
             c_eq=0.0, c_dirichlet=1.0, c_init=1.0, scheme=scheme)
    s = oracle.OracleSim(p, mask)
    s.step(5000)
    M = s.reacted()[0]
    b = (s.classes()[0] == oracle.BOUND) & (mask[0] == 1)
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    ang = np.arctan2(yy[b] - c, xx[b] - c)
    m = -M[b]
    quarter = np.mod(ang + math.pi / 8.0, math.pi / 2.0)
    axis, diag = m[quarter < math.pi / 4.0].sum(), m[quarter >= math.pi / 4.0].sum()
    exact = analytic.annulus_rate(R, R2, k_r, D, 1.0, 0.0)
    return m.sum() / exact, diag / axis


@pytest.fixture(scope="module")
def results():
    return {s: _run(s) for s in ("new", "verhaeghe", "patel_ju")}


def test_total_rate_against_closed_form(results):
    new, ve, pj = results["new"][0], results["verhaeghe"][0], results["patel_ju"][0]
    assert abs(new - 1.0) < 0.05
    assert ve < 0.8 * new < pj / 1.15


def test_diagonal_vs_axis_walls(results):
    assert abs(results["new"][1] - 1.0) < 0.1
    assert results["patel_ju"][1] > 1.2


def test_normals_flat_and_diagonal():
    n = 24
    mask = np.zeros((1, n, n), np.uint8)
    mask[0, :8, :] = 1
    p = dict(dim=2, nx=n, ny=n, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"))
    nrm = oracle.OracleSim(p, mask).normals()
    assert np.allclose(nrm[0, 7, :, :], [0.0, 1.0, 0.0], atol=1e-15)
    yy, xx = np.mgrid[0:n, 0:n]
    mask = np.where(yy < xx, 1, 0).astype(np.uint8)[None]
    p = dict(dim=2, nx=n, ny=n, flow_q=0, solute_q=5, bc=("wall", "wall", "periodic"))
    s = oracle.OracleSim(p, mask)
    nrm = s.normals()[0]
    b = s.classes()[0] == oracle.BOUND
    inner = b & (xx > 3) & (xx < n - 4)
    assert inner.sum() > 10
    assert np.allclose(nrm[inner], [-math.sqrt(0.5), math.sqrt(0.5), 0.0], atol=1e-14)
