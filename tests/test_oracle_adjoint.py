"""Pins of the oracle's discrete adjoint of the reacted mass (the paper has
no gradient; the adjoint differentiates the oracle's own step): the
gradients with respect to k_r, c_eq and a per-voxel k field against central
finite differences of the oracle's forward runs, for the three finite-k
schemes, BGK and TRT, with and without flow and with open boundaries; the
reacted mass is exactly linear in c_eq, so that derivative matches to
round-off.  A dropped term or a wrong sign in any transposed stage (pull,
reactive boundary condition, ledger, collision) moves these by far more than
the finite-difference error."""
import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import workloads


def _case(flow=True, scheme="new", trt=False, shape=(6, 8, 16)):
    nz, ny, nx = shape
    mask = workloads.sphere_pack(shape, 0.6, 1.5, 2.5, seed=13, periodic=(False, True, True), buffer_x=2)
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19 if flow else 0, solute_q=7, bc=("open", "periodic", "periodic"),
             tau_flow=0.8, magic_flow=3.0 / 16.0, tau_solute=0.9, magic_solute=0.25 if trt else -1.0,
             rest_fraction=0.4, k_r=0.05, c_eq=1.0, c_init=0.2, c_inlet=0.0, u_inlet=0.01, rho_outlet=1.0,
             molar_volume=0.1, scheme=scheme)
    return p, mask


def _J(p, mask, n, **init):
    o = oracle.OracleSim(p, mask, **init)
    L0 = o.ledger()["reacted"]
    o.step(n)
    return o.ledger()["reacted"] - L0


@pytest.mark.parametrize("flow,scheme,trt", [(True, "new", False), (True, "verhaeghe", True),
                                             (False, "patel_ju", False), (True, "new", True)])
def test_scalar_gradients_match_central_differences(flow, scheme, trt):
    p, mask = _case(flow, scheme, trt)
    n = 40
    J, dk, dc, _ = oracle.OracleSim(p, mask).adjoint(n)
    assert J == pytest.approx(_J(p, mask, n), rel=1e-13)
    h = 1e-4 * p["k_r"]
    fd = (_J(dict(p, k_r=p["k_r"] + h), mask, n) - _J(dict(p, k_r=p["k_r"] - h), mask, n)) / (2 * h)
    assert dk == pytest.approx(fd, rel=1e-6), (dk, fd)
    # J is affine in c_eq for fixed k: any step gives the exact derivative
    h = 0.25
    fd = (_J(dict(p, c_eq=p["c_eq"] + h), mask, n) - _J(dict(p, c_eq=p["c_eq"] - h), mask, n)) / (2 * h)
    assert dc == pytest.approx(fd, rel=1e-9), (dc, fd)
    assert dk != 0.0 and dc != 0.0


def test_kfield_gradient_matches_central_differences():
    p, mask = _case()
    n = 30
    kf = workloads.lognormal_k(mask.shape, 0.05, 0.5, seed=9)
    o = oracle.OracleSim(p, mask, k_field=kf)
    J, dk, dc, g = o.adjoint(n, field=True)
    cls = o.classes()
    assert np.all(g[cls != oracle.BOUND] == 0.0)
    assert dk == pytest.approx(g.sum(), rel=1e-12)
    bound = np.argwhere((cls == oracle.BOUND) & (mask == 1))
    rng = np.random.default_rng(1)
    for z, y, x in bound[rng.choice(len(bound), 5, replace=False)]:
        h = 1e-3 * kf[z, y, x]
        kp, km = kf.copy(), kf.copy()
        kp[z, y, x] += h
        km[z, y, x] -= h
        fd = (_J(p, mask, n, k_field=kp) - _J(p, mask, n, k_field=km)) / (2 * h)
        assert g[z, y, x] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(dk)), (x, y, z)


def test_dirichlet_cells_and_anti_bounce_back():
    # Dirichlet cells inject mass that is not reacted mass; under the
    # anti-bounce-back scheme J depends on c_eq only
    shape = (4, 10, 12)
    mask = workloads.sphere_pack(shape, 0.6, 1.5, 2.5, seed=5, periodic=(True, False, True))
    mask[:, -1, :] = workloads.DIRICHLET
    p = dict(dim=3, nx=12, ny=10, nz=4, flow_q=0, solute_q=7, bc=("periodic", "wall", "periodic"), tau_solute=0.8,
             k_r=0.1, c_eq=0.5, c_init=0.0, c_dirichlet=1.0, scheme="anti_bb")
    J, dk, dc, _ = oracle.OracleSim(p, mask).adjoint(25)
    assert dk == 0.0
    h = 0.1
    fd = (_J(dict(p, c_eq=0.5 + h), mask, 25) - _J(dict(p, c_eq=0.5 - h), mask, 25)) / (2 * h)
    assert dc == pytest.approx(fd, rel=1e-9)
    p2 = dict(p, scheme="new")
    J, dk, dc, _ = oracle.OracleSim(p2, mask).adjoint(25)
    hk = 1e-4 * p2["k_r"]
    fd = (_J(dict(p2, k_r=p2["k_r"] + hk), mask, 25) - _J(dict(p2, k_r=p2["k_r"] - hk), mask, 25)) / (2 * hk)
    assert dk == pytest.approx(fd, rel=1e-6)


def test_adjoint_needs_phase_change_off():
    p, mask = _case()
    with pytest.raises(ValueError):
        oracle.OracleSim(dict(p, phase_change=1), mask).adjoint(3)
