"""The oracle's bulk dynamics against textbook solutions: shear-wave decay
(nu = cs^2 (tau - 1/2), Eq. fluid_BGK / Eq. fluid_TRT_visc), plane Poiseuille
flow with halfway bounce-back walls that TRT with Lambda = 3/16 places exactly
half-way (Sec. 2.1), diffusion of a concentration wave with the rest-fraction
speed of sound (Eqs. solute_BGK, RestFractionCs2) and its advection with the
flow velocity (Eq. solute_equilibrium_function)."""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic


@pytest.mark.parametrize("q,dim,magic", [(9, 2, -1.0), (9, 2, 3.0 / 16.0), (19, 3, -1.0), (19, 3, 0.25)])
def test_shear_wave_decay(q, dim, magic):
    n, tau, U = 32, 0.9, 1e-4
    nz = 1 if dim == 2 else 2
    k = 2.0 * math.pi / n
    y = np.arange(n)
    u0 = np.zeros((nz, n, 2, 3))
    u0[..., 0] = U * np.sin(k * y)[None, :, None]
    p = dict(dim=dim, nx=2, ny=n, nz=nz, flow_q=q, solute_q=5 if dim == 2 else 7, bc=("periodic",) * 3,
             tau_flow=tau, magic_flow=magic, tau_solute=0.8)
    s = oracle.OracleSim(p, np.zeros((nz, n, 2), np.uint8), u_init=u0)
    proj = lambda: (s.fields()[0][..., 0] * np.sin(k * y)[None, :, None]).sum()
    s.step(200)
    a1 = proj()
    s.step(800)
    a2 = proj()
    rate = math.log(a1 / a2) / 800.0
    assert rate == pytest.approx(analytic.shear_wave_rate((tau - 0.5) / 3.0, k), rel=3e-3)


def _poiseuille_walls(magic):
    nx, ny, umax = 48, 18, 0.01
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0, :] = mask[0, ny - 1, :] = 1
    y = np.arange(ny, dtype=np.float64)
    prof = analytic.poiseuille(y, 0.5, ny - 1.5, umax)
    prof[0] = prof[-1] = 0.0
    p = dict(dim=2, nx=nx, ny=ny, flow_q=9, solute_q=5, bc=("open", "wall", "periodic"), tau_flow=0.8,
             magic_flow=magic, tau_solute=0.8, k_r=0.0)
    s = oracle.OracleSim(p, mask, inlet_ux=prof.reshape(1, ny))
    s.step(6000)
    u, rho, _, _ = s.fields()
    ux = u[0, 1:-1, nx // 2, 0]
    roots = np.sort(np.roots(np.polyfit(y[1:-1], ux, 2)).real)
    flux = (rho[0] * u[0, :, :, 0]).sum(axis=0)
    return roots, ux, prof[1:-1], flux


def test_poiseuille_trt_magic_puts_wall_halfway():
    roots, ux, prof, flux = _poiseuille_walls(3.0 / 16.0)
    assert roots[0] == pytest.approx(0.5, abs=1e-3) and roots[1] == pytest.approx(16.5, abs=1e-3)
    assert np.abs(ux / ux.max() - prof / prof.max()).max() < 1e-4
    assert flux.std() / flux.mean() < 1e-3
    # BGK at tau = 0.8 (Lambda = 0.09) visibly shifts the wall: the pin discriminates
    roots_bgk, _, _, _ = _poiseuille_walls(-1.0)
    assert abs(roots_bgk[0] - 0.5) > 5e-3


@pytest.mark.parametrize("q,dim,J0,magic", [(5, 2, -1.0, -1.0), (5, 2, 0.1, -1.0), (5, 2, 0.9, 3.0 / 16.0),
                                            (7, 3, -1.0, -1.0), (7, 3, 0.6, 0.25), (9, 2, -1.0, -1.0)])
def test_diffusion_wave(q, dim, J0, magic):
    n, tau = 40, 0.9 if J0 < 0.85 else 2.1
    nz = 1 if dim == 2 else 2
    k = 2.0 * math.pi / n
    x = np.arange(n)
    c0 = np.broadcast_to((1.0 + 0.1 * np.sin(k * x))[None, None, :], (nz, 2, n)).copy()
    p = dict(dim=dim, nx=n, ny=2, nz=nz, flow_q=0, solute_q=q, bc=("periodic",) * 3, tau_solute=tau,
             magic_solute=magic, rest_fraction=J0)
    s = oracle.OracleSim(p, np.zeros((nz, 2, n), np.uint8), c_init=c0)
    proj = lambda: ((s.fields()[2] - 1.0) * np.sin(k * x)[None, None, :]).sum()
    s.step(50)
    a1 = proj()
    s.step(300)
    a2 = proj()
    _, _, cs2, _ = oracle.lattice(q, dim, J0)
    rate = math.log(a1 / a2) / 300.0
    assert rate == pytest.approx(analytic.diffusion_wave_rate(cs2 * (tau - 0.5), k), rel=5e-3)


def test_advection_speed():
    # a uniform flow U advects the concentration wave at speed U
    n, U = 64, 0.02
    k = 2.0 * math.pi / n
    x = np.arange(n)
    c0 = np.broadcast_to((1.0 + 0.1 * np.sin(k * x))[None, None, :], (2, 2, n)).copy()
    u0 = np.zeros((2, 2, n, 3))
    u0[..., 0] = U
    p = dict(dim=3, nx=n, ny=2, nz=2, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.8,
             tau_solute=0.7, rest_fraction=0.4)
    s = oracle.OracleSim(p, np.zeros((2, 2, n), np.uint8), u_init=u0, c_init=c0)
    T = 400
    s.step(T)
    c = s.fields()[2][0, 0] - 1.0
    phase = math.atan2((c * np.cos(k * x)).sum(), (c * np.sin(k * x)).sum())
    assert -phase / k == pytest.approx(U * T, rel=1e-2)
