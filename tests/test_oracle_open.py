"""Pins of the oracle's open boundaries (Sec. 3.3 names a plug inlet, a fixed
outlet density and zero concentration gradient at the outlet; the schemes are
reading R9).  Inlet: moving-wall bounce-back for f and anti-bounce-back for g
with C = c_in at the wall half a cell before x = 0.  Outlet: pressure
anti-bounce-back for f and anti-bounce-back for g with the wall value set to
the outlet cell's own previous C, which makes the gradient vanish at the wall
half a cell beyond x = nx - 1.  Every mass that crosses an open face is booked
in the ledger's open-boundary term.

The pins: the uniform plug-flow state with C = c_in is an exact fixed point
(each rule reproduces the equilibrium exactly); the solute sum changes by the
open-boundary term and nothing else; an advancing front matches the
Ogata-Banks closed form; and pure diffusion between an inlet and the outlet
matches the Fourier series of the Dirichlet-Neumann problem, with the two
walls where the readings put them.  A flipped sign or weight in any of the
open rules breaks at least one of them (checked by planting each mistake in
a copy of the oracle).  Plain bounce-back at the outlet is also zero-gradient
for pure diffusion; the plug-flow fixed point is what rules it out."""
import math

import numpy as np
import pytest
from scipy.special import erfc

import oracle


def _plug(nx, ny, nz, u_in, c0, **over):
    shape = (nz, ny, nx)
    u0 = np.zeros(shape + (3,))
    u0[..., 0] = u_in
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"),
             tau_flow=0.8, tau_solute=0.9, c_inlet=1.0, u_inlet=u_in, rho_outlet=1.0)
    p.update(over)
    c0 = np.broadcast_to(np.asarray(c0, dtype=float), shape).copy()
    return oracle.OracleSim(p, np.zeros(shape, np.uint8), u_init=u0, c_init=c0), shape


@pytest.mark.parametrize("magic", [-1.0, 3.0 / 16.0])
@pytest.mark.parametrize("rest_fraction", [-1.0, 0.4])
def test_plug_flow_with_inlet_concentration_is_a_fixed_point(magic, rest_fraction):
    u_in, c_in = 0.05, 1.7
    s, shape = _plug(24, 3, 3, u_in, c_in, c_inlet=c_in, magic_flow=magic, magic_solute=magic,
                     rest_fraction=rest_fraction)
    s.step(60)
    u, rho, c, _ = s.fields()
    assert np.abs(c - c_in).max() < 1e-13
    assert np.abs(u[..., 0] - u_in).max() < 1e-14 and np.abs(u[..., 1:]).max() < 1e-14
    assert np.abs(rho - 1.0).max() < 1e-14
    # the inflow and outflow balance: the open-boundary term stays at round-off
    # while each face carries u_in * c_in per cell and step
    assert abs(s.ledger()["open_in"]) < 1e-11


def test_solute_sum_changes_by_the_open_boundary_term_every_step():
    # a front entering an empty plug-flow channel with reactive-free walls
    s, shape = _plug(30, 4, 3, 0.04, 0.0, bc=("open", "wall", "periodic"), k_r=0.0)
    c0 = s.fields()[2].sum()
    for _ in range(40):
        s.step(1)
        L = s.ledger()
        assert L["solute"] - c0 == pytest.approx(L["open_in"], rel=1e-13, abs=1e-14)
    assert L["open_in"] > 0.5


def test_open_channel_with_reactive_walls_balances_mass():
    # reaction on the walls and both open faces: solute + solid / V_m changes
    # by the open-boundary term only
    nz, ny, nx = 3, 6, 28
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, 0, :] = mask[:, -1, :] = 1
    u0 = np.zeros((nz, ny, nx, 3))
    u0[:, 1:-1, :, 0] = 0.03
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19, solute_q=7, bc=("open", "wall", "periodic"), tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.8, k_r=0.05, c_eq=0.2, c_init=0.0, c_inlet=1.0, u_inlet=0.03,
             molar_volume=0.5)
    s = oracle.OracleSim(p, mask, u_init=u0)
    L0 = s.ledger()
    s.step(120)
    L = s.ledger()
    assert L["reacted"] != 0.0 and L["open_in"] > 0.0
    I0 = L0["solute"] + L0["solid_over_vm"]
    I1 = L["solute"] + L["solid_over_vm"] - L["open_in"]
    assert I1 == pytest.approx(I0, rel=1e-13)


def test_inlet_front_matches_ogata_banks():
    # C(x, t) = 1/2 [erfc((x - u t) / 2 sqrt(D t)) + exp(u x / D) erfc((x + u t) / 2 sqrt(D t))]
    # with x measured from the inlet wall half a cell before the first cell.
    # The first-order equilibrium of Eq. solute_equilibrium_function carries
    # the numerical diffusion -(tau - 1/2) u^2 along the flow, so the
    # effective D is (tau - 1/2)(cs^2 - u^2); with the plain cs^2 (tau - 1/2)
    # the error is 7e-4.  Outlet 240 cells away: the front never reaches it.
    nx, u_in, tau, J0, T = 240, 0.02, 1.0, 0.25, 3000
    s, _ = _plug(nx, 1, 1, u_in, 0.0, tau_solute=tau, rest_fraction=J0)
    s.step(T)
    c = s.fields()[2][0, 0]
    D = (tau - 0.5) * ((1.0 - J0) / 3.0 - u_in ** 2)
    x = np.arange(nx) + 0.5
    ob = 0.5 * (erfc((x - u_in * T) / (2 * math.sqrt(D * T))) +
                np.exp(u_in * x / D) * erfc((x + u_in * T) / (2 * math.sqrt(D * T))))
    assert np.abs(c - ob).max() < 1e-3
    assert c[0] > 0.9 and c[-1] < 1e-9


@pytest.mark.parametrize("T", [2000, 8000, 30000])
def test_outlet_is_zero_gradient_half_a_cell_beyond_the_last_cell(T):
    # Pure diffusion (no flow lattice) from C = 1 at the inlet wall x' = 0 to
    # the zero-gradient outlet wall x' = L, x' = x + 1/2, L = nx:
    #   C = 1 - sum_n 4 / ((2n+1) pi) sin(k_n x') exp(-D k_n^2 t), k_n = (2n+1) pi / (2 L).
    # The series with the outlet wall one cell further in (L = nx - 1) differs
    # from this one by 2e-3 / 1.5e-2 / 8e-3 at the three times, so the test
    # fixes where the zero gradient sits.
    nx, tau, J0 = 60, 1.0, 0.25
    D = (1.0 - J0) / 3.0 * (tau - 0.5)
    p = dict(dim=3, nx=nx, ny=1, nz=1, flow_q=0, solute_q=7, bc=("open", "periodic", "periodic"), tau_solute=tau,
             rest_fraction=J0, c_init=0.0, c_inlet=1.0)
    s = oracle.OracleSim(p, np.zeros((1, 1, nx), np.uint8))
    s.step(T)
    c = s.fields()[2][0, 0]
    xp = np.arange(nx) + 0.5
    ser = np.ones(nx)
    for n in range(2000):
        k = (2 * n + 1) * math.pi / (2.0 * nx)
        ser -= 4.0 / ((2 * n + 1) * math.pi) * np.sin(k * xp) * np.exp(-D * k * k * T)
    assert np.abs(c - ser).max() < 2e-4
