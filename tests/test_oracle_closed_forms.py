"""The oracle against closed forms of steady reaction-diffusion toward a flat
wall (Eq. reactionRateBoundary, Eq. general_RBC) and against invariants.

A linear concentration profile is an exact steady state of the lattice; in
the wet-node reading of the reactive boundary condition the scheme with
gamma (Eq. k_i_S_New) reproduces the wall law k_r (C_wall - C_eq) = D dC/dn
exactly, the scheme without it (Eq. k_i_S_Ve) the law with k_r / gamma, and
the anti-bounce-back limit C_wall = C_eq (Sec. 3.1.1, Sec. 3.1.3)."""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_2306_10794_gb300 import workloads

CASES = [
    # (dim, solute_q, tau, magic, J0)
    (2, 9, 0.8, -1.0, -1.0),
    (2, 5, 0.8, -1.0, -1.0),
    (2, 5, 1.2, 3.0 / 16.0, 0.1),
    (3, 7, 0.9, -1.0, -1.0),
    (3, 7, 1.1, 0.25, 0.5),
]


def _cs2(q, dim, J0):
    return workloads.lattice_cs2(q, dim, J0)


@pytest.mark.parametrize("dim,q,tau,magic,J0", CASES)
@pytest.mark.parametrize("scheme", ["new", "verhaeghe", "anti_bb"])
def test_flat_wall_closed_form(dim, q, tau, magic, J0, scheme):
    ny = 32
    L = ny - 1.0
    D = _cs2(q, dim, J0) * (tau - 0.5)
    k_r = D / L  # PeDa = 1: the regime where gamma matters most
    gamma = tau / (tau - 0.5)
    k_eff = {"new": k_r, "verhaeghe": k_r / gamma, "anti_bb": math.inf}[scheme]
    if dim == 2:
        mask = workloads.reactive_wall_1d(2, ny)
    else:
        mask = workloads.reactive_wall_3d(2, ny, 2)
    y = np.arange(ny, dtype=np.float64)
    exact = analytic.wall_profile_1d(y, k_eff, D, L, 1.0, 0.25)
    c0 = np.broadcast_to(exact[None, :, None], mask.shape).copy()
    p = dict(dim=dim, nx=mask.shape[2], ny=ny, nz=mask.shape[0], flow_q=0, solute_q=q,
             bc=("periodic", "wall", "periodic"), tau_solute=tau, magic_solute=magic, rest_fraction=J0,
             k_r=k_r, c_eq=0.25, c_dirichlet=1.0, scheme=scheme)
    s = oracle.OracleSim(p, mask, c_init=c0)
    s.step(40000)
    c = s.fields()[2]
    err = np.abs(c - c0).max()
    assert err < 1e-9, err
    # the ledger books the diffusive flux -D dC/dy into the fluid per wall cell and step
    M = s.reacted()[:, 0, :]
    assert np.allclose(M, -D * (exact[1] - exact[0]), rtol=1e-7, atol=1e-14)


def test_flat_wall_discriminates_gamma():
    # S.New converged with k_r is *not* the S.V. profile (and vice versa)
    ny, tau = 32, 0.8
    D = (tau - 0.5) / 3.0
    k_r = D / (ny - 1)
    y = np.arange(ny, dtype=np.float64)
    new = analytic.wall_profile_1d(y, k_r, D, ny - 1.0, 1.0, 0.0)
    ve = analytic.wall_profile_1d(y, k_r / (tau / (tau - 0.5)), D, ny - 1.0, 1.0, 0.0)
    assert np.abs(new - ve).max() > 0.05


def test_zero_rate_is_inert():
    ny = 24
    mask = workloads.reactive_wall_1d(2, ny)
    p = dict(dim=2, nx=2, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.0, c_eq=0.0, c_dirichlet=1.0, c_init=0.3)
    s = oracle.OracleSim(p, mask)
    s.step(30000)
    c = s.fields()[2][0]
    assert np.abs(c - 1.0).max() < 1e-9


@pytest.mark.parametrize("phase_change", [0, 1])
def test_equilibrium_fixed_point(phase_change):
    # C = C_eq everywhere and a fluid at rest: nothing reacts, nothing moves
    mask = workloads.sphere_pack((12, 14, 16), 0.5, 2.0, 4.0, seed=3, periodic=(True, True, True))
    p = dict(dim=3, nx=16, ny=14, nz=12, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.9,
             magic_flow=3.0 / 16.0, tau_solute=0.8, k_r=0.05, c_eq=0.7, c_init=0.7, molar_volume=0.5,
             phase_change=phase_change)
    s = oracle.OracleSim(p, mask)
    s.step(60)
    u, rho, c, phi = s.fields()
    fl = mask == 0
    act = s.classes() != oracle.SOLID
    assert np.abs(c[act] - 0.7).max() < 1e-14
    assert np.abs(u).max() < 1e-16 and np.abs(rho[fl] - 1.0).max() < 1e-14
    assert np.abs(s.reacted()).max() < 1e-15
    assert len(s.events()) == 0



def test_zero_rate_cells_reduce_to_bounce_back_under_every_scheme():
    # Sec. 2.3: with k_r = 0 every scheme reduces to plain bounce-back, so the
    # four schemes must produce bit-identical runs (also where e.n vanishes,
    # which the S.P.J. coefficient would otherwise send to the anti-bounce-back
    # limit), the walls must not pull the solute towards C_eq, and the mass
    # invariant holds.
    mask = workloads.sphere_pack((10, 12, 14), 0.6, 2.0, 3.0, seed=4, periodic=(True, True, True))
    rng = np.random.default_rng(3)
    c0 = 1.0 + 0.2 * rng.standard_normal(mask.shape)
    runs = {}
    for scheme in ("new", "verhaeghe", "patel_ju", "anti_bb"):
        p = dict(dim=3, nx=14, ny=12, nz=10, flow_q=0, solute_q=7, bc=("periodic",) * 3, tau_solute=0.8,
                 k_r=0.3, c_eq=0.0, molar_volume=0.1, scheme=scheme)
        s = oracle.OracleSim(p, mask, k_field=np.zeros(mask.shape), c_init=c0)
        L0 = s.ledger()
        s.step(60)
        runs[scheme] = (s.fields()[2], s.ledger(), L0)
    c_ref, L_ref, L0 = runs["new"]
    for scheme, (c, L, _) in runs.items():
        assert np.array_equal(c, c_ref), scheme
        assert L["reacted"] == L_ref["reacted"], scheme
    inv = lambda L: L["solute"] + L["solid_over_vm"] + L["unpaid"] - L["dirichlet_in"]
    assert abs(inv(L_ref) - inv(L0)) < 1e-12 * abs(inv(L0))
    # no drain towards C_eq = 0: the solute changes only by the wet cells'
    # own adjustment, a small fraction of the total
    assert abs(L_ref["solute"] - L0["solute"]) < 0.01 * L0["solute"]
