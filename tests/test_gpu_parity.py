"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs, element by element.

Tolerances: the FP64 path must agree with the oracle to 1e-11 absolute on
O(1) fields (rounding only: deviation storage, fused multiply-add and a
different summation order); the FP32 path (deviation storage, FP32 collision)
to a relative L2 error <= 1e-5 on c and u, the accuracy target stated for
the FP32 path.  Grids are chosen to span several thread blocks with a ragged
tail (nx not a multiple of 128, odd sizes) and both step parities of the
in-place streaming."""
import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import lbrbc, workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


@pytest.fixture(params=["dense", "list"])
def sweep(request, monkeypatch):
    # the fluid sweep runs over the dense grid or the compacted fluid list
    monkeypatch.setenv("LBRBC_FLUID_SWEEP", request.param)
    return request.param


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()
    oracle.build()


def run_both(p, mask, steps, **init):
    g = lbrbc.Sim(p, mask, **init)
    o = oracle.OracleSim(p, mask, **init)
    g.step(steps)
    o.step(steps)
    return g, o


def compare64(g, o, fluid_only_u=True):
    ug, rg, cg, pg = g.fields()
    uo, ro, co, po = o.fields()
    assert np.array_equal(g.classes(), o.classes())
    errs = dict(u=np.abs(ug - uo).max(), rho=np.abs(rg - ro).max(), c=np.abs(cg - co).max(), phi=np.abs(pg - po).max())
    for k, v in errs.items():
        assert v < TOL64, (k, v, errs)
    return errs


def rel_l2(a, b):
    return np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300))


def pack(shape, seed, periodic=(True, True, True), por=0.55, r=(2.0, 4.0), buffer_x=0):
    return workloads.sphere_pack(shape, por, r[0], r[1], seed=seed, periodic=periodic, buffer_x=buffer_x)


@pytest.mark.parametrize("steps", [1, 2, 37])
@pytest.mark.parametrize("magic_f,magic_g", [(-1.0, -1.0), (3.0 / 16.0, 0.25)])
def test_sphere_pack_periodic_fp64(steps, magic_f, magic_g, sweep):
    shape = (13, 17, 139)
    mask = pack(shape, 1)
    rng = np.random.default_rng(2)
    u0 = np.zeros(shape + (3,))
    u0[..., 0] = 0.02
    u0[..., 1] = 0.01 * rng.standard_normal(shape)
    c0 = 1.0 + 0.3 * rng.standard_normal(shape)
    p = dict(dim=3, nx=139, ny=17, nz=13, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.7,
             magic_flow=magic_f, tau_solute=0.9, magic_solute=magic_g, rest_fraction=0.3, k_r=0.05, c_eq=0.8,
             c_init=1.0, molar_volume=0.1, precision="fp64")
    g, o = run_both(p, mask, steps, u_init=np.where(mask[..., None] == 0, u0, 0.0), c_init=c0)
    compare64(g, o)


@pytest.mark.parametrize("scheme", ["new", "verhaeghe", "patel_ju", "anti_bb"])
def test_schemes_walls_and_dirichlet_fp64(scheme, sweep):
    # non-periodic y/z walls, a Dirichlet slab and a reactive pack, k field
    shape = (11, 19, 45)
    mask = pack(shape, 3, periodic=(True, False, False), por=0.6)
    mask[:, -2:, :] = workloads.DIRICHLET
    kf = workloads.lognormal_k(shape, 0.05, 0.5, seed=4)
    p = dict(dim=3, nx=45, ny=19, nz=11, flow_q=19, solute_q=7, bc=("periodic", "wall", "wall"), tau_flow=0.9,
             tau_solute=0.75, k_r=0.05, c_eq=0.2, c_init=0.6, c_dirichlet=1.0, molar_volume=0.3, scheme=scheme,
             precision="fp64")
    g, o = run_both(p, mask, 25, k_field=kf)
    compare64(g, o)
    lg, lo = g.ledger(), o.ledger()
    for k in ("solute", "solid_over_vm", "dirichlet_in", "reacted"):
        assert abs(lg[k] - lo[k]) < 1e-9 * max(1.0, abs(lo[k])), (k, lg[k], lo[k])


def test_open_channel_fp64(sweep):
    p, mask, extra = workloads.case_channel(nx=70, ny=34, nz=30, theta_deg=30.0, h=10.0, Pe=10.0, Da=1.0)
    p["precision"] = "fp64"
    g, o = run_both(p, mask, 31, **extra)
    compare64(g, o)


@pytest.mark.parametrize("case", ["d2q9_solute", "d2q5_solute", "d2q9_d2q5_flow"])
def test_2d_fp64(case, sweep):
    if case == "d2q9_solute":
        p, mask, _ = workloads.case_wall_2d(nx=133, ny=40, tau=0.8, solute_q=9)
    elif case == "d2q5_solute":
        p, mask, _ = workloads.case_wall_2d(nx=133, ny=40, tau=1.1, solute_q=5)
        p.update(rest_fraction=0.2, magic_solute=3.0 / 16.0)
    else:
        mask = workloads.annulus(61, 9.0, 27.0, 0.3)[0]
        p = dict(dim=2, nx=61, ny=61, flow_q=9, solute_q=5, bc=("open", "wall", "periodic"), tau_flow=0.8,
                 magic_flow=3.0 / 16.0, tau_solute=0.8, k_r=0.01, c_eq=0.0, c_init=1.0, c_dirichlet=1.0,
                 c_inlet=1.0, u_inlet=0.01, rho_outlet=1.0)
    p["precision"] = "fp64"
    g, o = run_both(p, mask, 53)
    compare64(g, o)


def test_fp32_relative_l2(sweep):
    shape = (16, 20, 150)
    mask = pack(shape, 5)
    rng = np.random.default_rng(6)
    u0 = np.zeros(shape + (3,))
    u0[..., 0] = 0.03
    c0 = 1.0 + 0.2 * rng.standard_normal(shape)
    p = dict(dim=3, nx=150, ny=20, nz=16, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, rest_fraction=0.4, k_r=0.05, c_eq=1.0, c_init=1.0,
             molar_volume=0.1, precision="fp32")
    g, o = run_both(p, mask, 200, u_init=np.where(mask[..., None] == 0, u0, 0.0), c_init=c0)
    ug, _, cg, _ = g.fields()
    uo, _, co, _ = o.fields()
    assert rel_l2(cg, co) <= 1e-5, rel_l2(cg, co)
    assert rel_l2(ug, uo) <= 1e-5, rel_l2(ug, uo)


@pytest.mark.parametrize("c_init,phi_solid,kind", [(3.0, 1.0, 2), (0.0, 0.03, 1)])
def test_phase_change_events_identical_fp64(c_init, phi_solid, kind):
    # Events are threshold decisions on FP64 values that differ from the
    # oracle's by rounding only; identity holds unless a cell lands within
    # rounding of a threshold.
    shape = (14, 16, 36)
    mask = pack(shape, 7)
    rng = np.random.default_rng(8)
    phi0 = np.where(mask == 1, phi_solid * rng.uniform(0.5, 1.0, shape), 0.0)
    p = dict(dim=3, nx=36, ny=16, nz=14, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, k_r=0.2, c_eq=1.0, c_init=c_init, molar_volume=0.3,
             phase_change=1, precision="fp64", event_log_capacity=1 << 20)
    g, o = run_both(p, mask, 120, phi_init=phi0)
    eo, eg = o.events(), g.events()
    assert len(eo) > 0 and kind in set(eo[:, 2].tolist())
    key = lambda e: sorted(map(tuple, e.tolist()))
    assert key(eg) == key(eo)
    compare64(g, o)
    lg, lo = g.ledger(), o.ledger()
    inv = lambda L: L["solute"] + L["solid_over_vm"] + L["unpaid"] - L["dirichlet_in"]
    assert abs(inv(lg) - inv(lo)) < 1e-9 * abs(inv(lo))


def test_mass_invariant_gpu_fp64():
    shape = (12, 18, 40)
    mask = pack(shape, 9)
    p = dict(dim=3, nx=40, ny=18, nz=12, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.8,
             tau_solute=0.9, k_r=0.2, c_eq=1.0, c_init=2.5, molar_volume=0.3, phase_change=1, precision="fp64")
    g = lbrbc.Sim(p, mask)
    inv = lambda L: L["solute"] + L["solid_over_vm"] + L["unpaid"] - L["dirichlet_in"]
    I0 = inv(g.ledger())
    g.step(150)
    g.check()
    assert abs(inv(g.ledger()) - I0) < 1e-12 * abs(I0)


@pytest.mark.parametrize("scheme,angle", [("new", 0.0), ("patel_ju", 19.0)])
def test_phase_change_2d_grain_fp64(scheme, angle):
    # 2D precipitation on a star-shaped seed inside a circle of fixed
    # concentration (the setup of Sec. 3.2 at 61 x 61): identical events,
    # classes and fields, on aligned and turned seeds
    p, mask, _, _ = workloads.case_grain_2d(angle, scheme, n=61, k_r=0.02, molar_volume=0.5, precision="fp64")
    p["event_log_capacity"] = 1 << 16
    g, o = run_both(p, mask, 200)
    eo, eg = o.events(), g.events()
    assert len(eo) > 20 and set(eo[:, 2].tolist()) == {2}
    key = lambda e: sorted(map(tuple, e.tolist()))
    assert key(eg) == key(eo)
    compare64(g, o)
    lg, lo = g.ledger(), o.ledger()
    for k in ("solute", "solid_over_vm", "dirichlet_in", "reacted"):
        assert abs(lg[k] - lo[k]) < 1e-9 * max(1.0, abs(lo[k])), (k, lg[k], lo[k])
