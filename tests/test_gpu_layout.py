"""The two population layouts of the library (dense padded grid and active
cells with a neighbour table) run the same arithmetic in the same order, so
their fields, ledgers and phase-change events must agree bit for bit; the
active-cell layout must also match the FP64 oracle where dissolution grows
the pore space beyond the stored margin and the layout is repacked on the
device in the middle of a step."""
import os

import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import lbrbc, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()
    oracle.build()


def run(p, mask, steps, layout, **init):
    s = lbrbc.Sim(dict(p, layout=layout, event_log_capacity=1 << 20), mask, **init)
    assert s.layout_info()["layout"] == layout
    s.step(steps)
    s.check()
    out = dict(fields=s.fields(), ledger=s.ledger(), events=s.events(), classes=s.classes(),
               info=s.layout_info())
    s.close()
    return out


def by_step(ev):
    # the log order within a step follows the atomics of the event queue:
    # compare the events of each step as a set
    return ev[np.lexsort((ev[:, 2], ev[:, 1], ev[:, 0]))] if len(ev) else ev


def same(a, b):
    for x, y in zip(a["fields"], b["fields"]):
        assert np.array_equal(x, y)
    assert np.array_equal(a["classes"], b["classes"])
    assert np.array_equal(by_step(a["events"]), by_step(b["events"]))
    for k in ("solute", "solid_over_vm", "unpaid", "dirichlet_in", "reacted"):
        assert a["ledger"][k] == b["ledger"][k], k


def pack_case(precision, c_init, c_eq, phi_solid, shape=(20, 22, 40), seed=3):
    nz, ny, nx = shape
    mask = workloads.sphere_pack(shape, 0.5, 2.0, 4.0, seed=seed, periodic=(False, True, True), buffer_x=3)
    rng = np.random.default_rng(seed)
    phi0 = np.where(mask == 1, phi_solid * rng.uniform(0.5, 1.0, shape), 0.0)
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"), tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, rest_fraction=0.4, k_r=0.3, c_eq=c_eq, c_init=c_init,
             c_inlet=c_init, u_inlet=0.01, rho_outlet=1.0, molar_volume=0.3, phase_change=1, precision=precision)
    return p, mask, dict(phi_init=phi0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["precipitation", "dissolution"])
def test_layouts_bitwise_equal_through_phase_changes(precision, kind):
    if kind == "precipitation":
        p, mask, init = pack_case(precision, 3.0, 1.0, 1.0)
    else:
        p, mask, init = pack_case(precision, 0.0, 1.0, 0.05)
    steps = 61  # an odd count: the run ends in the odd-step storage form
    d = run(p, mask, steps, "dense", **init)
    s = run(p, mask, steps, "sparse", **init)
    assert len(d["events"]) > 0
    same(d, s)
    if kind == "precipitation":  # (dissolution here ends with every cell stored)
        assert s["info"]["stored_cells"] < mask.size


@pytest.mark.parametrize("case", ["channel", "grain2d", "periodic_box", "no_flow_walls"])
def test_layouts_bitwise_equal_other_geometries(case):
    if case == "channel":
        p, mask, init = workloads.case_channel(nx=48, ny=30, nz=30, h=9.0, theta_deg=30.0)
        p = dict(p, precision="fp32")
    elif case == "grain2d":
        p, mask, init, _ = workloads.case_grain_2d(0.0, "new", n=60, k_r=0.05, molar_volume=4.0)
        p = dict(p, precision="fp64")
    elif case == "periodic_box":
        shape = (9, 10, 33)
        mask = workloads.sphere_pack(shape, 0.6, 1.5, 3.0, seed=4, periodic=(True, True, True))
        p = dict(dim=3, nx=33, ny=10, nz=9, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.7,
                 tau_solute=0.8, k_r=0.1, c_eq=0.5, c_init=1.0, precision="fp64")
        init = {}
    else:
        shape = (6, 15, 23)
        rng = np.random.default_rng(7)
        mask = (rng.uniform(size=shape) < 0.35).astype(np.uint8)
        p = dict(dim=3, nx=23, ny=15, nz=6, flow_q=0, solute_q=7, bc=("wall", "periodic", "wall"), tau_solute=0.8,
                 k_r=0.2, c_eq=0.5, c_init=1.0, precision="fp32")
        init = dict(c_init=1.0 + 0.1 * rng.standard_normal(shape))
    d = run(p, mask, 37, "dense", **init)
    s = run(p, mask, 37, "sparse", **init)
    same(d, s)


def run_lists(p, mask, steps, layout, local, ev_max=None, **init):
    env = {"LBRBC_LOCAL_LISTS": "1" if local else "0"}
    if ev_max is not None:
        env["LBRBC_LOCAL_EV_MAX"] = str(ev_max)
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return run(p, mask, steps, layout, **init)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


@pytest.mark.parametrize("layout", ["dense", "sparse"])
@pytest.mark.parametrize("kind", ["precipitation", "dissolution"])
def test_local_list_maintenance_matches_full_rebuild(layout, kind):
    # After events the classes and lists are updated in the cubes around the
    # events (entries recomputed in place, dead entries skipped, new ones
    # appended in cell order) instead of over the whole grid: every field,
    # class and event must be the same bit for bit; the ledger sums the same
    # terms in another list order.
    if kind == "precipitation":
        p, mask, init = pack_case("fp64", 3.0, 1.0, 1.0)
    else:
        p, mask, init = pack_case("fp64", 0.0, 1.0, 0.05)
    steps = 61
    full = run_lists(p, mask, steps, layout, False, **init)
    loc = run_lists(p, mask, steps, layout, True, **init)
    assert len(full["events"]) > 20
    for x, y in zip(full["fields"], loc["fields"]):
        assert np.array_equal(x, y)
    assert np.array_equal(full["classes"], loc["classes"])
    assert np.array_equal(by_step(full["events"]), by_step(loc["events"]))
    for k in ("solute", "solid_over_vm", "unpaid", "dirichlet_in", "reacted"):
        assert loc["ledger"][k] == pytest.approx(full["ledger"][k], rel=1e-13, abs=1e-15), k


@pytest.mark.parametrize("layout", ["dense", "sparse"])
def test_local_and_whole_grid_steps_mixed_match_full_rebuild(layout):
    # with the local limit lowered to 40 events, steps with few events are
    # updated locally and steps with more over the whole grid, in one run;
    # the dead entries and appends of the local steps meet full compactions
    p, mask, init = pack_case("fp64", 3.0, 1.0, 1.0)
    steps = 61
    full = run_lists(p, mask, steps, layout, False, **init)
    mixed = run_lists(p, mask, steps, layout, True, ev_max=40, **init)
    per_step = np.bincount(full["events"][:, 0].astype(np.int64))
    per_step = per_step[per_step > 0]
    assert (per_step <= 40).any() and (per_step > 40).any()
    for x, y in zip(full["fields"], mixed["fields"]):
        assert np.array_equal(x, y)
    assert np.array_equal(full["classes"], mixed["classes"])
    assert np.array_equal(by_step(full["events"]), by_step(mixed["events"]))
    for k in ("solute", "solid_over_vm", "unpaid", "dirichlet_in", "reacted"):
        assert mixed["ledger"][k] == pytest.approx(full["ledger"][k], rel=1e-13, abs=1e-15), k


@pytest.mark.parametrize("c_init", [1.6, 0.4])
def test_local_list_maintenance_matches_full_rebuild_larger_pack(c_init):
    # a 48^3 pack, supersaturated (precipitation) or undersaturated with the
    # solid fraction of the grains near 0 (dissolution): many events per step
    shape = (48, 48, 48)
    mask = workloads.sphere_pack(shape, 0.5, 3.0, 6.0, seed=9, periodic=(False, True, True), buffer_x=3)
    rng = np.random.default_rng(9)
    phi0 = np.where(mask == 1, rng.uniform(0.0005, 0.05, shape), 0.0)
    p = dict(dim=3, nx=48, ny=48, nz=48, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"), tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, rest_fraction=0.4, k_r=0.3, c_eq=1.0, c_init=c_init,
             c_inlet=c_init, u_inlet=0.01, rho_outlet=1.0, molar_volume=2.0, phase_change=1, precision="fp32")
    full = run_lists(p, mask, 41, "sparse", False, phi_init=phi0)
    loc = run_lists(p, mask, 41, "sparse", True, phi_init=phi0)
    assert len(full["events"]) > 200, len(full["events"])
    for x, y in zip(full["fields"], loc["fields"]):
        assert np.array_equal(x, y)
    assert np.array_equal(full["classes"], loc["classes"])
    assert np.array_equal(by_step(full["events"]), by_step(loc["events"]))


def test_repacking_matches_oracle():
    # a thin, nearly dissolved solid layer between two fluid regions with a
    # solute-free inlet: dissolution fronts run through several cells, so
    # cells outside the stored margin gain fluid neighbours and the layout
    # is repacked on the device
    nz, ny, nx = 6, 16, 26
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, 4:12, 6:20] = 1
    rng = np.random.default_rng(11)
    phi0 = np.where(mask == 1, rng.uniform(0.002, 0.02, mask.shape), 0.0)
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"), tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, rest_fraction=0.4, k_r=0.5, c_eq=1.0, c_init=0.0, c_inlet=0.0,
             u_inlet=0.01, rho_outlet=1.0, molar_volume=0.3, phase_change=1, precision="fp64")
    g = lbrbc.Sim(dict(p, layout="sparse", event_log_capacity=1 << 16), mask, phi_init=phi0)
    o = oracle.OracleSim(p, mask, phi_init=phi0)
    for chunk in (7, 12, 20):
        g.step(chunk)
        o.step(chunk)
        g.check()
        assert np.array_equal(g.classes(), o.classes())
        for a, b in zip(g.fields(), o.fields()):
            assert np.abs(a - b).max() < 1e-11
        assert by_step(g.events()).tolist() == by_step(o.events()).tolist()
    assert g.layout_info()["repacks"] > 0
    lg, lo = g.ledger(), o.ledger()
    for k in ("solute", "solid_over_vm", "unpaid", "reacted"):
        assert lg[k] == pytest.approx(lo[k], rel=1e-12, abs=1e-13), k
    g.close()


def test_auto_layout_choice():
    mask = workloads.sphere_pack((24, 24, 24), 0.4, 3.0, 5.0, seed=5, periodic=(False, True, True), buffer_x=2)
    p = dict(dim=3, nx=24, ny=24, nz=24, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"), tau_flow=0.8,
             tau_solute=0.9, u_inlet=0.01, c_inlet=1.0, precision="fp32", layout="auto")
    s = lbrbc.Sim(p, mask)
    assert s.layout_info()["layout"] == "sparse"
    s.close()
    p2, m2, i2 = workloads.case_channel(nx=64, ny=32, nz=32, h=10.0, theta_deg=0.0)
    s = lbrbc.Sim(dict(p2, layout="auto"), m2, **i2)
    assert s.layout_info()["layout"] == "dense"
    s.close()
