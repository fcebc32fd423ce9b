"""Degenerate inputs through the C ABI against the FP64 oracle: no wet
boundary cells at all (an all-fluid periodic box: empty lists, zero
ledger), no fluid cells at all, periodic axes one cell wide (a cell is its
own neighbour), a single fluid cell enclosed by reactive solid (every link
reactive), a pure solute lattice next to the coupled one, and the
hand-evaluated dissolution events of the oracle's pins (an unpaid charge,
two simultaneous events sharing a payer)."""
import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import lbrbc

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()
    oracle.build()


def both(p, mask, steps, **init):
    g = lbrbc.Sim(p, mask, **init)
    o = oracle.OracleSim(p, mask, **init)
    g.step(steps)
    o.step(steps)
    g.check()
    assert np.array_equal(g.classes(), o.classes())
    for a, b in zip(g.fields(), o.fields()):
        assert np.abs(a - b).max() < TOL
    return g, o


BASE = dict(dim=3, flow_q=19, solute_q=7, tau_flow=0.8, magic_flow=3.0 / 16.0, tau_solute=0.9, k_r=0.1, c_eq=0.5,
            c_init=1.0, molar_volume=0.2, precision="fp64")


def test_all_fluid_box_has_empty_lists_and_zero_ledger():
    shape = (6, 7, 33)
    rng = np.random.default_rng(1)
    u0 = 0.02 * rng.standard_normal(shape + (3,))
    c0 = 1.0 + 0.1 * rng.standard_normal(shape)
    p = dict(BASE, nx=33, ny=7, nz=6, bc=("periodic",) * 3)
    g, o = both(p, np.zeros(shape, np.uint8), 21, u_init=u0, c_init=c0)
    assert g.info()["boundary_cells"] == 0
    L = g.ledger()
    assert L["reacted"] == 0.0 and L["dirichlet_in"] == 0.0
    assert abs(L["solute"] - c0.sum()) < 1e-10 * c0.sum()


def test_no_fluid_cells():
    shape = (5, 6, 7)
    p = dict(BASE, nx=7, ny=6, nz=5, bc=("periodic", "wall", "wall"))
    g, o = both(p, np.ones(shape, np.uint8), 6)
    assert g.info()["fluid_cells"] == 0 and g.info()["boundary_cells"] == 0
    assert g.ledger()["reacted"] == 0.0


@pytest.mark.parametrize("shape", [(1, 9, 40), (5, 1, 40), (5, 9, 1)])
def test_periodic_axes_one_cell_wide(shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(2)
    mask = (rng.uniform(size=shape) < 0.25).astype(np.uint8)
    mask.flat[0] = 0
    assert 0 < mask.sum() < mask.size
    c0 = 1.0 + 0.2 * rng.standard_normal(shape)
    p = dict(BASE, nx=nx, ny=ny, nz=nz, bc=("periodic",) * 3)
    g, o = both(p, mask, 17, c_init=c0)
    lg, lo = g.ledger(), o.ledger()
    assert abs(lg["reacted"] - lo["reacted"]) < 1e-9 * max(1.0, abs(lo["reacted"]))


@pytest.mark.parametrize("scheme", ["new", "patel_ju", "anti_bb"])
def test_single_fluid_cell_enclosed(scheme):
    shape = (5, 5, 5)
    mask = np.ones(shape, np.uint8)
    mask[2, 2, 2] = 0
    p = dict(BASE, nx=5, ny=5, nz=5, bc=("wall",) * 3, scheme=scheme)
    g, o = both(p, mask, 12)
    assert g.info()["fluid_cells"] == 1
    lg, lo = g.ledger(), o.ledger()
    for k in ("solute", "solid_over_vm", "reacted"):
        assert abs(lg[k] - lo[k]) < 1e-9 * max(1.0, abs(lo[k])), k


def test_pure_solute_lattice_with_walls():
    shape = (4, 11, 37)
    rng = np.random.default_rng(3)
    mask = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    p = dict(BASE, nx=37, ny=11, nz=4, flow_q=0, bc=("wall", "periodic", "wall"))
    both(p, mask, 15, c_init=1.0 + 0.1 * rng.standard_normal(shape))


def _events(x):
    # events of one step in a fixed order (the GPU logs a step's events in
    # the order of its atomics)
    return sorted(map(tuple, x.events().tolist()))


@pytest.mark.parametrize("case", ["unpaid", "shared_payer", "adjacent", "enclosed_precipitation", "mixed"])
def test_hand_evaluated_phase_change_events_match_oracle(case):
    # the phase-change configurations the oracle is pinned on by hand: an
    # isolated wet cell whose charge goes unpaid, two simultaneous
    # dissolutions two cells apart sharing a paying neighbour, two adjacent
    # simultaneous dissolutions, a precipitation left with no fluid
    # neighbour, and a dissolution and a precipitation in the same step
    Vm = 0.4
    c_init, c_eq, bc = 0.5, 1.0, ("periodic", "wall", "periodic")
    if case == "unpaid":
        nx = ny = 5
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 2, 2] = 1
        phi0 = np.where(mask == 1, 1e-12, 0.0)
        bc = ("periodic",) * 3
        n_ev = 1
    elif case == "mixed":
        nx, ny = 8, 6
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 0:2, :] = 1
        phi0 = np.where(mask == 1, 1.0, 0.0)
        phi0[0, 1, 1] = 1e-12
        phi0[0, 2, 5] = 1.0 - 1e-12
        c_eq = 0.5
        n_ev = 2
    elif case == "enclosed_precipitation":
        nx = ny = 5
        mask = np.ones((1, ny, nx), np.uint8)
        mask[0, 2, 2] = 0
        phi0 = np.where(mask == 1, 1.0, 1.0 - 1e-12)
        c_init, c_eq, bc = 1.0, 0.0, ("periodic",) * 3
        n_ev = 1
    else:
        nx, ny = (5, 6) if case == "shared_payer" else (6, 6)
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 0:2, :] = 1
        phi0 = np.where(mask == 1, 1.0, 0.0)
        cells = (1, 3) if case == "shared_payer" else (2, 3)
        phi0[0, 1, cells[0]] = phi0[0, 1, cells[1]] = 1e-12
        n_ev = 2
    init = dict(phi_init=phi0)
    if case == "mixed":
        c0 = np.zeros((1, ny, nx))
        c0[0, :, 4:] = 1.0
        init["c_init"] = c0
    elif case != "enclosed_precipitation":
        init["c_init"] = np.where(mask == 1, 0.0, 0.5)
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=bc, tau_solute=1.0, k_r=0.5, c_eq=c_eq, c_init=c_init,
             molar_volume=Vm, phase_change=1, precision="fp64", event_log_capacity=1024)
    g, o = both(p, mask, 3, **init)
    assert _events(g) == _events(o) and len(_events(o)) == n_ev
    lg, lo = g.ledger(), o.ledger()
    for k in ("solute", "solid_over_vm", "unpaid", "reacted"):
        assert lg[k] == pytest.approx(lo[k], rel=1e-12, abs=1e-13), k
    if case == "unpaid":
        assert lo["unpaid"] < 0.0


@pytest.mark.parametrize("case", ["corner_precipitations", "wall_precipitations", "dirichlet_neighbour",
                                  "inlet_face"])
def test_hand_evaluated_events_near_other_boundaries_match_oracle(case):
    # the further configurations the oracle is pinned on by hand: two
    # precipitations sharing a fluid neighbour (concave corner: 5 : 1 split
    # along the post-event normals; flat wall: nothing sideways), a
    # dissolution above a Dirichlet cell, and a dissolution on the inlet face
    Vm = 0.4
    p = dict(dim=2, flow_q=0, solute_q=5, tau_solute=1.0, k_r=0.5, molar_volume=Vm, phase_change=1,
             precision="fp64", event_log_capacity=1024)
    init = {}
    if case == "corner_precipitations":
        # (the open-fluid pair of the oracle pin starts at phi = 1, which the
        # C ABI rejects: on the GPU only cells next to reactive cells test the
        # threshold, so a fluid cell must reach phi >= 1 through its shares)
        nx = ny = 8
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 0:2, :] = 1
        mask[0, :, 0:2] = 1
        phi0 = np.where(mask == 1, 1.0, 0.0)
        phi0[0, 3, 2] = phi0[0, 2, 3] = 1.0 - 1e-12
        p.update(bc=("periodic",) * 3, c_eq=0.0, c_init=1.0)
    elif case == "wall_precipitations":
        nx, ny = 5, 6
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 0:2, :] = 1
        phi0 = np.where(mask == 1, 1.0, 0.0)
        phi0[0, 2, 1] = phi0[0, 2, 3] = 1.0 - 1e-12
        p.update(bc=("periodic", "wall", "periodic"), c_eq=0.0, c_init=1.0)
    elif case == "dirichlet_neighbour":
        nx, ny = 5, 6
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 0:2, :] = 1
        mask[0, 0, 2] = 2
        phi0 = np.where(mask == 1, 1.0, 0.0)
        phi0[0, 1, 2] = 1e-12
        init["c_init"] = np.where(mask == 0, 0.5, 0.0)
        p.update(bc=("periodic", "wall", "periodic"), c_eq=1.0, c_init=0.5, c_dirichlet=0.7)
    else:
        nx, ny = 6, 6
        mask = np.zeros((1, ny, nx), np.uint8)
        mask[0, 0:2, :] = 1
        phi0 = np.where(mask == 1, 1.0, 0.0)
        phi0[0, 1, 0] = 1e-12
        init["c_init"] = np.where(mask == 0, 0.5, 0.0)
        p.update(bc=("open", "wall", "periodic"), c_eq=1.0, c_init=0.5, c_inlet=0.9)
    p.update(nx=nx, ny=ny)
    g, o = both(p, mask, 6, phi_init=phi0, **init)
    assert _events(g) == _events(o) and len(_events(o)) >= 1
    lg, lo = g.ledger(), o.ledger()
    for k in ("solute", "solid_over_vm", "unpaid", "dirichlet_in", "reacted"):
        assert lg[k] == pytest.approx(lo[k], rel=1e-12, abs=1e-13), k


def test_fields_as_device_tensors():
    # the fields as float64 torch tensors on the simulation's GPU equal the
    # host copies bit for bit
    torch = pytest.importorskip("torch")
    shape = (6, 9, 21)
    rng = np.random.default_rng(4)
    mask = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    p = dict(BASE, nx=21, ny=9, nz=6, bc=("periodic",) * 3)
    g = lbrbc.Sim(p, mask)
    g.step(9)
    host = g.fields()
    dev = g.fields(device=True)
    for h, d in zip(host, dev):
        assert d.is_cuda and d.dtype == torch.float64 and tuple(d.shape) == h.shape
        assert np.array_equal(d.cpu().numpy(), h)
    # a mask given as a torch tensor on the GPU gives the same simulation
    g2 = lbrbc.Sim(p, torch.from_numpy(mask).cuda())
    g2.step(9)
    for a, b in zip(g2.fields(), host):
        assert np.array_equal(a, b)
    g2.close()
