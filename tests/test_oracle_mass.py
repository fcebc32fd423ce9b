"""Mass conservation of the oracle: solute plus precipitated solid
(sum C + sum phi / V_m, Eq. solidFractionUpdate with the conserving sign),
closed by the Dirichlet-cell and unpaid terms, through phase changes
(Sec. 2.4).  The phase-change redistribution rules themselves are not fixed
by the paper (parity unpinned beyond this invariant and the event checks)."""
import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import workloads


def _invariant(L):
    return L["solute"] + L["solid_over_vm"] + L["unpaid"] - L["dirichlet_in"] - L["open_in"]


@pytest.mark.parametrize("c_init,c_eq,phi_solid,label", [
    (3.0, 1.0, 1.0, "precipitation"),
    (0.0, 1.0, 0.02, "dissolution"),
])
def test_closed_box_with_phase_change(c_init, c_eq, phi_solid, label):
    shape = (14, 16, 18)
    mask = workloads.sphere_pack(shape, 0.55, 2.0, 3.5, seed=7, periodic=(True, True, True))
    rng = np.random.default_rng(5)
    phi0 = np.where(mask == 1, phi_solid * rng.uniform(0.5, 1.0, shape), 0.0)
    p = dict(dim=3, nx=18, ny=16, nz=14, flow_q=19, solute_q=7, bc=("periodic",) * 3, tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, k_r=0.2, c_eq=c_eq, c_init=c_init, molar_volume=0.3,
             phase_change=1)
    s = oracle.OracleSim(p, mask, phi_init=phi0)
    I0 = _invariant(s.ledger())
    s.step(150)
    I1 = _invariant(s.ledger())
    ev = s.events()
    kinds = set(ev[:, 2].tolist())
    want = oracle.EV_PRECIPITATE if label == "precipitation" else oracle.EV_DISSOLVE
    assert want in kinds, "the case must exercise %s events" % label
    assert abs(I1 - I0) <= 1e-12 * abs(I0)
    # every cell class is consistent with the new geometry
    cls = s.classes()
    assert set(np.unique(cls)) <= {0, 1, 2}


def test_dirichlet_ledger_closes_balance():
    mask = workloads.reactive_wall_1d(6, 20)
    p = dict(dim=2, nx=6, ny=20, flow_q=0, solute_q=9, bc=("periodic", "wall", "periodic"), tau_solute=0.9,
             k_r=0.01, c_eq=0.0, c_dirichlet=1.0, c_init=0.2)
    s = oracle.OracleSim(p, mask)
    I0 = _invariant(s.ledger())
    s.step(500)
    L = s.ledger()
    assert L["dirichlet_in"] > 0.0 and L["reacted"] < 0.0
    assert abs(_invariant(L) - I0) < 1e-12 * abs(I0)


def test_single_dissolution_event_by_hand():
    """A boundary cell whose phi goes to <= 0 turns fluid with the mean
    concentration of its fluid neighbours; its solid neighbours pay
    V_m (C_init - C_b) - phi_b in equal shares (Sec. 2.4).  Expected values
    are taken from a run without phase change, evaluated by hand."""
    nx, ny, Vm = 5, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1  # two solid rows; row 1 is the wet boundary row
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 1, 2] = 1e-12  # this cell dissolves in the first step
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=1.0, c_init=0.0, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0)
    s.step(1)
    ev = s.events()
    assert ev.tolist() == [[0, 2 + nx * 1, oracle.EV_DISSOLVE]]
    cls = s.classes()[0]
    assert cls[1, 2] == oracle.FLUID and cls[0, 2] == oracle.BOUND
    _, _, c, phi = s.fields()
    c_init = c_ref[0, 2, 2]  # the only fluid neighbour of (x=2, y=1)
    assert c[0, 1, 2] == pytest.approx(c_init, rel=1e-14)
    assert phi[0, 1, 2] == 0.0
    Q = Vm * (c_init - c_ref[0, 1, 2]) - phi_ref[0, 1, 2]
    paid = phi_ref[0, [1, 1, 0], [1, 3, 2]] - phi[0, [1, 1, 0], [1, 3, 2]]
    assert np.allclose(paid, Q / 3.0, rtol=1e-12)


def test_single_precipitation_event_by_hand():
    """A fluid cell whose phi reaches >= 1 turns solid (Sec. 2.4, reading
    R5): phi += V_m C, its solute is removed, phi := 1, and the excess goes
    to its fluid neighbours as concentration, weighted by the new link
    coefficients (e_o.n)+.  Here the new cell is a bump on a flat wall: the
    isotropic gradient of the solid indicator at the bump, evaluated by hand
    with the D2Q9 weights, is 3 * (w_axis (0,-1) + w_diag ((1,-1) + (-1,-1)))
    = (0, -1/2), so n = (0, 1): the upward link has kappa = 1 and the two
    sideways links kappa = 0, and the whole excess goes up.  The wall cell
    below the bump loses its last fluid neighbour (D2Q5) and turns its
    solute into phi.  Expected values are taken from a run without phase
    change."""
    nx, ny, Vm = 5, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 2, 2] = 1.0 - 1e-12  # this fluid cell precipitates in the first step
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=0.0, c_init=1.0, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0)
    s.step(1)
    assert s.events().tolist() == [[0, 2 + nx * 2, oracle.EV_PRECIPITATE]]
    cls = s.classes()[0]
    assert cls[2, 2] == oracle.BOUND and cls[1, 2] == oracle.SOLID
    assert cls[1, 1] == oracle.BOUND and cls[1, 3] == oracle.BOUND
    _, _, c, phi = s.fields()
    excess = phi_ref[0, 2, 2] + Vm * c_ref[0, 2, 2] - 1.0
    assert excess > 0.0
    assert phi[0, 2, 2] == 1.0 and c[0, 2, 2] == 0.0
    assert c[0, 3, 2] == pytest.approx(c_ref[0, 3, 2] + excess / Vm, rel=1e-14)
    assert c[0, 2, 1] == pytest.approx(c_ref[0, 2, 1], rel=1e-14)
    assert c[0, 2, 3] == pytest.approx(c_ref[0, 2, 3], rel=1e-14)
    assert phi[0, 1, 2] == pytest.approx(phi_ref[0, 1, 2] + Vm * c_ref[0, 1, 2], rel=1e-14)


def test_dissolution_without_solid_neighbours_is_unpaid_by_hand():
    """An isolated wet cell that dissolves has no solid neighbour left to pay
    its charge V_m (C_init - C_b) - phi_b (Sec. 2.4, reading R5): the charge
    goes to the unpaid ledger term as -charge / V_m, and the new fluid cell
    takes the mean concentration of its four fluid neighbours.  Expected
    values are taken from a run without phase change, evaluated by hand."""
    n, Vm = 5, 0.4
    mask = np.zeros((1, n, n), np.uint8)
    mask[0, 2, 2] = 1
    phi0 = np.where(mask == 1, 1e-12, 0.0)
    p = dict(dim=2, nx=n, ny=n, flow_q=0, solute_q=5, bc=("periodic", "periodic", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=1.0, c_init=0.5, molar_volume=Vm)
    c0 = np.where(mask == 1, 0.0, 0.5)  # a solute-free wet cell: its charge is not zero
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0, c_init=c0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0, c_init=c0)
    L0 = s.ledger()
    s.step(1)
    assert s.events().tolist() == [[0, 2 + n * 2, oracle.EV_DISSOLVE]]
    assert (s.classes()[0] == oracle.FLUID).all()
    _, _, c, phi = s.fields()
    c_init = np.mean([c_ref[0, 1, 2], c_ref[0, 3, 2], c_ref[0, 2, 1], c_ref[0, 2, 3]])
    assert c[0, 2, 2] == pytest.approx(c_init, rel=1e-14)
    assert (phi == 0.0).all()
    Q = Vm * (c_init - c_ref[0, 2, 2]) - phi_ref[0, 2, 2]
    assert Q > 0.0
    L = s.ledger()
    assert L["unpaid"] == pytest.approx(-Q / Vm, rel=1e-12)
    assert _invariant(L) == pytest.approx(_invariant(L0), rel=1e-13, abs=1e-13)


def test_simultaneous_dissolutions_share_a_payer_by_hand():
    """Two wet cells two apart on a wall dissolve in the same step.  Events
    of a step act together on the pre-event state (reading R5): each charge
    is split equally over its own post-event solid neighbours (including the
    formerly interior cell below it), and the solid cell between the two
    pays a third of each charge.  Expected values are taken from a run
    without phase change, evaluated by hand."""
    nx, ny, Vm = 5, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1  # two solid rows; row 1 is the wet boundary row
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 1, 1] = phi0[0, 1, 3] = 1e-12
    c0 = np.where(mask == 1, 0.0, 0.5)  # solute-free wall cells: the charges are not zero
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=1.0, c_init=0.5, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0, c_init=c0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0, c_init=c0)
    s.step(1)
    assert s.events().tolist() == [[0, 1 + nx, oracle.EV_DISSOLVE], [0, 3 + nx, oracle.EV_DISSOLVE]]
    cls = s.classes()[0]
    assert cls[1, 1] == oracle.FLUID and cls[1, 3] == oracle.FLUID
    assert cls[0, 1] == oracle.BOUND and cls[0, 3] == oracle.BOUND and cls[1, 2] == oracle.BOUND
    _, _, c, phi = s.fields()
    # the only fluid neighbour of each event cell before the events is the cell above it
    assert c[0, 1, 1] == pytest.approx(c_ref[0, 2, 1], rel=1e-14)
    assert c[0, 1, 3] == pytest.approx(c_ref[0, 2, 3], rel=1e-14)
    Q1 = Vm * (c_ref[0, 2, 1] - c_ref[0, 1, 1]) - phi_ref[0, 1, 1]
    Q3 = Vm * (c_ref[0, 2, 3] - c_ref[0, 1, 3]) - phi_ref[0, 1, 3]
    assert Q1 > 0.0 and Q3 > 0.0
    expected = {(1, 0): Q1 / 3, (0, 1): Q1 / 3, (1, 2): Q1 / 3 + Q3 / 3, (1, 4): Q3 / 3, (0, 3): Q3 / 3}
    for (y, x), q in expected.items():
        assert phi_ref[0, y, x] - phi[0, y, x] == pytest.approx(q, rel=1e-12), (y, x)
    # solid cells neither event touches pay nothing
    for (y, x) in ((0, 0), (0, 2), (0, 4)):
        assert phi[0, y, x] == phi_ref[0, y, x]
    assert phi[0, 1, 1] == 0.0 and phi[0, 1, 3] == 0.0


def test_adjacent_simultaneous_dissolutions_by_hand():
    """Two neighbouring wet cells dissolve in the same step (reading R5:
    events act together on the pre-event state).  Neither counts the other
    as a fluid neighbour when it takes its concentration, and neither pays
    the other's charge (both are fluid after the events): each charge is
    split over the other two solid neighbours only."""
    nx, ny, Vm = 6, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 1, 2] = phi0[0, 1, 3] = 1e-12
    c0 = np.where(mask == 1, 0.0, 0.5)
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=1.0, c_init=0.5, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0, c_init=c0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0, c_init=c0)
    s.step(1)
    assert s.events().tolist() == [[0, 2 + nx, oracle.EV_DISSOLVE], [0, 3 + nx, oracle.EV_DISSOLVE]]
    _, _, c, phi = s.fields()
    assert c[0, 1, 2] == pytest.approx(c_ref[0, 2, 2], rel=1e-14)
    assert c[0, 1, 3] == pytest.approx(c_ref[0, 2, 3], rel=1e-14)
    Q2 = Vm * (c_ref[0, 2, 2] - c_ref[0, 1, 2]) - phi_ref[0, 1, 2]
    Q3 = Vm * (c_ref[0, 2, 3] - c_ref[0, 1, 3]) - phi_ref[0, 1, 3]
    expected = {(1, 1): Q2 / 2, (0, 2): Q2 / 2, (1, 4): Q3 / 2, (0, 3): Q3 / 2}
    for (y, x), q in expected.items():
        assert phi_ref[0, y, x] - phi[0, y, x] == pytest.approx(q, rel=1e-12), (y, x)
    assert phi[0, 1, 2] == 0.0 and phi[0, 1, 3] == 0.0


def test_precipitation_without_fluid_neighbours_by_hand():
    """A fluid cell enclosed by reactive solid precipitates (reading R5): with
    no fluid neighbour after the event there is nowhere to send the excess,
    so the cell keeps phi + V_m C (above 1) and its solute is removed; the
    balance sum C + sum phi / V_m is unchanged by the event."""
    n, Vm = 5, 0.4
    mask = np.ones((1, n, n), np.uint8)
    mask[0, 2, 2] = 0
    phi0 = np.where(mask == 1, 1.0, 1.0 - 1e-12)
    p = dict(dim=2, nx=n, ny=n, flow_q=0, solute_q=5, bc=("periodic", "periodic", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=0.0, c_init=1.0, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    L_ref = ref.ledger()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0)
    s.step(1)
    assert s.events().tolist() == [[0, 2 + n * 2, oracle.EV_PRECIPITATE]]
    assert (s.classes()[0] == oracle.SOLID).all()
    _, _, c, phi = s.fields()
    assert phi[0, 2, 2] == pytest.approx(phi_ref[0, 2, 2] + Vm * c_ref[0, 2, 2], rel=1e-14)
    assert phi[0, 2, 2] > 1.0 and c[0, 2, 2] == 0.0
    L = s.ledger()
    assert _invariant(L) == pytest.approx(_invariant(L_ref), rel=1e-13)


def test_dissolution_and_precipitation_in_one_step_by_hand():
    """A wall under a solute-free column dissolves at one cell while a bump
    grows on it under a supersaturated column, in the same step (reading R5:
    every event of a step follows its own rule on the pre-event state).  The
    dissolving cell takes the concentration of the cell above it and charges
    its three solid neighbours; the precipitating cell keeps phi := 1 and
    sends its whole excess up (the flat-wall normal, as in
    test_single_precipitation_event_by_hand), and the wall cell under it,
    left without a fluid neighbour, turns its solute into phi."""
    nx, ny, Vm = 8, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 1, 1] = 1e-12        # dissolves
    phi0[0, 2, 5] = 1.0 - 1e-12  # precipitates
    c0 = np.zeros((1, ny, nx))
    c0[0, :, 4:] = 1.0           # supersaturated columns x >= 4, solute-free columns x < 4 (c_eq = 0.5)
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=0.5, c_init=0.5, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0, c_init=c0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0, c_init=c0)
    L0 = s.ledger()
    s.step(1)
    assert s.events().tolist() == [[0, 1 + nx, oracle.EV_DISSOLVE], [0, 5 + 2 * nx, oracle.EV_PRECIPITATE]]
    _, _, c, phi = s.fields()
    # dissolution
    assert c[0, 1, 1] == pytest.approx(c_ref[0, 2, 1], rel=1e-14)
    Q = Vm * (c_ref[0, 2, 1] - c_ref[0, 1, 1]) - phi_ref[0, 1, 1]
    for (y, x) in ((1, 0), (1, 2), (0, 1)):
        assert phi_ref[0, y, x] - phi[0, y, x] == pytest.approx(Q / 3, rel=1e-12), (y, x)
    assert phi[0, 1, 1] == 0.0
    # precipitation
    excess = phi_ref[0, 2, 5] + Vm * c_ref[0, 2, 5] - 1.0
    assert excess > 0.0
    assert phi[0, 2, 5] == 1.0 and c[0, 2, 5] == 0.0
    assert c[0, 3, 5] == pytest.approx(c_ref[0, 3, 5] + excess / Vm, rel=1e-14)
    assert c[0, 2, 4] == pytest.approx(c_ref[0, 2, 4], rel=1e-14)
    assert c[0, 2, 6] == pytest.approx(c_ref[0, 2, 6], rel=1e-14)
    assert phi[0, 1, 5] == pytest.approx(phi_ref[0, 1, 5] + Vm * c_ref[0, 1, 5], rel=1e-14)
    assert _invariant(s.ledger()) == pytest.approx(_invariant(L0), rel=1e-13)


def test_simultaneous_precipitations_share_a_fluid_neighbour_by_hand():
    """Two fluid cells two apart reach phi = 1 in the same step (reading R5).
    In open fluid the solid indicator around each new solid cell is zero, so
    its normal is undefined, every link counts as aligned, and its excess
    V_m C goes to its four fluid neighbours in equal shares; the cell between
    the two receives a share from each.  On a flat wall the same pair sends
    its whole excess up along the wall normal and the cell between them
    receives nothing.  Expected values are taken from a run without phase
    change, evaluated by hand."""
    n, Vm = 7, 0.4
    mask = np.zeros((1, 5, n), np.uint8)
    phi0 = np.zeros((1, 5, n))
    phi0[0, 2, 2] = phi0[0, 2, 4] = 1.0
    p = dict(dim=2, nx=n, ny=5, flow_q=0, solute_q=5, bc=("periodic",) * 3, tau_solute=1.0, k_r=0.5, c_eq=0.0,
             c_init=0.8, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0)
    L0 = s.ledger()
    s.step(1)
    assert s.events().tolist() == [[0, 2 + 2 * n, oracle.EV_PRECIPITATE], [0, 4 + 2 * n, oracle.EV_PRECIPITATE]]
    _, _, c, phi = s.fields()
    share = {x: (phi_ref[0, 2, x] + Vm * c_ref[0, 2, x] - 1.0) / Vm / 4.0 for x in (2, 4)}
    assert share[2] > 0.0 and share[4] > 0.0
    assert c[0, 2, 3] == pytest.approx(c_ref[0, 2, 3] + share[2] + share[4], rel=1e-14)
    for (y, x), src in {(2, 1): 2, (1, 2): 2, (3, 2): 2, (2, 5): 4, (1, 4): 4, (3, 4): 4}.items():
        assert c[0, y, x] == pytest.approx(c_ref[0, y, x] + share[src], rel=1e-14), (y, x)
    for x in (2, 4):
        assert phi[0, 2, x] == 1.0 and c[0, 2, x] == 0.0
    assert _invariant(s.ledger()) == pytest.approx(_invariant(L0), rel=1e-13)

    # the same pair as bumps on a flat wall
    nx, ny = 5, 6
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 2, 1] = phi0[0, 2, 3] = 1.0 - 1e-12
    p = dict(p, nx=nx, ny=ny, bc=("periodic", "wall", "periodic"), c_init=1.0)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0)
    s.step(1)
    assert len(s.events()) == 2
    _, _, c, phi = s.fields()
    assert c[0, 2, 2] == pytest.approx(c_ref[0, 2, 2], rel=1e-14)
    for x in (1, 3):
        excess = phi_ref[0, 2, x] + Vm * c_ref[0, 2, x] - 1.0
        assert c[0, 3, x] == pytest.approx(c_ref[0, 3, x] + excess / Vm, rel=1e-14)


def test_dissolution_next_to_a_dirichlet_cell_by_hand():
    """A wet cell above a Dirichlet cell dissolves (reading R5): only the
    reactive solid neighbours pay its charge (here two, half each); the
    Dirichlet cell, which gains a fluid neighbour, becomes a boundary cell
    holding C = 0 and pays nothing.  The balance, which books what Dirichlet
    cells inject, is unchanged through the event and after it."""
    nx, ny, Vm = 5, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1
    mask[0, 0, 2] = 2  # Dirichlet cell under the dissolving one
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 1, 2] = 1e-12
    c0 = np.where(mask == 0, 0.5, 0.0)
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("periodic", "wall", "periodic"), tau_solute=1.0,
             k_r=0.5, c_eq=1.0, c_init=0.5, c_dirichlet=0.7, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0, c_init=c0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0, c_init=c0)
    L0 = s.ledger()
    s.step(1)
    assert s.events().tolist() == [[0, 2 + nx, oracle.EV_DISSOLVE]]
    cls = s.classes()[0]
    assert cls[1, 2] == oracle.FLUID and cls[0, 2] == oracle.BOUND
    _, _, c, phi = s.fields()
    assert c[0, 1, 2] == pytest.approx(c_ref[0, 2, 2], rel=1e-14)
    assert c[0, 0, 2] == 0.0 and phi[0, 0, 2] == phi_ref[0, 0, 2]
    Q = Vm * (c_ref[0, 2, 2] - c_ref[0, 1, 2]) - phi_ref[0, 1, 2]
    assert Q > 0.0
    for x in (1, 3):
        assert phi_ref[0, 1, x] - phi[0, 1, x] == pytest.approx(Q / 2, rel=1e-12), x
    assert _invariant(s.ledger()) == pytest.approx(_invariant(L0), rel=1e-13)
    s.step(5)
    assert s.ledger()["dirichlet_in"] != L0["dirichlet_in"]
    assert _invariant(s.ledger()) == pytest.approx(_invariant(L0), rel=1e-13)


def test_dissolution_at_the_inlet_face_by_hand():
    """A wet cell on the inlet face x = 0 dissolves (reading R5 with the open
    boundary of reading R9): the inlet is not a cell, so the new fluid cell
    takes the concentration of its one fluid neighbour and its charge is
    split over its two reactive solid neighbours; from the next step on its
    inlet link injects solute, booked in the open-boundary term."""
    nx, ny, Vm = 6, 6, 0.4
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0:2, :] = 1
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 1, 0] = 1e-12
    c0 = np.where(mask == 0, 0.5, 0.0)
    p = dict(dim=2, nx=nx, ny=ny, flow_q=0, solute_q=5, bc=("open", "wall", "periodic"), tau_solute=1.0, k_r=0.5,
             c_eq=1.0, c_init=0.5, c_inlet=0.9, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0, c_init=c0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0, c_init=c0)
    L0 = s.ledger()
    s.step(1)
    assert s.events().tolist() == [[0, nx, oracle.EV_DISSOLVE]]
    _, _, c, phi = s.fields()
    assert s.classes()[0, 1, 0] == oracle.FLUID
    assert c[0, 1, 0] == pytest.approx(c_ref[0, 2, 0], rel=1e-14)
    Q = Vm * (c_ref[0, 2, 0] - c_ref[0, 1, 0]) - phi_ref[0, 1, 0]
    for (y, x) in ((1, 1), (0, 0)):
        assert phi_ref[0, y, x] - phi[0, y, x] == pytest.approx(Q / 2, rel=1e-12), (y, x)
    assert _invariant(s.ledger()) == pytest.approx(_invariant(L0), rel=1e-13)
    open_before = s.ledger()["open_in"]
    s.step(5)
    L = s.ledger()
    assert L["open_in"] > open_before
    assert _invariant(L) == pytest.approx(_invariant(L0), rel=1e-13)


def test_corner_precipitations_split_by_post_event_normals_by_hand():
    """Two bumps precipitate in the same step in a concave corner (walls at
    x <= 1 and y <= 1), each next to one wall, diagonal to each other, with
    the fluid cell (3, 3) as a shared neighbour (reading R5).  The normals are
    taken on the post-event geometry, so each bump sees the other: at (2, 3)
    the isotropic gradient of the solid indicator (D2Q9 weights times 36) is
    4 (-1, 0) + (-1, -1) + (-1, 1) + (1, -1) = (-5, -1), n = (5, 1) / sqrt(26),
    and the excess splits 5 : 1 between the links +x and +y (the link -y has
    (e.n)+ = 0); by symmetry (3, 2) splits 5 : 1 between +y and +x.  The
    shared cell receives 5/6 of each excess, the corner cell (2, 2) none."""
    n, Vm = 8, 0.4
    mask = np.zeros((1, n, n), np.uint8)
    mask[0, 0:2, :] = 1
    mask[0, :, 0:2] = 1
    phi0 = np.where(mask == 1, 1.0, 0.0)
    phi0[0, 3, 2] = phi0[0, 2, 3] = 1.0 - 1e-12
    p = dict(dim=2, nx=n, ny=n, flow_q=0, solute_q=5, bc=("periodic",) * 3, tau_solute=1.0, k_r=0.5, c_eq=0.0,
             c_init=1.0, molar_volume=Vm)
    ref = oracle.OracleSim(dict(p, phase_change=0), mask, phi_init=phi0)
    ref.step(1)
    _, _, c_ref, phi_ref = ref.fields()
    s = oracle.OracleSim(dict(p, phase_change=1), mask, phi_init=phi0)
    L0 = s.ledger()
    s.step(1)
    assert s.events().tolist() == [[0, 3 + 2 * n, oracle.EV_PRECIPITATE], [0, 2 + 3 * n, oracle.EV_PRECIPITATE]]
    nrm = s.normals()[0]
    assert np.allclose(nrm[3, 2, :2], np.array([5.0, 1.0]) / np.sqrt(26.0), rtol=1e-15)
    assert np.allclose(nrm[2, 3, :2], np.array([1.0, 5.0]) / np.sqrt(26.0), rtol=1e-15)
    _, _, c, phi = s.fields()
    eA = (phi_ref[0, 3, 2] + Vm * c_ref[0, 3, 2] - 1.0) / Vm
    eB = (phi_ref[0, 2, 3] + Vm * c_ref[0, 2, 3] - 1.0) / Vm
    assert eA > 0.0 and eB > 0.0
    assert c[0, 3, 3] == pytest.approx(c_ref[0, 3, 3] + 5.0 / 6.0 * (eA + eB), rel=1e-13)
    assert c[0, 4, 2] == pytest.approx(c_ref[0, 4, 2] + eA / 6.0, rel=1e-13)
    assert c[0, 2, 4] == pytest.approx(c_ref[0, 2, 4] + eB / 6.0, rel=1e-13)
    assert c[0, 2, 2] == pytest.approx(c_ref[0, 2, 2], rel=1e-14)
    assert phi[0, 3, 2] == 1.0 and phi[0, 2, 3] == 1.0
    assert _invariant(s.ledger()) == pytest.approx(_invariant(L0), rel=1e-13)


def test_threaded_cell_loop_changes_nothing_but_the_sum_order():
    # the all-cores timing mode of the oracle: z-slabs on host threads
    shape = (13, 10, 24)
    mask = workloads.sphere_pack(shape, 0.55, 2.0, 3.5, seed=9, periodic=(False, True, True), buffer_x=2)
    p = dict(dim=3, nx=24, ny=10, nz=13, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"), tau_flow=0.8,
             magic_flow=3.0 / 16.0, tau_solute=0.9, k_r=0.2, c_eq=1.0, c_init=2.0, c_inlet=2.0, u_inlet=0.02,
             molar_volume=0.3, phase_change=1)
    a, b = oracle.OracleSim(p, mask), oracle.OracleSim(p, mask)
    b.set_threads(4)
    a.step(30)
    b.step(30)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    assert a.events().tolist() == b.events().tolist()
    La, Lb = a.ledger(), b.ledger()
    for k in ("open_in", "reacted", "dirichlet_in"):
        assert Lb[k] == pytest.approx(La[k], rel=1e-12, abs=1e-15), k
