"""Pins of the oracle's building blocks against what the paper prints and
what the mathematics fixes: velocity sets (Appendix A), rest-fraction
weights (Eqs. RestFraction, RestFractionCs2; Table S1), equilibrium moments
(Eqs. fluid_Equilib, solute_equilibrium_function) and the limits of the
reactive boundary condition (Eq. general_RBC, Sec. 2.3)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2306_10794_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_appendix_a_tables():
    rows = _read("appendix_a_lattices.txt")
    for name, q in (("D2Q9", 9), ("D2Q5", 5)):
        e, w, cs2, _ = oracle.lattice(q, 2)
        mine = [r for r in rows if r[0] == name]
        assert len(mine) == q
        for r in mine:
            i = int(r[1])
            assert (e[i, 0], e[i, 1]) == (int(r[2]), int(r[3]))
            assert w[i] == pytest.approx(float(Fraction(r[4])), abs=1e-16)
        assert cs2 == pytest.approx(1.0 / 3.0, abs=1e-16)


@pytest.mark.parametrize("q,dim,J0", [(9, 2, -1), (5, 2, -1), (5, 2, 0.1), (5, 2, 0.9), (19, 3, -1),
                                      (7, 3, -1), (7, 3, 0.4), (7, 3, 0.994)])
def test_isotropy(q, dim, J0):
    e, w, cs2, opp = oracle.lattice(q, dim, J0)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-16
    second = np.einsum("i,ia,ib->ab", w, e, e)
    expect = cs2 * np.eye(3)
    if dim == 2:
        expect[2, 2] = 0.0
    assert np.abs(second - expect).max() < 1e-15
    assert all((e[opp[i]] == -e[i]).all() for i in range(q))


def test_rest_fraction_table_s1():
    for J0, cs2_printed, tau_printed in [[float(x) for x in r] for r in _read("table_s1_rest_fraction.txt")]:
        e, w, cs2, _ = oracle.lattice(5, 2, J0)
        assert cs2 == pytest.approx(cs2_printed, abs=1e-12)
        assert w[0] == pytest.approx(J0, abs=1e-15)
        assert np.allclose(w[1:], cs2 / 2.0, atol=1e-16)
        # tau_AD of Text S2 follows from keeping D = cs2 (tau - 1/2) fixed
        D = (1.0 / 3.0) * (0.74 - 0.5)
        assert 0.5 + D / cs2 == pytest.approx(tau_printed, abs=1e-12)
        got = workloads.params_from_dimensionless(Pe=1.0, L=80.0, U=0.001, rest_fraction=J0, solute_q=5, dim=2)
        assert got["tau_solute"] == pytest.approx(tau_printed, abs=1e-12)


def test_rest_fraction_default_weights():
    # J0 = 1/3 (D2Q5) and 1/4 (D3Q7) give the common weights (Sec. 2.2)
    _, w, cs2, _ = oracle.lattice(5, 2, 1.0 / 3.0)
    _, w0, cs20, _ = oracle.lattice(5, 2, -1)
    assert np.allclose(w, w0, atol=1e-16) and cs2 == pytest.approx(cs20, abs=1e-16)
    _, w7, cs27, _ = oracle.lattice(7, 3, 0.25)
    assert np.allclose(w7, [0.25] + [0.125] * 6, atol=1e-16) and cs27 == 0.25


@pytest.mark.parametrize("q,dim", [(9, 2), (19, 3)])
def test_flow_equilibrium_moments(q, dim):
    e, w, cs2, _ = oracle.lattice(q, dim)
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        if dim == 2:
            u[2] = 0.0
        feq = oracle.equilibrium(q, dim, rho, u, solute=False)
        assert feq.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose((feq[:, None] * e).sum(0), rho * u, atol=1e-15)
        pi = np.einsum("i,ia,ib->ab", feq, e, e)
        expect = rho * cs2 * np.eye(3) + rho * np.outer(u, u)
        if dim == 2:
            expect[2, :] = expect[:, 2] = 0.0
        assert np.abs(pi - expect).max() < 1e-14


@pytest.mark.parametrize("q,dim,J0", [(5, 2, -1), (5, 2, 0.1), (7, 3, -1), (7, 3, 0.9), (9, 2, -1)])
def test_solute_equilibrium_moments(q, dim, J0):
    e, w, cs2, _ = oracle.lattice(q, dim, J0)
    u = np.array([0.01, -0.02, 0.015 if dim == 3 else 0.0])
    geq = oracle.equilibrium(q, dim, 0.7, u, solute=True, rest_fraction=J0)
    assert geq.sum() == pytest.approx(0.7, abs=1e-15)
    assert np.allclose((geq[:, None] * e).sum(0), 0.7 * u, atol=1e-15)


def test_rbc_limits():
    w, ceq = 1.0 / 6.0, 0.3
    for gt in (0.0, 0.05, 0.2):
        # k_r = 0: plain bounce-back of the incoming population
        assert oracle.rbc(0.0, w, ceq, gt) == gt
        # k_r -> infinity: anti-bounce-back 2 w C_eq - g~
        assert oracle.rbc(1e12, w, ceq, gt) == pytest.approx(2 * w * ceq - gt, abs=1e-12)
        assert oracle.rbc(0.0, w, ceq, gt, infinite=True) == pytest.approx(2 * w * ceq - gt, abs=1e-16)
    # an incoming population at the reaction equilibrium is reflected unchanged, for any k
    for k in (0.0, 0.1, 1.0, 7.0, 1e6):
        assert oracle.rbc(k, w, ceq, w * ceq) == pytest.approx(w * ceq, abs=1e-15)
