"""Reactive disc in a channel flow (Sec. 3.3, Table 2) on the GPU: cases 1-3
(transport-limited, below) and case 4
(Pe = 6, Da = 0.178: the reaction-limited case that separates the schemes),
at half the paper's resolution (600 x 300 cells, disc of 120 cells; Re, Pe,
Da and tau kept).  Steady average reaction rate R_avg (Eq.
avgReactionRateMolins) of the four k_i schemes against the paper's values
(tests/golden/table2_molins.txt):

* anti-bounce-back (reaction not limiting) within 5 % of the paper;
* the new scheme within 12 % (the paper's run has twice the resolution);
* the ratios S.V. / S.New and S.P.J. / S.New near the paper's 0.43 and 1.6;
* the outlet integral equals the reacted mass per step of the ledger (the
  steady mass balance) to 1 % of the inflow rate C_in U H / (pi D): the
  integral of C u_x is not the exact discrete flux through the outlet
  plane, an absolute error of the definition."""
import os

import numpy as np
import pytest

from paper_2306_10794_gb300 import experiments, lbrbc, workloads

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_molins.txt")
STEPS, CHUNK = 800_000, 200_000


def paper_table():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        c, pe, da, sv, spj, snew, abb = line.split()
        out[int(c)] = dict(verhaeghe=float(sv), patel_ju=float(spj), new=float(snew), anti_bb=float(abb))
    return out


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()


@pytest.fixture(scope="module")
def rates():
    out = {}
    for scheme in ("verhaeghe", "patel_ju", "new", "anti_bb"):
        p, mask, init, geom = workloads.case_molins(4, scheme, scale=0.5)
        s = lbrbc.Sim(p, mask, **init)
        s.step(STEPS - CHUNK)
        led0 = s.ledger()["reacted"]
        s.step(CHUNK)
        led1 = s.ledger()["reacted"]
        u, _, c, _ = s.fields()
        s.check()
        s.close()
        r_out = experiments.molins_ravg(u, c, geom)[1]
        r_led = -(led1 - led0) / CHUNK / (np.pi * geom["d_obj"]) * geom["to_paper"]
        out[scheme] = (r_out, r_led)
    out["inflow"] = geom["c_in"] * geom["U"] * geom["H"] / (np.pi * geom["d_obj"]) * geom["to_paper"]
    print(out)
    return out


def test_anti_bounce_back_and_new_scheme_against_table_2(rates):
    ref = paper_table()[4]
    assert rates["anti_bb"][0] == pytest.approx(ref["anti_bb"], rel=0.05)
    assert rates["new"][0] == pytest.approx(ref["new"], rel=0.12)


def test_scheme_ratios(rates):
    ref = paper_table()[4]
    new = rates["new"][0]
    assert rates["verhaeghe"][0] / new == pytest.approx(ref["verhaeghe"] / ref["new"], rel=0.2)
    assert rates["patel_ju"][0] / new == pytest.approx(ref["patel_ju"] / ref["new"], rel=0.2)
    assert rates["verhaeghe"][0] < new < rates["patel_ju"][0] < rates["anti_bb"][0]


# Cases 1-3 (Pe = 600, Da = 178; Pe = 600, Da = 17800; Pe = 6, Da = 178) are
# transport-limited: every scheme consumes nearly all the solute that reaches
# the disc and the paper's four columns differ by at most 5 %.  Run at half
# the paper's resolution with the new scheme and, for case 1 where the
# paper's columns differ most, the scheme without gamma; measured 4.62 / 4.62
# / 74.8 for the new scheme and 4.62 for case 1 without gamma (paper 4.64 /
# 4.70 / 75.8 and 4.48).  Asserted: within 5 % of the paper for Pe = 600
# (the outlet integral there deviates from the exact ledger rate by 4 %,
# dispersion of C over the outlet plane at this Peclet number), within 2 %
# for case 3.
@pytest.mark.parametrize("case,scheme,tol", [(1, "new", 0.05), (1, "verhaeghe", 0.05), (2, "new", 0.05),
                                             (3, "new", 0.02)])
def test_transport_limited_cases_against_table_2(case, scheme, tol):
    p, mask, init, geom = workloads.case_molins(case, scheme, scale=0.5)
    s = lbrbc.Sim(p, mask, **init)
    steps = 500_000 if case == 3 else 1_125_000
    s.step(steps)
    u, _, c, _ = s.fields()
    s.check()
    s.close()
    r_out = experiments.molins_ravg(u, c, geom)[1]
    assert r_out == pytest.approx(paper_table()[case][scheme], rel=tol), r_out


def test_outlet_integral_matches_ledger(rates):
    for scheme in ("verhaeghe", "patel_ju", "new", "anti_bb"):
        r_out, r_led = rates[scheme]
        assert abs(r_out - r_led) < 0.01 * rates["inflow"], scheme
