"""Batched stepping of independent, uneven domains: each domain of a batch
must evolve exactly as it does alone (and as the oracle says), whatever
schedule the autotuner picks."""
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


def _cases(precision, n=7):
    cases, meta = workloads.case_batch(n=n, L_min=9, L_max=37, seed=5, precision=precision)
    # a Dirichlet slab and a k field in two of them
    cases[1][1][:, :, -2:] = workloads.DIRICHLET
    cases[1][0]["c_dirichlet"] = 0.5
    cases[2] = (cases[2][0], cases[2][1], dict(k_field=workloads.lognormal_k(cases[2][1].shape, 0.01, 0.5, 3)))
    return cases


def test_batch_matches_oracle_fp64():
    cases = _cases("fp64")
    b = lbrbc.Batch(cases)
    steps = 23
    b.step(steps)
    for i, (p, mask, init) in enumerate(cases):
        o = oracle.OracleSim(p, mask, **init)
        o.step(steps)
        ug, rg, cg, pg = b.fields(i)
        uo, ro, co, po = o.fields()
        for a, c in ((ug, uo), (rg, ro), (cg, co), (pg, po)):
            assert np.abs(a - c).max() < 1e-11, i


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_autotuned_equals_single_domains(precision):
    cases = _cases(precision)
    b = lbrbc.Batch(cases)
    choice = b.autotune(pairs=1)
    assert choice["ms_per_step"] > 0.0
    # every candidate ran 1 warm-up pair + 1 timed pair: 4 persistent-kernel
    # policies x 2 orders x 3 grids, and the domain-graph schedule with 3
    # branch counts
    n_auto = (4 * 2 * 3 + 3) * 4
    b.step(5)
    total = n_auto + 5
    for i, (p, mask, init) in enumerate(cases):
        s = lbrbc.Sim(p, mask, **init)
        s.step(total)
        ug, _, cg, pg = b.fields(i)
        us, _, cs, ps = s.fields()
        tol = 1e-11 if precision == "fp64" else 2e-6
        for a, c in ((cg, cs), (ug, us), (pg, ps)):
            assert np.abs(a - c).max() <= tol * max(1.0, np.abs(c).max()), i
        led_b = lbrbc.lbrbc_mass_ledger(b.domain(i))
        led_s = lbrbc.lbrbc_mass_ledger(s._h)
        assert np.allclose(led_b[:5], led_s[:5], rtol=1e-6, atol=1e-9)
        assert led_b[5] == total
        s.close()


def test_batch_domain_handles_are_borrowed():
    cases = _cases("fp32", n=3)
    b = lbrbc.Batch(cases)
    h = b.domain(0)
    lbrbc.lbrbc_destroy(h)  # ignored
    with pytest.raises(lbrbc.LbrbcError):
        lbrbc.lbrbc_step(h, 1)
    b.step(2)
    assert np.isfinite(b.fields(1)[2]).all()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_many_small_domains(precision):
    # a hundred-odd small domains: the work items of many domains share every
    # block of the persistent launches, each domain still evolving as it does
    # alone under every tile policy and order and as a branch of the domain
    # graph
    cases, _ = workloads.case_batch(n=110, L_min=9, L_max=16, seed=11, precision=precision)
    b = lbrbc.Batch(cases)
    choice = b.autotune(pairs=1)
    total = (4 * 2 * 3 + 3) * 4 + 3
    b.step(3)
    for i in range(0, 110, 7):
        p, mask, init = cases[i]
        s = lbrbc.Sim(p, mask, **init)
        s.step(total)
        tol = 1e-11 if precision == "fp64" else 2e-6
        for a, c in zip(b.fields(i), s.fields()):
            assert np.abs(a - c).max() <= tol * max(1.0, np.abs(c).max()), (i, choice)
        s.close()


@pytest.mark.parametrize("schedule", [(0, 0, 4), (2, 1, 8), (3, 1, 16), (4, 0, 4), (4, 0, 16)])
def test_batch_fixed_schedules_equal_single_domains(schedule):
    # every schedule, fixed without timing, over 19 steps: the domain-graph
    # schedule then runs its 8-step graphs twice, a pair and a single step
    cases = _cases("fp32", n=9)
    b = lbrbc.Batch(cases)
    b.schedule(*schedule)
    b.step(19)
    for i, (p, mask, init) in enumerate(cases):
        s = lbrbc.Sim(p, mask, **init)
        s.step(19)
        for a, c in zip(b.fields(i), s.fields()):
            assert np.abs(a - c).max() <= 2e-6 * max(1.0, np.abs(c).max()), (i, schedule)
        assert lbrbc.lbrbc_mass_ledger(b.domain(i))[5] == 19
        s.close()
    with pytest.raises(lbrbc.LbrbcError):
        b.schedule(5)
