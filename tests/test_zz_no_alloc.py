"""lbrbc_mass_ledger_noalloc, the mass balance for callers that cannot
allocate device memory at that point (a program whose GPU memory belongs to
its own pool allocator, or a loop that must not pay cudaFree's device-wide
synchronisation).  It must return what lbrbc_mass_ledger returns, to
round-off, on consecutive calls.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2306_10794_gb300 import lbrbc, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_ledger_matches_allocating_ledger(precision):
    shape = (12, 18, 150)
    mask = workloads.sphere_pack(shape, 0.55, 2.0, 4.0, seed=21, periodic=(True, False, False))
    mask[:, -2:, :] = workloads.DIRICHLET
    p = dict(dim=3, nx=150, ny=18, nz=12, flow_q=19, solute_q=7, bc=("periodic", "wall", "wall"), tau_flow=0.8,
             tau_solute=0.9, k_r=0.2, c_eq=1.0, c_init=2.5, c_dirichlet=2.0, molar_volume=0.3, phase_change=1,
             precision=precision)
    sim = lbrbc.Sim(p, mask)
    for steps in (0, 37, 12):
        sim.step(steps)
        ref = lbrbc.lbrbc_mass_ledger(sim._h)
        first = lbrbc.lbrbc_mass_ledger_noalloc(sim._h)
        second = lbrbc.lbrbc_mass_ledger_noalloc(sim._h)
        for got in (first, second):
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), (got, ref)
        assert np.array_equal(first, second)
    sim.close()
