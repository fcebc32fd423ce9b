"""lbrbc_mass_ledger_noalloc, the mass balance for callers that cannot
allocate device memory at that point (a program whose GPU memory belongs to
its own pool allocator, or a loop that must not pay cudaFree's device-wide
synchronisation).  It must return what lbrbc_mass_ledger returns, to
round-off, on consecutive calls, also on grids whose reduction spans several
blocks of the static scratch.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2306_10794_gb300 import lbrbc, workloads


@pytest.fixture(scope="module")
def built():
    from paper_2306_10794_gb300 import _build

    _build.build()


def test_noalloc_size_rule_names_the_limit(built):
    # host arithmetic only: the same check the entry point applies before any GPU work
    assert lbrbc.lbrbc_noalloc_size_check(4096 * 65536)[0] == lbrbc.LBRBC_OK
    st, msg = lbrbc.lbrbc_noalloc_size_check(4096 * 65536 + 1)
    assert st == lbrbc.LBRBC_ERR_ARG and "268435456 cells" in msg
    st, msg = lbrbc.lbrbc_noalloc_size_check(65537, max_blocks=1, cells_per_block=65536)
    assert st == lbrbc.LBRBC_ERR_ARG and "65536 cells" in msg
    assert lbrbc.lbrbc_noalloc_size_check(65536, max_blocks=1, cells_per_block=65536)[0] == lbrbc.LBRBC_OK


# (nz, ny, nx): one reduction block (32 400 cells) and four (240 000 cells)
@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(12, 18, 150), (40, 40, 150)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_ledger_matches_allocating_ledger(built, precision, shape):
    nz, ny, nx = shape
    mask = workloads.sphere_pack(shape, 0.55, 2.0, 4.0, seed=21, periodic=(True, False, False))
    mask[:, -2:, :] = workloads.DIRICHLET
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19, solute_q=7, bc=("periodic", "wall", "wall"), tau_flow=0.8,
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
