"""The discrete adjoint (lbrbc_adjoint) against central finite differences
of the reacted mass -- through the independent FP64 oracle and through the
FP64 CUDA path -- for the scalar k_r, c_eq and sampled cells of a per-voxel
k field; FP32 forward against the FP64 gradients; the torch autograd
wrapper."""
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


def _case(flow=True, scheme="new", trt=False):
    shape = (10, 14, 30)
    mask = workloads.sphere_pack(shape, 0.6, 2.0, 3.5, seed=13, periodic=(False, True, True), buffer_x=2)
    p = dict(dim=3, nx=30, ny=14, nz=10, flow_q=19 if flow else 0, solute_q=7, bc=("open", "periodic", "periodic"),
             tau_flow=0.8, magic_flow=3.0 / 16.0, tau_solute=0.9, magic_solute=0.25 if trt else -1.0,
             rest_fraction=0.4, k_r=0.05, c_eq=1.0, c_init=0.2, c_inlet=0.0, u_inlet=0.01, rho_outlet=1.0,
             molar_volume=0.1, scheme=scheme, precision="fp64")
    return p, mask


def _J_oracle(p, mask, n, **init):
    o = oracle.OracleSim(p, mask, **init)
    L0 = o.ledger()["reacted"]
    o.step(n)
    return o.ledger()["reacted"] - L0


@pytest.mark.parametrize("flow,scheme,trt", [(True, "new", False), (True, "verhaeghe", True), (False, "new", False)])
def test_scalar_gradients_vs_oracle_fd(flow, scheme, trt):
    p, mask = _case(flow, scheme, trt)
    n = 60
    sim = lbrbc.Sim(p, mask)
    J, dk, dc, _ = sim.adjoint(n)
    assert J == pytest.approx(_J_oracle(p, mask, n), rel=1e-11)
    for key, g in (("k_r", dk), ("c_eq", dc)):
        h = 1e-4 * p[key]
        Jp = _J_oracle(dict(p, **{key: p[key] + h}), mask, n)
        Jm = _J_oracle(dict(p, **{key: p[key] - h}), mask, n)
        fd = (Jp - Jm) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-4), (key, g, fd)


def test_kfield_gradient_vs_fd_and_state_advance():
    p, mask = _case()
    n = 50
    kf = workloads.lognormal_k(mask.shape, 0.05, 0.5, seed=9)
    sim = lbrbc.Sim(p, mask, k_field=kf)
    J, dk, dc, g = sim.adjoint(n, field=True)
    cls = sim.classes()
    # after the adjoint the simulation stands n steps later, as after step(n)
    ref = lbrbc.Sim(p, mask, k_field=kf)
    ref.step(n)
    assert np.abs(sim.fields()[2] - ref.fields()[2]).max() < 1e-13
    assert sim.ledger()["reacted"] == pytest.approx(ref.ledger()["reacted"], rel=1e-12)
    assert dk == pytest.approx(g.sum(), rel=1e-10)
    assert np.all(g[cls != lbrbc.CLASS_BOUND] == 0.0)
    bound = np.argwhere(cls == lbrbc.CLASS_BOUND)
    rng = np.random.default_rng(1)
    for z, y, x in bound[rng.choice(len(bound), 4, replace=False)]:
        h = 1e-3 * kf[z, y, x]
        kp, km = kf.copy(), kf.copy()
        kp[z, y, x] += h
        km[z, y, x] -= h
        fd = (_J_oracle(p, mask, n, k_field=kp) - _J_oracle(p, mask, n, k_field=km)) / (2 * h)
        assert g[z, y, x] == pytest.approx(fd, rel=1e-4, abs=1e-12 * abs(dk)), (x, y, z)


def test_fp32_forward_gradients_close_to_fp64():
    p, mask = _case()
    n = 60
    g64 = lbrbc.Sim(p, mask).adjoint(n)
    g32 = lbrbc.Sim(dict(p, precision="fp32"), mask).adjoint(n)
    for a, b in zip(g32[:3], g64[:3]):
        assert a == pytest.approx(b, rel=1e-4)


def test_torch_autograd_wrapper():
    torch = pytest.importorskip("torch")
    p, mask = _case()
    kf = torch.tensor(workloads.lognormal_k(mask.shape, 0.05, 0.5, seed=2), dtype=torch.float64, requires_grad=True)
    ceq = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = lbrbc.reacted_mass(p, mask, 40, kf, ceq)
    J.backward()
    sim = lbrbc.Sim(dict(p, c_eq=1.0), mask, k_field=kf.detach().numpy())
    J2, dk, dc, g = sim.adjoint(40, field=True)
    assert float(J.detach()) == pytest.approx(J2, rel=1e-13)
    assert np.allclose(kf.grad.numpy(), g, rtol=1e-12, atol=0)
    assert float(ceq.grad) == pytest.approx(dc, rel=1e-12)


@pytest.mark.parametrize("flow,scheme,trt", [(True, "new", False), (True, "verhaeghe", True),
                                             (False, "patel_ju", False)])
def test_gradients_match_oracle_discrete_adjoint(flow, scheme, trt):
    # the FP64 CUDA adjoint against the oracle's own discrete adjoint,
    # element by element (per-voxel k field) and for the scalars
    p, mask = _case(flow, scheme, trt)
    n = 45
    kf = workloads.lognormal_k(mask.shape, 0.05, 0.5, seed=21)
    J, dk, dc, g = lbrbc.Sim(p, mask, k_field=kf).adjoint(n, field=True)
    Jo, dko, dco, go = oracle.OracleSim(p, mask, k_field=kf).adjoint(n, field=True)
    assert J == pytest.approx(Jo, rel=1e-11)
    assert dk == pytest.approx(dko, rel=1e-10)
    assert dc == pytest.approx(dco, rel=1e-10)
    scale = np.abs(go).max()
    assert scale > 0.0
    assert np.abs(g - go).max() <= 1e-10 * scale
    nz = go != 0.0
    assert np.array_equal(g != 0.0, nz)
    assert np.allclose(g[nz], go[nz], rtol=1e-9, atol=1e-12 * scale)
