"""GPU parity of the optimisation loop around the solve (filter, adjoint, OC update,
compliance, one guarded SIMP-OC iteration) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import gf_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    from paper_2607_26382_b300 import build
    build.build()
    import paper_2607_26382_b300 as gf
    return gf


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("dims", [(16, 8, 8), (13, 6, 4)])
@pytest.mark.parametrize("r", [1.5, 2.5])
def test_filter_and_adjoint_parity(gf, dims, r):
    nx, ny, nz = dims
    g = gf.create_grid(nx, ny, nz, levels=1 if nx == 13 else 2)
    m = O.Mesh(nx, ny, nz)
    Hf = O.filter_weights(m, r)
    x = synth.uniform_density(nx, ny, nz, 1)
    out = torch.zeros(g.n_elem, dtype=torch.float64, device="cuda")
    g.filter(dev(x), out, r)
    ref = O.density_filter(Hf, x)
    assert np.abs(host(out) - ref).max() <= 1e-13
    gs = synth.random_vector(m.n_elem, 2)
    g.filter_adjoint(dev(gs), out, r)
    ref = O.density_filter_adjoint(Hf, gs)
    assert np.abs(host(out) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_oc_update_parity(gf):
    nx, ny, nz = 16, 8, 8
    g = gf.create_grid(nx, ny, nz, levels=2)
    x = 0.1 + 0.5 * synth.uniform_density(nx, ny, nz, 3)
    dc = -(0.05 + synth.uniform_density(nx, ny, nz, 4))
    dv = 0.5 + synth.uniform_density(nx, ny, nz, 5)
    xn = torch.zeros(g.n_elem, dtype=torch.float64, device="cuda")
    g.oc_update(dev(x), dev(dc), dev(dv), xn, 0.3, 0.2)
    ref = O.oc_update(x, dc, dv, 0.3, move=0.2)
    assert np.abs(host(xn) - ref).max() <= 1e-12
    assert abs(host(xn).mean() - 0.3) < 2e-3


def test_compliance(gf):
    g = gf.create_grid(8, 4, 4, levels=1)
    f, u = synth.random_vector(g.n_dof, 1), synth.random_vector(g.n_dof, 2)
    assert abs(g.compliance(dev(f), dev(u)) - f @ u) <= 1e-13 * np.abs(f * u).sum()


def test_oc_iterations_match_oracle(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    m = O.Mesh(nx, ny, nz)
    f = O.cantilever_load(m)
    x = np.full(m.n_elem, 0.3)
    g = gf.create_grid(nx, ny, nz, levels=L)
    pol = gf.policy_defaults(rho0=1e-6, ladder=[1e-5, 1e-4, 1e-3], kmax=200)
    xd = dev(x)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    kw = dict(rho0=1e-6, ladder=[1e-5, 1e-4, 1e-3], tau=1e-6, kmax=200, probe_iters=100)
    for it in range(3):
        out = g.oc_iteration(xd, dev(f), u, pol, p=3.0, volfrac=0.3, r_min=1.5, move=0.2)
        x, res, C = O.oc_iteration(m, x, f, 3.0, 0.3, 1.5, 0.2, kw, L)
        assert out["status"] == res.status and out["floor_index"] == res.floor_index
        assert abs(out["compliance"] - C) <= 1e-6 * abs(C)
        assert np.abs(host(xd) - x).max() <= 1e-5
