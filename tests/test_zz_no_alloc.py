"""The allocation-free guard (gf_true_residual_noalloc) against the grid-based one.

gf_true_residual_noalloc serves callers that cannot allocate device memory (work
recorded into a CUDA graph or under stream capture, fixed memory budgets): its
scratch is a static array inside the library. It must return the same acceptance
residual as gf_true_residual. This file is collected last on purpose and works both
alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synth
from oracle import gf_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the tolerance the FP64 guard parity tests use (relative)
RTOL = 1e-10


@pytest.fixture(scope="module")
def gf():
    from paper_2607_26382_b300 import build
    build.build()
    import paper_2607_26382_b300 as gf
    return gf


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("dims", [(24, 12, 8), (96, 48, 48)])
def test_noalloc_guard_matches_grid_guard_twice(gf, dims):
    nx, ny, nz = dims
    rho = _dev(synth.smoothed_gaussian_density(nx, ny, nz, 3))
    m_ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    f = torch.zeros(m_ndof, dtype=torch.float64, device="cuda")
    g = gf.create_grid(nx, ny, nz, levels=2 if nx == 24 else 5)
    g.cantilever_load(f)
    g.set_density(rho, 3.0)
    g.set_floor(1e-4)
    eta = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    # two calls in a row on different inputs: the shared scratch keeps the first
    # call's contents, which must not leak into the second
    for seed, scale in ((1, 1e-2), (2, 3.0)):
        u = _dev(synth.random_vector(m_ndof, seed) * scale)
        ref = g.true_residual(f, u)
        gf.true_residual_noalloc(nx, ny, nz, rho, 3.0, 1e-4, f, u, eta)
        torch.cuda.synchronize()
        got = float(eta.item())
        assert abs(got - ref) <= RTOL * ref, (got, ref)
    g.close()


def test_noalloc_guard_rejects_oversize_grid(gf):
    nx, ny, nz = 128, 64, 64            # 1,622,400 DOFs > 1,048,576
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rho = torch.zeros(nx * ny * nz, dtype=torch.float64, device="cuda")
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gf.GFError) as e:
        gf.true_residual_noalloc(nx, ny, nz, rho, 3.0, 1e-3, x, x, eta)
    assert e.value.code == -1 and "1048576" in str(e.value)


def test_noalloc_guard_scaling_and_fractional_p(gf):
    """h, E0 and nu away from their defaults and a non-integer p (the paper's 4.5, which
    takes the pow() branch of the modulus): the same residual as gf_true_residual on a
    grid created with the same parameters, and as the oracle's FP64 guard."""
    nx, ny, nz = 16, 6, 4
    h, E0, nu, p, rho_min = 0.37, 210.0, 0.27, 4.5, 1e-5
    rho_h = synth.uniform_density(nx, ny, nz, 11)
    rho = _dev(rho_h)
    g = gf.create_grid(nx, ny, nz, h=h, E0=E0, nu=nu, levels=2)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    g.set_density(rho, p)
    g.set_floor(rho_min)
    u_h = synth.random_vector(g.n_dof, 12)
    u = _dev(u_h)
    ref = g.true_residual(f, u)
    eta = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    gf.true_residual_noalloc(nx, ny, nz, rho, p, rho_min, f, u, eta, h=h, E0=E0, nu=nu)
    got = float(eta.item())
    assert abs(got - ref) <= RTOL * ref, (got, ref)
    m = O.Mesh(nx, ny, nz, h)
    E = E0 * O.young_modulus(rho_h, rho_min, p)
    oracle = O.true_residual(m, E, O.element_stiffness(h, 1.0, nu), f.cpu().numpy(), u_h)
    assert abs(got - oracle) <= RTOL * oracle, (got, oracle)
    g.close()


def test_noalloc_guard_zero_load_gives_nan(gf):
    """A load that vanishes on every free DOF has no relative residual: the call still
    returns GF_OK and writes NaN, which no tolerance accepts."""
    nx, ny, nz = 8, 4, 4
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    rho = _dev(synth.uniform_density(nx, ny, nz, 1))
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    f[0:3] = 1.0                      # node 0 sits on the clamped face: masked out
    u = _dev(synth.random_vector(n, 2))
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    gf.true_residual_noalloc(nx, ny, nz, rho, 3.0, 1e-3, f, u, eta)
    got = float(eta.item())
    assert np.isnan(got) and not (got <= 1e-6)
