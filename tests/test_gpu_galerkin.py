"""GPU parity of the Galerkin coarse operators (gf_set_coarse_operator, Table
solver-config's K_{l+1} = P^T K_l P) against the oracle's assembled Galerkin hierarchy:
V-cycles in FP64 and mixed (Jacobi and Chebyshev smoothing, the line search, the
coarse-level Krylov solve), solve histories, the constant-modulus case where Galerkin and
rediscretised coarse levels coincide, and switching between the two."""
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


def bf16_round(x):
    return torch.as_tensor(x).to(torch.bfloat16).to(torch.float64).numpy()


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def galerkin_grid(gf, nx, ny, nz, L, rho, rho_min, p=3.0):
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), p)
    g.set_coarse_operator(gf.GF_COARSE_GALERKIN)
    g.set_floor(rho_min)
    return g


# grids with 2..4 levels, odd coarse counts, a one-element-thick coarsest level
GRIDS = [(16, 8, 8, 3), (24, 10, 6, 2), (32, 16, 16, 4), (52, 24, 20, 3), (8, 4, 4, 3)]


@pytest.mark.parametrize("nx,ny,nz,L", GRIDS)
@pytest.mark.parametrize("kind", ["uniform", "bernoulli"])
def test_vcycle_fp64_galerkin_parity(gf, nx, ny, nz, L, kind):
    rho = (synth.uniform_density(nx, ny, nz, 2) if kind == "uniform"
           else synth.bernoulli_density(nx, ny, nz, 2, 0.35))
    m = O.Mesh(nx, ny, nz)
    g = galerkin_grid(gf, nx, ny, nz, L, rho, 1e-6)
    E = O.young_modulus(rho, 1e-6, 3.0)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    for nu in (1, 2):
        H = O.build_hierarchy(m, E, L, nu1=nu, nu2=nu, coarse="galerkin")
        z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.vcycle(dev(v), z, gf.GF_FP64, nu1=nu, nu2=nu)
        assert relerr(host(z), O.vcycle(H, v)) <= 1e-9
    g.close()


@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (32, 16, 16, 4)])
def test_vcycle_mixed_galerkin_parity(gf, nx, ny, nz, L):
    # FP32 element matrices come from the BF16-density moduli; the coarsest inverse
    # from the FP64 ones
    rho = synth.smoothed_gaussian_density(nx, ny, nz, 3)
    m = O.Mesh(nx, ny, nz)
    g = galerkin_grid(gf, nx, ny, nz, L, rho, 1e-3)
    H = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L, coarse="galerkin")
    H64 = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L, coarse="galerkin")
    H.levels[-1].chol = H64.levels[-1].chol
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_MIXED)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-4
    g.close()


def test_vcycle_galerkin_with_coarse_krylov_parity(gf):
    # the coarse-level inner Krylov solve on the assembled Galerkin coarsest operator
    nx, ny, nz, L = 32, 16, 16, 4
    rho = synth.bernoulli_density(nx, ny, nz, 5, 0.3)
    m = O.Mesh(nx, ny, nz)
    g = galerkin_grid(gf, nx, ny, nz, L, rho, 1e-3)
    H = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L, coarse="galerkin", coarse_steps=10)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64, coarse_steps=10)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-9
    g.close()


@pytest.mark.parametrize("theta", [0.1, 1e30])
def test_vcycle_galerkin_with_line_search_parity(gf, theta):
    # the line-searched coarse correction on Galerkin levels: K c with the level's
    # assembled operator (theta = 1e30 rejects every correction: smoothing only)
    nx, ny, nz, L = 32, 16, 16, 4
    rho = synth.bernoulli_density(nx, ny, nz, 6, 0.3)
    m = O.Mesh(nx, ny, nz)
    g = galerkin_grid(gf, nx, ny, nz, L, rho, 1e-3)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    H = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L, coarse="galerkin", ls_ratio=theta)
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64, ls_ratio=theta)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-9
    Hm = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L, coarse="galerkin", ls_ratio=theta)
    Hm.levels[-1].chol = H.levels[-1].chol
    z.zero_()
    g.vcycle(dev(v), z, gf.GF_MIXED, ls_ratio=theta)
    assert relerr(host(z), O.vcycle(Hm, v)) <= 1e-4
    g.close()


@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (32, 16, 16, 4)])
def test_chebyshev_on_galerkin_levels_parity(gf, nx, ny, nz, L):
    # Chebyshev smoothing on the assembled levels: lambda_max of D^{-1} K by the power
    # method and the V-cycle, in FP64 and mixed
    rho = synth.bernoulli_density(nx, ny, nz, 8, 0.3)
    m = O.Mesh(nx, ny, nz)
    g = galerkin_grid(gf, nx, ny, nz, L, rho, 1e-3)
    H = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L, coarse="galerkin", smoother="chebyshev")
    assert np.allclose(g.chebyshev_lambda(gf.GF_FP64), [lev.lam for lev in H.levels[:-1]], rtol=1e-10, atol=0)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64, smoother=1)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-9
    Hm = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L, coarse="galerkin",
                           smoother="chebyshev")
    Hm.levels[-1].chol = H.levels[-1].chol
    assert np.allclose(g.chebyshev_lambda(gf.GF_MIXED), [lev.lam for lev in Hm.levels[:-1]], rtol=1e-5, atol=0)
    z.zero_()
    g.vcycle(dev(v), z, gf.GF_MIXED, smoother=1)
    assert relerr(host(z), O.vcycle(Hm, v)) <= 1e-4
    f = dev(O.cantilever_load(m))
    u = torch.zeros_like(z)
    assert g.solve(f, u, smoother=1, kmax=200)["flag"] == gf.GF_FLAG_CONVERGED
    g.close()


def test_galerkin_equals_rediscretised_at_constant_modulus(gf):
    # Q1 spaces are nested: at constant modulus P^T K_h P = K_2h, so both coarse forms
    # give the same V-cycle (to rounding)
    nx, ny, nz, L = 32, 16, 8, 3
    rho = np.ones(nx * ny * nz)
    v = dev(synth.random_vector(3 * (nx + 1) * (ny + 1) * (nz + 1), 4))
    out = []
    for kind in (gf.GF_COARSE_REDISCRETISED, gf.GF_COARSE_GALERKIN):
        g = gf.create_grid(nx, ny, nz, levels=L)
        g.set_density(dev(rho), 3.0)
        g.set_coarse_operator(kind)
        g.set_floor(1e-3)
        z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.vcycle(v, z, gf.GF_FP64)
        out.append(host(z))
        g.close()
    assert relerr(out[1], out[0]) <= 1e-10


# Bernoulli state at rho_min 1e-3 (59 oracle steps, 61 rediscretised) and a smoothed
# Gaussian one at 1e-6 (25 and 27)
@pytest.mark.parametrize("prec,outer", [(0, 0), (1, 2)])
@pytest.mark.parametrize("kind,rho_min", [("bernoulli", 1e-3), ("gauss", 1e-6)])
def test_solve_galerkin_parity(gf, prec, outer, kind, rho_min):
    nx, ny, nz, L = 16, 8, 8, 3
    rho = (synth.bernoulli_density(nx, ny, nz, 4, 0.35) if kind == "bernoulli"
           else synth.smoothed_gaussian_density(nx, ny, nz, 4))
    m = O.Mesh(nx, ny, nz)
    f = O.cantilever_load(m)
    g = galerkin_grid(gf, nx, ny, nz, L, rho, rho_min)
    res, E, K0 = O.solve_at_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L, coarse="galerkin"), f, rho_min, 200,
                                  1e-6)
    assert res.flag == O.CONVERGED
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, restart=30, kmax=200, tol=1e-6, prec=prec, outer=outer)
    assert out["flag"] == res.flag
    if prec == 0:
        assert abs(out["iters"] - res.iters) <= 1
        k = min(out["iters"], res.iters)
        h_gpu, h_ref = np.array(out["history"][:k + 1]), res.history[:k + 1]
        assert np.all(np.abs(h_gpu - h_ref) <= 1e-6 * h_ref + 1e-15)
    else:   # FP32 smoothing on the BF16 density: the same count within the mixed tolerance
        assert abs(out["iters"] - res.iters) <= max(2, res.iters // 10)
    if res.flag == O.CONVERGED:
        assert O.true_residual(m, E, K0, f, host(u)) <= 1.5e-6
    g.close()


def test_galerkin_options_and_switching(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    rho = synth.uniform_density(nx, ny, nz, 1)
    m = O.Mesh(nx, ny, nz)
    f, u = dev(O.cantilever_load(m)), torch.zeros(3 * (nx + 1) * (ny + 1) * (nz + 1), dtype=torch.float64,
                                                  device="cuda")
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), 3.0)
    g.set_floor(1e-3)
    with pytest.raises(gf.GFError):
        g.set_coarse_operator(7)
    it_re = g.solve(f, u, kmax=60)["iters"]
    g.set_coarse_operator(gf.GF_COARSE_GALERKIN)
    with pytest.raises(gf.GFError):          # the floor was cleared
        g.solve(f, u.zero_(), kmax=60)
    g.set_floor(1e-3)
    out = g.solve(f, u.zero_(), kmax=60, fine_steps=5)   # the fine-level correction composes
    assert out["flag"] == gf.GF_FLAG_CONVERGED
    g.set_coarse_operator(gf.GF_COARSE_REDISCRETISED)
    g.set_floor(1e-3)
    assert g.solve(f, u.zero_(), kmax=60)["iters"] == it_re
    g.close()
