"""The bridge geometry on the GPU (Table geometries: point supports at (0, 0, z) and
rollers free in x at (x_max, 0, z) for z at the two faces and the mid-plane of the depth,
a unit pressure on the top face) against the oracle's BridgeMesh and bridge_load.

The GPU reads the supports from a per-node bit mask on every level (coarse levels by
injection, like the oracle's Mesh.coarsen); partly fixed nodes (the rollers) keep their
free component in every operator, smoother and transfer.
"""
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def bf16_round(x):
    return torch.as_tensor(x).to(torch.bfloat16).to(torch.float64).numpy()


# grids: nz even (mid-depth supports); the 16x4x8 / 32x8x16 hierarchies keep the mid
# support on every level, 24x6x4 drops it on level 1 (nz / 2 = 2 -> mid at K = 1 of 2 ok),
# 12x4x6 puts it on an odd coarse extent (nz = 3 on level 1: the mid support vanishes)
BRIDGE = [(16, 4, 8, 3), (24, 6, 4, 2), (32, 8, 16, 3), (12, 4, 6, 2), (4, 2, 2, 1)]


def make(gf, nx, ny, nz, L, seed=0, rho_min=1e-3, p=3.0, kind="smooth"):
    if kind == "smooth":
        rho = synth.smoothed_gaussian_density(nx, ny, nz, seed, 2.0, 0.4)
    elif kind == "bernoulli":
        rho = synth.bernoulli_density(nx, ny, nz, seed, 0.5)
    else:
        rho = synth.uniform_density(nx, ny, nz, seed)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_geometry(gf.GF_GEOM_BRIDGE)
    g.set_density(dev(rho), p)
    g.set_floor(rho_min)
    return g, O.BridgeMesh(nx, ny, nz), rho


@pytest.mark.parametrize("nx,ny,nz,L", BRIDGE)
def test_bridge_mask_and_load_match_the_oracle(gf, nx, ny, nz, L):
    g = gf.create_grid(nx, ny, nz, levels=L, h=0.5)
    g.set_geometry(gf.GF_GEOM_BRIDGE)
    m = O.BridgeMesh(nx, ny, nz, h=0.5)
    mask = torch.zeros(g.n_dof, dtype=torch.uint8, device="cuda")
    g.free_mask(mask)
    assert np.array_equal(mask.cpu().numpy().astype(bool), m.free)          # bit-exact
    f = torch.full((g.n_dof,), 7.0, dtype=torch.float64, device="cuda")
    g.bridge_load(f)
    assert np.array_equal(host(f), O.bridge_load(m))                        # exact (multiples of h^2/4)


@pytest.mark.parametrize("nx,ny,nz,L", BRIDGE)
def test_bridge_apply_K_fp64_and_fp32_parity(gf, nx, ny, nz, L, monkeypatch):
    g, m, rho = make(gf, nx, ny, nz, L, seed=nx, kind="uniform")
    E = O.young_modulus(rho, 1e-3, 3.0)
    K0 = O.element_stiffness()
    u = synth.random_vector(m.n_dof, 3)
    ref = O.apply_K(m, E, K0, u)
    y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
    g.apply_K(dev(u), y)                         # modal operator with the support mask
    got = host(y)
    assert relerr(got, ref) <= 1e-10 and np.all(got[m.fixed] == 0.0)
    monkeypatch.setenv("GF_MODAL", "0")          # the dense FP64 node stencil, masked
    gd, _, _ = make(gf, nx, ny, nz, L, seed=nx, kind="uniform")
    yd = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
    gd.apply_K(dev(u), yd)
    assert relerr(host(yd), ref) <= 1e-10
    u32 = u.astype(np.float32)
    y32 = torch.zeros(g.n_dof, dtype=torch.float32, device="cuda")
    g.apply_K_f32(dev(u32, torch.float32), y32)  # the FP32 V-cycle operator (BF16 density)
    ref32 = O.apply_K(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), K0, u32.astype(np.float64))
    assert relerr(host(y32), ref32) <= 2e-5


@pytest.mark.parametrize("nx,ny,nz,L", BRIDGE)
def test_bridge_vcycle_parity(gf, nx, ny, nz, L):
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, kind="bernoulli")
    E = O.young_modulus(rho, 1e-3, 3.0)
    H = O.build_hierarchy(m, E, L)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-9
    # the mixed V-cycle: FP32 levels from the BF16 density, FP64 coarsest inverse
    H16 = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L)
    H16.levels[-1].chol = H.levels[-1].chol
    z32 = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z32, gf.GF_MIXED)
    assert relerr(host(z32), O.vcycle(H16, v)) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [(16, 4, 8, 3, 1e-3), (32, 8, 16, 3, 1e-6)])
def test_bridge_solve_parity_and_oracle_guard(gf, case, prec):
    nx, ny, nz, L, rm = case
    g, m, rho = make(gf, nx, ny, nz, L, seed=5, rho_min=rm)
    f = O.bridge_load(m)
    res, E, K0 = O.solve_at_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L), f, rm, 200, 1e-6)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, kmax=200, tol=1e-6, prec=gf.GF_FP64 if prec == "fp64" else gf.GF_MIXED)
    assert out["flag"] == res.flag and abs(out["iters"] - res.iters) <= (1 if prec == "fp64" else 2)
    k = min(out["iters"], res.iters)
    if prec == "fp64":
        h_gpu, h_ref = np.array(out["history"][:k + 1]), res.history[:k + 1]
        assert np.all(np.abs(h_gpu - h_ref) <= 1e-6 * h_ref + 1e-15)
    uh = host(u)
    assert np.all(uh[m.fixed] == 0.0)
    eta = O.true_residual(m, E, K0, f, uh)
    assert eta <= 1.5e-6
    # the GPU guard against the oracle's on the same u: at a converged u, f - K u cancels,
    # so a 1e-10 relative error in K u moves eta by up to 1e-10 ||K u|| / ||f||
    ku = np.linalg.norm(O.apply_K(m, E, K0, uh))
    assert abs(g.true_residual(dev(f), u) - eta) <= 1e-10 * ku / np.linalg.norm(f)


@pytest.mark.parametrize("seed", [3, 8])
def test_bridge_select_floor_parity(gf, seed):
    """Algorithm 1 on a bridge state: the same probe features, decision, attempts and
    accepted floor as the oracle, and the oracle's guard on the GPU's solution."""
    nx, ny, nz, L = 32, 8, 16, 3
    rho = synth.bernoulli_density(nx, ny, nz, seed, 0.45)
    m = O.BridgeMesh(nx, ny, nz)
    f = O.bridge_load(m)
    ladder = [1e-5, 1e-4, 1e-3]
    ref = O.select_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L), f, 1e-8, ladder, tau=1e-6, kmax=80,
                         probe_iters=100)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_geometry(gf.GF_GEOM_BRIDGE)
    g.set_density(dev(rho), 3.0)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.select_floor(dev(f), u, gf.policy_defaults(rho0=1e-8, ladder=ladder, kmax=80))
    assert out["status"] == ref.status and out["floor_index"] == ref.floor_index
    assert out["escalated"] == ref.escalated
    if not np.isnan(ref.r50):
        assert abs(out["r50"] - ref.r50) <= 1e-4 * ref.r50 and abs(out["r100"] - ref.r100) <= 1e-4 * ref.r100
    assert len(out["attempts"]) == len(ref.attempts)
    for a, b in zip(out["attempts"], ref.attempts):
        assert a["rho_min"] == b.rho_min and abs(a["iters"] - b.iters) <= 1 and a["accepted"] == b.accepted
    if out["status"] == gf.GF_ACCEPTED:
        E = O.young_modulus(rho, out["rho_min"], 3.0)
        assert O.true_residual(m, E, O.element_stiffness(), f, host(u)) <= 1e-6 * (1 + 1e-9)


def test_bridge_refuses_the_cantilever_only_options(gf):
    g, m, rho = make(gf, 16, 4, 8, 3)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.bridge_load(f)
    u = torch.zeros_like(f)
    for kw in (dict(outer=2), dict(outer=1), dict(smoother=1), dict(ls_ratio=0.1), dict(fine_steps=4),
               dict(coarse_steps=4)):
        with pytest.raises(gf.GFError):
            g.solve(f, u, prec=gf.GF_MIXED, **kw)
    with pytest.raises(gf.GFError):
        g.apply_K_split(f, u)
    with pytest.raises(gf.GFError):
        g.set_coarse_operator(gf.GF_COARSE_GALERKIN)
    with pytest.raises(gf.GFError):
        g.set_geometry(7)
    # back to the cantilever: the clamped face again, bit-identical to a fresh grid
    g.set_geometry(gf.GF_GEOM_CANTILEVER)
    g.set_floor(1e-3)
    fresh = gf.create_grid(16, 4, 8, levels=3)
    fresh.set_density(dev(rho), 3.0)
    fresh.set_floor(1e-3)
    x = dev(synth.random_vector(g.n_dof, 4))
    a, b = torch.zeros_like(x), torch.zeros_like(x)
    g.vcycle(x, a, gf.GF_MIXED)
    fresh.vcycle(x, b, gf.GF_MIXED)
    assert torch.equal(a, b)


def test_bridge_modal_operator_forced_run_lengths(gf, monkeypatch):
    """The masked modal operator under forced launch plans (runs of 1, 3 and 5 node
    planes, both tile shapes): the same K*u to rounding."""
    nx, ny, nz, L = 40, 10, 12, 2
    m = O.BridgeMesh(nx, ny, nz)
    rho = synth.uniform_density(nx, ny, nz, 7)
    u = synth.random_vector(m.n_dof, 8)
    ref = O.apply_K(m, O.young_modulus(rho, 1e-4, 3.0), O.element_stiffness(), u)
    for bx in ("32", "16"):
        for chunk in ("1", "3", "5"):
            monkeypatch.setenv("GF_MODAL_BX", bx)
            monkeypatch.setenv("GF_MODAL_CHUNK", chunk)
            g = gf.create_grid(nx, ny, nz, levels=L)
            g.set_geometry(gf.GF_GEOM_BRIDGE)
            g.set_density(dev(rho), 3.0)
            g.set_floor(1e-4)
            y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
            g.apply_K(dev(u), y)
            assert relerr(host(y), ref) <= 1e-10, (bx, chunk)


def test_bridge_half_sm_shapes_are_bit_identical(gf):
    """gf_set_sm_share(1) on the bridge (the masked modal kernels on 16 x 16 tiles, the
    fix-up with per-node supports): FP64 K*u, FP32 K*u and the mixed V-cycle equal those of
    the full-SM shapes bit for bit, and K*u matches the oracle."""
    nx, ny, nz, L = 48, 24, 12, 2
    m = O.BridgeMesh(nx, ny, nz)
    rho = synth.smoothed_gaussian_density(nx, ny, nz, 4, 2.0, 0.4)
    u = synth.random_vector(m.n_dof, 9)
    outs = []
    for share in (0, 1):
        g = gf.create_grid(nx, ny, nz, levels=L)
        g.set_sm_share(share)
        g.set_geometry(gf.GF_GEOM_BRIDGE)
        g.set_density(dev(rho), 3.0)
        g.set_floor(1e-4)
        y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
        g.apply_K(dev(u), y)
        y32 = torch.full((g.n_dof,), np.nan, dtype=torch.float32, device="cuda")
        g.apply_K_f32(dev(u).float(), y32)
        z = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
        g.vcycle(dev(u * m.free), z, gf.GF_MIXED)
        outs.append((host(y), host(y32), host(z)))
        g.close()
    for a, b in zip(outs[0], outs[1]):
        assert not np.isnan(a).any()
        assert np.array_equal(a, b)
    ref = O.apply_K(m, O.young_modulus(rho, 1e-4, 3.0), O.element_stiffness(), u)
    assert relerr(outs[1][0], ref) <= 1e-10
