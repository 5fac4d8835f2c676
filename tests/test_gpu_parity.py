"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical
seeded inputs.

Tolerances: FP64 operator / guard / sensitivity 1e-10 relative (the stated bar);
FP64 V-cycle 1e-9 relative (a composite of smoothers, transfers and a dense inverse
whose rounding is amplified by the coarse condition number); FP32/BF16 paths are
compared against the oracle evaluated on the same BF16-rounded density, with FP32
tolerances; whole FGMRES solves to +-1 iteration and 1e-6 relative on the history
(the cross-platform agreement the paper reports, Sec. 4.5.2), and every GPU
solution is re-checked by the oracle's own FP64 guard.
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


def bf16_round(x):
    return torch.as_tensor(x).to(torch.bfloat16).to(torch.float64).numpy()


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


GRIDS = [(16, 8, 8, 3), (24, 10, 6, 2), (2, 2, 2, 1), (1, 2, 2, 1), (38, 6, 4, 2), (8, 4, 4, 3)]


def make(gf, nx, ny, nz, L, seed=0, rho_min=1e-3, p=3.0, kind="uniform"):
    if kind == "uniform":
        rho = synth.uniform_density(nx, ny, nz, seed)
    elif kind == "bernoulli":
        rho = synth.bernoulli_density(nx, ny, nz, seed, 0.35)
    else:
        rho = synth.smoothed_gaussian_density(nx, ny, nz, seed)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), p)
    g.set_floor(rho_min)
    m = O.Mesh(nx, ny, nz)
    return g, m, rho


# ------------------------------------------------------------- a1: integer work --
@pytest.mark.parametrize("nx,ny,nz,L", GRIDS)
def test_load_and_mask_bit_exact(gf, nx, ny, nz, L):
    g = gf.create_grid(nx, ny, nz, levels=L)
    m = O.Mesh(nx, ny, nz)
    f = torch.full((g.n_dof,), 7.0, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    assert np.array_equal(host(f), O.cantilever_load(m))
    mask = torch.zeros(g.n_dof, dtype=torch.uint8, device="cuda")
    g.free_mask(mask)
    assert np.array_equal(mask.cpu().numpy().astype(bool), m.free)
    assert (g.n_dof, g.n_elem, g.n_nodes) == (m.n_dof, m.n_elem, m.n_nodes)


# ------------------------------------------------------------- a4: K*u ----------
@pytest.mark.parametrize("nx,ny,nz,L", GRIDS)
@pytest.mark.parametrize("p", [3.0, 4.5])
def test_apply_K_fp64_parity(gf, nx, ny, nz, L, p):
    g, m, rho = make(gf, nx, ny, nz, L, seed=nx, p=p)
    u = synth.random_vector(m.n_dof, 11)
    y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
    g.apply_K(dev(u), y)
    E = O.young_modulus(rho, 1e-3, p)
    ref = O.apply_K(m, E, O.element_stiffness(), u)
    got = host(y)
    assert relerr(got, ref) <= 1e-10
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.all(got[m.fixed] == 0.0)


@pytest.mark.parametrize("nx,ny,nz,L", GRIDS[:3] + GRIDS[4:5])
@pytest.mark.parametrize("variant", [256, 0, -128])
def test_apply_K_f32_parity(gf, nx, ny, nz, L, variant):
    g, m, rho = make(gf, nx, ny, nz, L, seed=3)
    g.set_stencil_blocks(256, variant)        # linear / shared-memory tiled / 27-neighbour gather
    u = synth.random_vector(m.n_dof, 5).astype(np.float32)
    y = torch.zeros(g.n_dof, dtype=torch.float32, device="cuda")
    g.apply_K_f32(dev(u, torch.float32), y)
    E = O.young_modulus(bf16_round(rho), 1e-3, 3.0)
    ref = O.apply_K(m, E, O.element_stiffness(), u.astype(np.float64))
    assert relerr(host(y), ref) <= 2e-5


def test_apply_K_linear_and_symmetric_on_gpu(gf):
    g, m, rho = make(gf, 12, 6, 6, 2, seed=1)
    a, b = synth.random_vector(m.n_dof, 1), synth.random_vector(m.n_dof, 2)
    ya, yb, yab = (torch.zeros(g.n_dof, dtype=torch.float64, device="cuda") for _ in range(3))
    g.apply_K(dev(a), ya)
    g.apply_K(dev(b), yb)
    g.apply_K(dev(2 * a - b), yab)
    A, B, AB = host(ya), host(yb), host(yab)
    assert relerr(AB, 2 * A - B) < 1e-13
    am, bm = np.where(m.fixed, 0, a), np.where(m.fixed, 0, b)
    assert abs(am @ B - bm @ A) < 1e-12 * np.linalg.norm(A) * np.linalg.norm(b)


# ------------------------------------------------------------- a5: V-cycle ------
@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (24, 12, 8, 3), (8, 4, 4, 2), (2, 2, 2, 1)])
def test_vcycle_fp64_parity(gf, nx, ny, nz, L):
    g, m, rho = make(gf, nx, ny, nz, L, seed=2)
    E = O.young_modulus(rho, 1e-3, 3.0)
    H = O.build_hierarchy(m, E, L)
    v = synth.random_vector(m.n_dof, 9)
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64)
    vm = np.where(m.fixed, 0, v)
    ref = O.vcycle(H, vm)
    assert relerr(host(z), ref) <= 1e-9


def test_vcycle_mixed_parity(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=2)
    # the mixed V-cycle builds its level moduli from the BF16 density in FP32; its
    # coarsest inverse comes from the FP64 moduli
    E16 = O.young_modulus(bf16_round(rho), 1e-3, 3.0)
    H = O.build_hierarchy(m, E16, L)
    H64 = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L)
    H.levels[-1].chol = H64.levels[-1].chol
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_MIXED)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-4


# ----------------------------------------------- FP32 node stencil with paired FMAs --
# The default FP32 node stencil advances the x and y output chains of each element with
# one paired FMA; GF_F32X2=0 selects the scalar kernel. Every chain keeps the scalar
# kernel's order and the node-block update is written out in explicit FMAs, so K*u, the
# V-cycle and a whole mixed solve are bit-identical between the two.
@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (38, 6, 4, 2), (52, 24, 20, 3)])
def test_paired_fma_stencil_bit_identical(gf, nx, ny, nz, L, monkeypatch):
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("GF_F32X2", flag)
        g, m, rho = make(gf, nx, ny, nz, L, seed=6, rho_min=1e-6)
        u = synth.random_vector(m.n_dof, 8)
        yf = torch.full((g.n_dof,), np.nan, dtype=torch.float32, device="cuda")
        g.apply_K_f32(dev(u, torch.float32), yf)
        z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.vcycle(dev(np.where(m.fixed, 0, u)), z, gf.GF_MIXED)
        x = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        out = g.solve(dev(O.cantilever_load(m)), x, prec=gf.GF_MIXED, outer=2)
        outs.append((yf, z, x, out["iters"]))
    (a_y, a_z, a_x, a_it), (b_y, b_z, b_x, b_it) = outs
    assert relerr(host(a_y), O.apply_K(m, O.young_modulus(bf16_round(rho), 1e-6, 3.0),
                                       O.element_stiffness(), u.astype(np.float32).astype(np.float64))) <= 2e-5
    assert torch.equal(a_y, b_y) and torch.equal(a_z, b_z)
    assert a_it == b_it and torch.equal(a_x, b_x)


# ------------------------------------------------- FP32 stencil on the tensor cores --
# GF_STENCIL_TC=1 runs every FP32 level stencil as stencil_tc32_kernel (3xTF32 element
# products); 0 keeps the CUDA-core kernel. Grids span several 16x8-element tiles in x
# and y, ragged tiles, and z chunks of 4..16 node layers with a ragged last chunk.
TC_GRIDS = [(16, 8, 8, 3), (24, 10, 6, 2), (2, 2, 2, 1), (1, 2, 2, 1), (38, 6, 4, 2), (52, 24, 20, 3)]


@pytest.mark.parametrize("nx,ny,nz,L", TC_GRIDS)
def test_apply_K_f32_tensor_core_parity(gf, nx, ny, nz, L, monkeypatch):
    monkeypatch.setenv("GF_STENCIL_TC", "1")
    g, m, rho = make(gf, nx, ny, nz, L, seed=3)
    monkeypatch.setenv("GF_STENCIL_TC", "0")
    g0, _, _ = make(gf, nx, ny, nz, L, seed=3)
    u = synth.random_vector(m.n_dof, 5).astype(np.float32)
    y, y0 = (torch.full((g.n_dof,), np.nan, dtype=torch.float32, device="cuda") for _ in range(2))
    g.apply_K_f32(dev(u, torch.float32), y)
    g0.apply_K_f32(dev(u, torch.float32), y0)
    E = O.young_modulus(bf16_round(rho), 1e-3, 3.0)
    ref = O.apply_K(m, E, O.element_stiffness(), u.astype(np.float64))
    got = host(y)
    assert relerr(got, ref) <= 2e-5
    assert np.all(got[m.fixed] == 0.0)
    # within 3xTF32 rounding of the CUDA-core kernel, and not the same kernel
    absref = O.apply_K(m, E, np.abs(O.element_stiffness()), np.abs(u.astype(np.float64)))
    assert np.linalg.norm(got - host(y0)) <= 2e-6 * np.linalg.norm(absref)
    if m.n_dof > 3000:
        assert not np.array_equal(got, host(y0))


@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (52, 24, 20, 3)])
def test_vcycle_mixed_tensor_core_parity(gf, nx, ny, nz, L, monkeypatch):
    monkeypatch.setenv("GF_STENCIL_TC", "1")
    g, m, rho = make(gf, nx, ny, nz, L, seed=2)
    E16 = O.young_modulus(bf16_round(rho), 1e-3, 3.0)
    H64 = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    for nu in (1, 2, 3):
        H = O.build_hierarchy(m, E16, L, nu1=nu, nu2=nu)
        H.levels[-1].chol = H64.levels[-1].chol
        z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.vcycle(dev(v), z, gf.GF_MIXED, nu1=nu, nu2=nu)
        assert relerr(host(z), O.vcycle(H, v)) <= 1e-4


def test_solve_mixed_tensor_core_stencil(gf, monkeypatch):
    # the mixed solve with every FP32 stencil on the tensor cores reaches the FP64
    # oracle's iteration count (within one) and an accepted true residual
    nx, ny, nz, L = 16, 8, 8, 3
    res = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("GF_STENCIL_TC", tc)
        g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=1e-6, kind="uniform")
        f = O.cantilever_load(m)
        u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        res[tc] = (g.solve(dev(f), u, prec=gf.GF_MIXED, outer=2), host(u))
    a, b = res["1"][0], res["0"][0]
    assert a["flag"] == b["flag"] == gf.GF_FLAG_CONVERGED and abs(a["iters"] - b["iters"]) <= 1
    E = O.young_modulus(rho, 1e-6, 3.0)
    assert O.true_residual(m, E, O.element_stiffness(), f, res["1"][1]) <= 1.5e-6


# -------------------------------------------- line-searched coarse correction --
# gf_solve_opts.ls_ratio = theta: every level's coarse correction scaled by the
# energy-optimal alpha = (c.r)/(c.Kc) and kept only if alpha >= theta (theta 1e30
# rejects all corrections: the V-cycle is then smoothing only).
@pytest.mark.parametrize("theta", [0.1, 0.9, 1e30])
@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (24, 10, 6, 2), (8, 4, 4, 3)])
def test_vcycle_line_search_fp64_parity(gf, nx, ny, nz, L, theta):
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, kind="bernoulli")
    E = O.young_modulus(rho, 1e-3, 3.0)
    H = O.build_hierarchy(m, E, L, ls_ratio=theta)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64, ls_ratio=theta)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-10


def test_vcycle_line_search_mixed_parity(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, kind="bernoulli")
    H = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L, ls_ratio=0.1)
    H.levels[-1].chol = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L).levels[-1].chol
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_MIXED, ls_ratio=0.1)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-4


def test_solve_line_search_fp64_parity(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=43, rho_min=1e-6, kind="bernoulli")
    E = O.young_modulus(rho, 1e-6, 3.0)
    f = O.cantilever_load(m)
    ref = O.solve_at_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L, ls_ratio=0.1), f, 1e-6, 120, 1e-6)[0]
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, kmax=120, prec=gf.GF_FP64, ls_ratio=0.1)
    assert abs(out["iters"] - ref.iters) <= 1 and out["flag"] == ref.flag
    h = min(out["iters"], ref.iters)
    assert np.allclose(out["history"][:h], ref.history[:h], rtol=1e-6)
    for prec, outer in ((gf.GF_MIXED, 2), (gf.GF_FP64, 0)):   # mixed runs the tiled V-cycle, captured graphs
        u.zero_()
        o2 = g.solve(dev(f), u, kmax=120, prec=prec, outer=outer, ls_ratio=0.1)
        if o2["flag"] == gf.GF_FLAG_CONVERGED:
            assert O.true_residual(m, E, O.element_stiffness(), f, host(u)) <= 1.5e-6


def test_line_search_arguments(gf):
    g, m, rho = make(gf, 8, 4, 4, 2, seed=1)
    f = dev(O.cantilever_load(m))
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    for kw in (dict(ls_ratio=float("inf")), dict(ls_ratio=-0.1), dict(ls_ratio=0.9, smoother=1)):
        with pytest.raises(gf.GFError):
            g.solve(f, u, kmax=5, **kw)
    g1, m1, _ = make(gf, 4, 2, 2, 1, seed=1)
    with pytest.raises(gf.GFError):
        g1.solve(dev(O.cantilever_load(m1)), torch.zeros(g1.n_dof, dtype=torch.float64, device="cuda"),
                 kmax=5, ls_ratio=0.9)


# ---------------------------------------------- fine-level adaptive correction --
# gf_solve_opts.fine_steps = k: after the V-cycle, k steps of an inner FGMRES(k) with the
# node-block Jacobi operator on the fine-level residual equation, applied only if the
# recomputed residual norm drops (oracle precondition()).
@pytest.mark.parametrize("steps", [1, 5, 20])
@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (8, 4, 4, 3)])
def test_fine_correction_fp64_parity(gf, nx, ny, nz, L, steps):
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, kind="bernoulli")
    H = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L, fine_steps=steps)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64, fine_steps=steps)
    ref = O.precondition(H, v)
    assert relerr(host(z), ref) <= 1e-9
    assert not np.allclose(ref, O.vcycle(H, v))                 # the correction took effect


def test_fine_correction_mixed_lowers_the_residual(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, kind="bernoulli")
    E = O.young_modulus(rho, 1e-3, 3.0)
    H = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L, fine_steps=20)
    H.levels[-1].chol = O.build_hierarchy(m, E, L).levels[-1].chol
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z0, z1 = (torch.zeros(g.n_dof, dtype=torch.float64, device="cuda") for _ in range(2))
    g.vcycle(dev(v), z0, gf.GF_MIXED)
    g.vcycle(dev(v), z1, gf.GF_MIXED, fine_steps=20)
    K0 = O.element_stiffness()
    r0 = np.linalg.norm(v - O.apply_K(m, E, K0, host(z0)))
    r1 = np.linalg.norm(v - O.apply_K(m, E, K0, host(z1)))
    assert r1 < 0.5 * r0
    assert relerr(host(z1), O.precondition(H, v)) <= 1e-3


def test_solve_fine_correction_fp64_parity(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=43, rho_min=1e-3, kind="bernoulli")
    f = O.cantilever_load(m)
    ref = O.solve_at_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L, fine_steps=20), f, 1e-3, 120, 1e-6)[0]
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, kmax=120, prec=gf.GF_FP64, fine_steps=20)
    assert abs(out["iters"] - ref.iters) <= 1 and out["flag"] == ref.flag == gf.GF_FLAG_CONVERGED
    h = min(out["iters"], ref.iters)
    assert np.allclose(out["history"][:h], ref.history[:h], rtol=1e-6)
    plain = g.solve(dev(f), torch.zeros_like(u), kmax=120, prec=gf.GF_FP64)
    assert out["iters"] < plain["iters"]
    u2 = torch.zeros_like(u)                       # mixed, captured graphs
    o2 = g.solve(dev(f), u2, kmax=120, prec=gf.GF_MIXED, outer=2, fine_steps=20)
    assert o2["flag"] == gf.GF_FLAG_CONVERGED and abs(o2["iters"] - ref.iters) <= 3
    E = O.young_modulus(rho, 1e-3, 3.0)
    assert O.true_residual(m, E, O.element_stiffness(), f, host(u2)) <= 1.5e-6


def test_fine_correction_arguments(gf):
    g, m, rho = make(gf, 8, 4, 4, 2, seed=1)
    f = dev(O.cantilever_load(m))
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    for k in (-1, 33):
        with pytest.raises(gf.GFError):
            g.solve(f, u, kmax=5, fine_steps=k)


# ------------------------------------------------------------- Chebyshev smoother --
@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (24, 10, 6, 2), (8, 4, 4, 3)])
def test_chebyshev_lambda_and_vcycle_fp64_parity(gf, nx, ny, nz, L):
    g, m, rho = make(gf, nx, ny, nz, L, seed=2)
    E = O.young_modulus(rho, 1e-3, 3.0)
    H = O.build_hierarchy(m, E, L, smoother="chebyshev")
    lam = g.chebyshev_lambda(gf.GF_FP64)
    ref = [lev.lam for lev in H.levels[:-1]]
    assert len(lam) == L - 1
    assert np.allclose(lam, ref, rtol=1e-10, atol=0)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    for rep in range(2):   # the second call reuses the bounds
        z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.vcycle(dev(v), z, gf.GF_FP64, smoother=1)
        assert relerr(host(z), O.vcycle(H, v)) <= 1e-9
    # a new floor recomputes the bounds
    g.set_floor(1e-6)
    H6 = O.build_hierarchy(m, O.young_modulus(rho, 1e-6, 3.0), L, smoother="chebyshev")
    assert np.allclose(g.chebyshev_lambda(gf.GF_FP64), [lev.lam for lev in H6.levels[:-1]], rtol=1e-10, atol=0)


def test_chebyshev_vcycle_mixed_parity(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=2)
    E16 = O.young_modulus(bf16_round(rho), 1e-3, 3.0)
    H = O.build_hierarchy(m, E16, L, smoother="chebyshev")
    H64 = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L)
    H.levels[-1].chol = H64.levels[-1].chol
    lam = g.chebyshev_lambda(gf.GF_MIXED)
    assert np.allclose(lam, [lev.lam for lev in H.levels[:-1]], rtol=1e-5, atol=0)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_MIXED, smoother=1)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-4


@pytest.mark.parametrize("case", [(16, 8, 8, 3, "uniform", 1e-3), (16, 8, 8, 3, "bernoulli", 1e-6)])
def test_solve_chebyshev_fp64_parity(gf, case):
    nx, ny, nz, L, kind, rm = case
    g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=rm, kind=kind)
    f = O.cantilever_load(m)
    setup = O.SolverSetup(m, rho, p=3.0, n_levels=L, restart=30, smoother="chebyshev")
    res, E, K0 = O.solve_at_floor(setup, f, rm, 200, 1e-6)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, restart=30, kmax=200, tol=1e-6, prec=gf.GF_FP64, smoother=1)
    assert abs(out["iters"] - res.iters) <= 1 and out["flag"] == res.flag
    k = min(out["iters"], res.iters)
    h_gpu, h_ref = np.array(out["history"][:k + 1]), res.history[:k + 1]
    assert np.all(np.abs(h_gpu - h_ref) <= 1e-6 * h_ref + 1e-15)
    if res.flag == O.CONVERGED:
        assert O.true_residual(m, E, K0, f, host(u)) <= 1.5e-6


def test_solve_chebyshev_mixed_converges(gf):
    """The mixed form (FP32 Chebyshev V-cycle, FP64-class Krylov) converges in about the
    oracle's FP64 iteration count (59 here) and passes the oracle's guard."""
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=1e-3, kind="bernoulli")
    f = O.cantilever_load(m)
    res, E, K0 = O.solve_at_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L, smoother="chebyshev"), f, 1e-3, 200,
                                  1e-6)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, prec=gf.GF_MIXED, outer=2, smoother=1)
    assert out["flag"] == gf.GF_FLAG_CONVERGED and res.flag == O.CONVERGED
    assert abs(out["iters"] - res.iters) <= max(2, res.iters // 10)
    assert O.true_residual(m, E, K0, f, host(u)) <= 1.5e-6


# ------------------------------------------------------------- a6/a7: solve ------
def _oracle_solve(m, rho, rho_min, L, f, kmax=200, restart=30, tol=1e-6):
    setup = O.SolverSetup(m, rho, p=3.0, n_levels=L, restart=restart)
    return O.solve_at_floor(setup, f, rho_min, kmax, tol)


# outer = 2 runs the same FP64 V-cycle with the FP64-class forms of the Krylov
# operator (split-integer K*u) and of CGS2 (double-float passes): the oracle's FP64
# history must still be matched to the same tolerance.
@pytest.mark.parametrize("outer", [0, 2])
@pytest.mark.parametrize("case", [(16, 8, 8, 3, "uniform", 1e-3, 30), (16, 8, 8, 3, "bernoulli", 1e-6, 30),
                                  (24, 12, 8, 3, "smooth", 1e-3, 8)])
def test_solve_fp64_parity(gf, case, outer):
    nx, ny, nz, L, kind, rm, restart = case
    g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=rm, kind=kind)
    f = O.cantilever_load(m)
    res, E, K0 = _oracle_solve(m, rho, rm, L, f, restart=restart)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, restart=restart, kmax=200, tol=1e-6, prec=gf.GF_FP64, outer=outer)
    assert abs(out["iters"] - res.iters) <= 1
    assert out["flag"] == res.flag
    k = min(out["iters"], res.iters)
    h_gpu, h_ref = np.array(out["history"][:k + 1]), res.history[:k + 1]
    assert np.all(np.abs(h_gpu - h_ref) <= 1e-6 * h_ref + 1e-15)
    # the oracle's own guard on the GPU's solution, and the GPU guard against it. At a
    # converged u, f - K u cancels: a 1e-10 relative error in K u moves eta by up to
    # 1e-10 * ||K u|| / ||f||, so that is the bound (not 1e-10 * eta).
    uh = host(u)
    eta_oracle = O.true_residual(m, E, K0, f, uh)
    eta_gpu = g.true_residual(dev(f), u)
    if res.flag == O.CONVERGED:
        assert eta_oracle <= 1.5e-6
    ku = np.linalg.norm(O.apply_K(m, E, K0, uh))
    assert abs(eta_gpu - eta_oracle) <= 1e-10 * ku / np.linalg.norm(f)


# Restarts above 32 basis vectors: the Gram-Schmidt passes run over slices of 32
# vectors (FP64 for outer 0 and 1, double-float for outer 2). The Bernoulli state needs
# 148 steps at restart 45 (cycles whose bases end in a ragged slice) and 99 / 122 at
# restart 300 (one cycle, four slices), so the histories are matched well past the
# fused passes' 32 vectors.
@pytest.mark.parametrize("outer", [0, 1, 2])
@pytest.mark.parametrize("case", [(16, 8, 8, 3, 45), (16, 8, 8, 3, 300), (24, 12, 8, 3, 300)])
def test_solve_long_restart_parity(gf, case, outer):
    nx, ny, nz, L, restart = case
    g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=1e-6, kind="bernoulli")
    f = O.cantilever_load(m)
    res, E, K0 = _oracle_solve(m, rho, 1e-6, L, f, restart=restart)
    assert res.iters > 2 * 32 and res.flag == O.CONVERGED
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, restart=restart, kmax=200, tol=1e-6, prec=gf.GF_FP64, outer=outer)
    assert abs(out["iters"] - res.iters) <= 1 and out["flag"] == res.flag
    k = min(out["iters"], res.iters)
    h_gpu, h_ref = np.array(out["history"][:k + 1]), res.history[:k + 1]
    # outer 1 and 2: the split-integer operator is exact to ~2^-48 relative (and the
    # double-float passes to ~2^-47), not FP64's 2^-53; over ~150 slowly converging steps
    # on this kappa ~ 1e10 state the histories then part by up to ~1e-12 absolute
    # (measured for outer 1: 1.6e-14 at step 1, 1e-12 near the stop)
    atol = 1e-15 if outer == 0 else 2e-12
    assert np.all(np.abs(h_gpu - h_ref) <= 1e-6 * h_ref + atol)
    assert O.true_residual(m, E, K0, f, host(u)) <= 1.5e-6


def test_long_restart_limits(gf):
    g, m, _ = make(gf, 8, 4, 4, 2, seed=1)
    f, u = dev(O.cantilever_load(m)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    for kw in (dict(restart=301), dict(restart=301, outer=2), dict(restart=0)):
        with pytest.raises(gf.GFError):
            g.solve(f, u, **kw)
    for outer in (1, 2):
        assert g.solve(f, u, restart=300, outer=outer, kmax=40)["flag"] in (gf.GF_FLAG_CONVERGED,
                                                                          gf.GF_FLAG_MAX_ITERS)


# ------------------------------------------------ coarse-level inner Krylov solve --
# coarse_steps = k replaces the coarsest level's dense inverse by k steps of an inner
# FGMRES(k) from 0, preconditioned by the coarsest level's node-block Jacobi operator
# (Table solver-config's inner Krylov steps on the coarse level), on the device.
@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (24, 10, 6, 2), (32, 16, 16, 4)])
@pytest.mark.parametrize("k", [1, 10])
def test_vcycle_coarse_krylov_fp64_parity(gf, nx, ny, nz, L, k):
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, rho_min=1e-3, kind="bernoulli")
    H = O.build_hierarchy(m, O.young_modulus(rho, 1e-3, 3.0), L, coarse_steps=k)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_FP64, coarse_steps=k)
    ref = O.vcycle(H, v)
    assert relerr(host(z), ref) <= 1e-9
    z0 = torch.zeros_like(z)
    g.vcycle(dev(v), z0, gf.GF_FP64)                     # the exact coarse solve differs
    assert relerr(host(z0), ref) > 1e-6


def test_vcycle_coarse_krylov_mixed_parity(gf):
    # FP32 levels from the BF16 density; the coarse inner solve accumulates its Gram-
    # Schmidt dots per thread in FP32 (block and grid sums in FP64), so its solution
    # carries FP32 rounding amplified by the coarse operator's conditioning
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=2, rho_min=1e-3)
    H = O.build_hierarchy(m, O.young_modulus(bf16_round(rho), 1e-3, 3.0), L, coarse_steps=10)
    v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
    z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.vcycle(dev(v), z, gf.GF_MIXED, coarse_steps=10)
    assert relerr(host(z), O.vcycle(H, v)) <= 1e-3


@pytest.mark.parametrize("nx,ny,nz,L", [(16, 8, 8, 3), (32, 16, 16, 4), (24, 10, 6, 2)])
def test_coarse_krylov_one_cta_matches_multi_launch(gf, nx, ny, nz, L, monkeypatch):
    # the default one-CTA coarse solve (coarse_fgmres_kernel) against the multi-launch
    # inner solve (GF_COARSE_FUSED=0): the same steps, sums in another order
    for prec, tol in ((gf.GF_FP64, 1e-11), (gf.GF_MIXED, 1e-4)):
        zs = []
        for fused in ("1", "0"):
            monkeypatch.setenv("GF_COARSE_FUSED", fused)
            g, m, rho = make(gf, nx, ny, nz, L, seed=3, rho_min=1e-3, kind="bernoulli")
            v = np.where(m.fixed, 0, synth.random_vector(m.n_dof, 9))
            z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
            g.vcycle(dev(v), z, prec, coarse_steps=10)
            zs.append(host(z))
            g.close()
        assert relerr(zs[0], zs[1]) <= tol


@pytest.mark.parametrize("kind,rho_min", [("bernoulli", 1e-3), ("gauss", 1e-6)])
def test_solve_coarse_krylov_fp64_parity(gf, kind, rho_min):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=rho_min, kind=kind)
    f = O.cantilever_load(m)
    res, E, K0 = O.solve_at_floor(O.SolverSetup(m, rho, p=3.0, n_levels=L, coarse_steps=10), f, rho_min, 200, 1e-6)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, restart=30, kmax=200, tol=1e-6, prec=gf.GF_FP64, coarse_steps=10)
    assert abs(out["iters"] - res.iters) <= 1 and out["flag"] == res.flag
    k = min(out["iters"], res.iters)
    h_gpu, h_ref = np.array(out["history"][:k + 1]), res.history[:k + 1]
    assert np.all(np.abs(h_gpu - h_ref) <= 1e-6 * h_ref + 1e-15)
    if res.flag == O.CONVERGED:
        assert O.true_residual(m, E, K0, f, host(u)) <= 1.5e-6
    with pytest.raises(gf.GFError):
        g.solve(dev(f), u, coarse_steps=33)
    mixed = g.solve(dev(f), u.zero_(), prec=gf.GF_MIXED, outer=2, coarse_steps=10, fine_steps=5, kmax=200)
    assert mixed["flag"] == gf.GF_FLAG_CONVERGED


def test_solve_mixed_converges_and_guard(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=0, rho_min=1e-3)
    f = O.cantilever_load(m)
    res, E, K0 = _oracle_solve(m, rho, 1e-3, L, f)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(dev(f), u, prec=gf.GF_MIXED)
    assert out["flag"] == gf.GF_FLAG_CONVERGED and abs(out["iters"] - res.iters) <= 2
    eta = O.true_residual(m, E, K0, f, host(u))
    assert eta <= 1.5e-6
    # error against the FP64 oracle solution: u, compliance, sensitivity (measured ~1e-12 to
    # 2e-11: the residual left at the stop is high-frequency, which K^{-1} damps)
    ug, ur = host(u), res.x
    assert np.linalg.norm(ug - ur) <= 1e-4 * np.linalg.norm(ur)
    assert abs(f @ ug - f @ ur) <= 1e-5 * abs(f @ ur)
    dc = torch.zeros(g.n_elem, dtype=torch.float64, device="cuda")
    g.sensitivity(u, dc)
    sr = O.sensitivity(m, rho, 1e-3, 3.0, K0, ur)
    assert np.linalg.norm(host(dc) - sr) <= 1e-6 * np.linalg.norm(sr)


def test_true_residual_parity_and_one_apply(gf):
    g, m, rho = make(gf, 16, 8, 8, 3, seed=1)
    f = O.cantilever_load(m)
    u = synth.random_vector(m.n_dof, 3) * 1e-2
    E = O.young_modulus(rho, 1e-3, 3.0)
    g.reset_stats()
    eta = g.true_residual(dev(f), dev(u))
    assert g.stats()["apply_K_fp64"] == 1     # the guard costs exactly one operator application
    ref = O.true_residual(m, E, O.element_stiffness(), f, u)
    assert abs(eta - ref) <= 1e-12 * ref
    assert g.true_residual(dev(f), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")) == 1.0


def test_solve_edge_cases(gf):
    g, m, rho = make(gf, 8, 4, 4, 2, seed=1)
    f = dev(O.cantilever_load(m))
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.solve(f, u, kmax=0)
    assert out["iters"] == 0 and out["flag"] == gf.GF_FLAG_MAX_ITERS and out["history"] == [1.0]
    assert torch.all(u == 0)
    out = g.solve(f, u, restart=1, kmax=5)          # restart every step
    assert out["iters"] == 5 and out["flag"] == gf.GF_FLAG_MAX_ITERS
    ref = O.SolverSetup(m, rho, p=3.0, n_levels=2, restart=1)
    r, _, _ = O.solve_at_floor(ref, O.cantilever_load(m), 1e-3, 5, 1e-6)
    assert np.allclose(out["history"], r.history, rtol=1e-8)
    # restart from the previous iterate: history[0] is its true residual
    eta0 = g.true_residual(f, u)
    out2 = g.solve(f, u, restart=30, kmax=3)
    assert abs(out2["history"][0] - eta0) <= 1e-12 * eta0


def test_errors(gf):
    with pytest.raises(gf.GFError):
        gf.create_grid(16, 7, 8, levels=1)           # odd ny
    with pytest.raises(gf.GFError):
        gf.create_grid(12, 8, 8, levels=4)           # not divisible
    g = gf.create_grid(4, 2, 2, levels=1)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(gf.GFError) as e:
        g.apply_K(u, u.clone())
    assert e.value.code == -6                         # GF_ERR_STATE
    bad = np.full(g.n_elem, 0.5)
    bad[3] = np.nan
    with pytest.raises(gf.GFError) as e:
        g.set_density(dev(bad), 3.0)
    assert e.value.code == -4                         # GF_ERR_NONFINITE
    bad[3] = 1.5
    with pytest.raises(gf.GFError):
        g.set_density(dev(bad), 3.0)
    with pytest.raises(TypeError):
        g.set_density(dev(np.ones(g.n_elem), torch.float32), 3.0)
    g.set_density(dev(np.full(g.n_elem, 0.5)), 3.0)
    g.set_floor(1e-3)
    for outer in (-1, 3):                             # Krylov operator form out of range
        with pytest.raises(gf.GFError) as e:
            g.solve(u.clone(), u.clone(), outer=outer)
        assert e.value.code == -1                     # GF_ERR_ARG
    for smoother in (-1, 2):                          # smoother out of range
        with pytest.raises(gf.GFError) as e:
            g.solve(u.clone(), u.clone(), smoother=smoother)
        assert e.value.code == -1


# ------------------------------------------------------------- reuse selector ------
@pytest.mark.parametrize("seed,q", [(43, 0.35), (47, 0.30)])
@pytest.mark.parametrize("first", [0, 2])
def test_reuse_selector_matches_oracle(gf, seed, q, first):
    """GF_SEL_REUSE: the previous decision without a probe, Algorithm 1 from scratch when
    the guard rejects it. Same attempts (floor, accepted) and outcome as the oracle."""
    nx, ny, nz = 16, 8, 8
    m = O.Mesh(nx, ny, nz)
    rho = synth.bernoulli_density(nx, ny, nz, seed, q)
    f = O.cantilever_load(m)
    ladder = [1e-5, 1e-4, 1e-3]
    ref = O.select_floor(O.SolverSetup(m, rho, p=3.0, n_levels=3), f, 1e-8, ladder, kmax=120,
                         selector="reuse", first_index=first)
    g = gf.create_grid(nx, ny, nz, levels=3)
    g.set_density(dev(rho), 3.0)
    pol = gf.policy_defaults(rho0=1e-8, ladder=ladder, kmax=120, selector=gf.GF_SEL_REUSE, first_index=first,
                             solve_prec=gf.GF_FP64)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.select_floor(dev(f), u, pol)
    assert out["status"] == ref.status and out["floor_index"] == ref.floor_index
    assert [(a["rho_min"], bool(a["accepted"])) for a in out["attempts"]] == \
        [(a.rho_min, bool(a.accepted)) for a in ref.attempts]
    for a, b in zip(out["attempts"], ref.attempts):
        assert abs(a["iters"] - b.iters) <= 1
    if ref.status == O.ACCEPTED:
        E = O.young_modulus(rho, out["rho_min"], 3.0)
        assert O.true_residual(m, E, O.element_stiffness(), f, host(u)) <= 1e-6 * (1 + 1e-9)


# Periodic true-residual checks during the probe and their detector (Sec. 4.1.1's
# untested checkpointed variant; the detector rule is a reading). ratio 10: the estimate
# tracks the residual, nothing fires; ratio 0.5: every check fires, the probe escalates.
@pytest.mark.parametrize("fuse", [1, 0])
@pytest.mark.parametrize("ratio", [10.0, 0.5])
def test_true_checks_match_oracle(gf, ratio, fuse):
    nx, ny, nz = 16, 8, 8
    m = O.Mesh(nx, ny, nz)
    rho = synth.bernoulli_density(nx, ny, nz, 43, 0.35)
    f = O.cantilever_load(m)
    ladder = [1e-5, 1e-4, 1e-3]
    ref = O.select_floor(O.SolverSetup(m, rho, p=3.0, n_levels=3), f, 1e-8, ladder, kmax=120,
                         probe_iters=60, true_check_every=7, true_check_ratio=ratio)
    g = gf.create_grid(nx, ny, nz, levels=3)
    g.set_density(dev(rho), 3.0)
    pol = gf.policy_defaults(rho0=1e-8, ladder=ladder, kmax=120, probe_iters=60, true_check_every=7,
                             true_check_ratio=ratio, fuse_probe=fuse, solve_prec=gf.GF_FP64)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.select_floor(dev(f), u, pol)
    assert [c[0] for c in out["true_checks"]] == [c[0] for c in ref.checks] and len(ref.checks) >= 3
    for (k, est, eta), (_, est_r, eta_r) in zip(out["true_checks"], ref.checks):
        assert abs(est - est_r) <= 1e-6 * est_r and abs(eta - eta_r) <= 1e-6 * eta_r
    assert out["true_check_fired"] == ref.detector == (ratio < 1)
    assert out["escalated"] == ref.escalated and out["floor_index"] == ref.floor_index
    assert [(a["rho_min"], bool(a["accepted"])) for a in out["attempts"]] == \
        [(a.rho_min, bool(a.accepted)) for a in ref.attempts]


def test_true_checks_leave_the_solve_unchanged(gf):
    """Checks only read the state: the accepted iterate is bit-identical with and without them."""
    nx, ny, nz = 16, 8, 8
    rho = synth.bernoulli_density(nx, ny, nz, 47, 0.30)
    f = dev(O.cantilever_load(O.Mesh(nx, ny, nz)))
    outs = []
    for every in (0, 9):
        g = gf.create_grid(nx, ny, nz, levels=3)
        g.set_density(dev(rho), 3.0)
        pol = gf.policy_defaults(rho0=1e-6, kmax=120, true_check_every=every, solve_prec=gf.GF_MIXED,
                                 solve_outer=2)
        u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        outs.append((g.select_floor(f, u, pol), u.clone()))
        g.close()
    (a, ua), (b, ub) = outs
    assert a["true_checks"] == [] and len(b["true_checks"]) >= 1 and not b["true_check_fired"]
    assert a["floor_index"] == b["floor_index"] and torch.equal(ua, ub)
    assert [x["iters"] for x in a["attempts"]] == [x["iters"] for x in b["attempts"]]


def test_true_check_arguments(gf):
    g = gf.create_grid(8, 4, 4, levels=2)
    g.set_density(dev(np.full(8 * 4 * 4, 0.5)), 3.0)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    u = torch.zeros_like(f)
    for kw in (dict(true_check_every=-1), dict(true_check_every=5, probe_iters=100),
               dict(true_check_every=10, true_check_ratio=0.0),
               dict(true_check_every=10, selector=gf.GF_SEL_FULL)):
        with pytest.raises(gf.GFError):
            g.select_floor(f, u, gf.policy_defaults(**kw))


# Floor-conditioning diagnostic (Sec. 4.1.3): extreme eigenvalues by Lanczos on K and on
# its dense inverse (one-level grid), against the oracle's dense eigensolver; the direct
# solution's guard residual within the backward-error envelope kappa * eps.
@pytest.mark.parametrize("nx,ny,nz,rm", [(4, 2, 2, 1e-3), (8, 4, 4, 1e-6), (6, 2, 2, 1e-8)])
def test_conditioning_matches_oracle(gf, nx, ny, nz, rm):
    m = O.Mesh(nx, ny, nz)
    rho = synth.bernoulli_density(nx, ny, nz, 43, 0.35)
    f = O.cantilever_load(m)
    lo, hi, eta = O.conditioning(m, O.young_modulus(rho, rm, 3.0), O.element_stiffness(), f)
    g = gf.create_grid(nx, ny, nz, levels=1)
    g.set_density(dev(rho), 3.0)
    g.set_floor(rm)
    out = g.conditioning(dev(f), iters=min(512, m.n_dof))
    kappa_eps = hi / lo * 2.0 ** -52
    assert abs(out["lambda_max"] / hi - 1) <= 1e-9
    assert abs(out["lambda_min"] / lo - 1) <= max(1e-7, 100 * kappa_eps)
    assert out["eta_direct"] <= 1e3 * kappa_eps + 1e-13 and eta <= 1e3 * kappa_eps + 1e-13
    assert gf.conditioning_screen(out["lambda_min"], out["lambda_max"], rm, 1e-6) == \
        pytest.approx(O.conditioning_screen(lo, hi, rm, 1e-6), rel=max(1e-6, 200 * kappa_eps))


def test_conditioning_arguments(gf):
    g = gf.create_grid(4, 2, 2, levels=2)
    g.set_density(dev(np.full(16, 0.5)), 3.0)
    g.set_floor(1e-3)
    with pytest.raises(gf.GFError):
        g.conditioning(iters=20)                  # needs levels == 1
    g1 = gf.create_grid(4, 2, 2, levels=1)
    g1.set_density(dev(np.full(16, 0.5)), 3.0)
    with pytest.raises(gf.GFError):
        g1.conditioning(iters=20)                 # before set_floor
    g1.set_floor(1e-3)
    for it in (1, 513):
        with pytest.raises(gf.GFError):
            g1.conditioning(iters=it)


# ------------------------------------------------------------- a8: policy --------
@pytest.mark.parametrize("seed,q", [(43, 0.35), (47, 0.30)])
def test_select_floor_parity(gf, seed, q):
    nx, ny, nz, L = 16, 8, 8, 3
    rho = synth.bernoulli_density(nx, ny, nz, seed, q)
    m = O.Mesh(nx, ny, nz)
    f = O.cantilever_load(m)
    setup = O.SolverSetup(m, rho, p=3.0, n_levels=L)
    ladder = [1e-5, 1e-4, 1e-3]
    ref = O.select_floor(setup, f, 1e-9, ladder, tau=1e-6, kmax=60, probe_iters=100)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), 3.0)
    pol = gf.policy_defaults(rho0=1e-9, ladder=ladder, kmax=60)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.select_floor(dev(f), u, pol)
    assert abs(out["r50"] - ref.r50) <= 1e-4 * ref.r50
    assert abs(out["r100"] - ref.r100) <= 1e-4 * ref.r100
    assert out["escalated"] == ref.escalated
    assert out["status"] == ref.status and out["floor_index"] == ref.floor_index
    assert len(out["attempts"]) == len(ref.attempts)
    for a, b in zip(out["attempts"], ref.attempts):
        assert a["rho_min"] == b.rho_min and abs(a["iters"] - b.iters) <= 1
        assert a["accepted"] == b.accepted
    if out["status"] == gf.GF_ACCEPTED:
        E = O.young_modulus(rho, out["rho_min"], 3.0)
        assert O.true_residual(m, E, O.element_stiffness(), f, host(u)) <= 1e-6 * (1 + 1e-9)


def test_select_floor_no_admissible(gf):
    nx, ny, nz, L = 8, 4, 4, 2
    rho = synth.bernoulli_density(nx, ny, nz, 1, 0.3)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), 3.0)
    f = dev(O.cantilever_load(O.Mesh(nx, ny, nz)))
    pol = gf.policy_defaults(rho0=1e-6, ladder=[1e-5], kmax=1, probe_iters=1, selector=gf.GF_SEL_FULL)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    out = g.select_floor(f, u, pol)
    assert out["status"] == gf.GF_NO_ADMISSIBLE_FLOOR and out["floor_index"] == -1
    assert len(out["attempts"]) == 2 and not any(a["accepted"] for a in out["attempts"])


# ------------------------------------------------------------- a12: sensitivity ---
def test_sensitivity_parity(gf):
    g, m, rho = make(gf, 12, 6, 6, 2, seed=5)
    u = synth.random_vector(m.n_dof, 4)
    dc = torch.zeros(g.n_elem, dtype=torch.float64, device="cuda")
    g.sensitivity(dev(u), dc)
    ref = O.sensitivity(m, rho, 1e-3, 3.0, O.element_stiffness(), u)
    assert relerr(host(dc), ref) <= 1e-10


# ------------------------------------------------------------- full-size samples --
@pytest.mark.parametrize("dims", [(96, 48, 48, 4), (192, 96, 96, 5)])
def test_full_size_apply_sampled(gf, dims):
    nx, ny, nz, L = dims
    rho = synth.smoothed_gaussian_density(nx, ny, nz, 0) if nx == 96 else synth.uniform_density(nx, ny, nz, 0)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), 3.0)
    g.set_floor(1e-6)
    u = synth.random_vector(g.n_dof, 1)
    y = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.apply_K(dev(u), y)
    ys = torch.zeros_like(y)
    g.apply_K_split(dev(u), ys)                 # the Krylov operator of the mixed form
    rng = np.random.default_rng(0)
    nodes = rng.choice(g.n_nodes, 300, replace=False)
    nodes[:3] = [0, g.n_nodes - 1, nx]          # corners / fixed face
    E = O.young_modulus(rho, 1e-6, 3.0)
    ref = _apply_at_nodes(nx, ny, nz, E, u, nodes)
    scale = np.abs(ref).max()
    for out in (y, ys):
        assert np.abs(host(out).reshape(-1, 3)[nodes] - ref).max() <= 1e-10 * scale
    # the FP32 V-cycle operator (BF16-stored densities) at the same nodes
    y32 = torch.zeros(g.n_dof, dtype=torch.float32, device="cuda")
    u32 = u.astype(np.float32)
    g.apply_K_f32(dev(u32, torch.float32), y32)
    ref32 = _apply_at_nodes(nx, ny, nz, O.young_modulus(bf16_round(rho), 1e-6, 3.0), u32.astype(np.float64), nodes)
    assert np.abs(host(y32).reshape(-1, 3)[nodes] - ref32).max() <= 2e-5 * np.abs(ref32).max()


@pytest.mark.parametrize("dims", [(96, 48, 48, 5), (192, 96, 96, 5)])
def test_full_size_guard_matches_oracle(gf, dims):
    """At the full sizes, in the bench's mixed configuration: the library's FP64 guard on
    the accepted solution equals the oracle's recomputed residual over every DOF."""
    nx, ny, nz, L = dims
    m = O.Mesh(nx, ny, nz)
    rho = synth.smoothed_gaussian_density(nx, ny, nz, 0)
    g = gf.create_grid(nx, ny, nz, levels=L)
    g.set_density(dev(rho), 3.0)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    u = torch.zeros_like(f)
    out = g.select_floor(f, u, gf.policy_defaults(solve_prec=gf.GF_MIXED, solve_outer=2))
    assert out["status"] == gf.GF_ACCEPTED
    eta_ref = O.true_residual(m, O.young_modulus(rho, out["rho_min"], 3.0), O.element_stiffness(), host(f), host(u))
    assert eta_ref <= 1e-6 * (1 + 1e-9) and abs(out["eta"] - eta_ref) <= 1e-8 * eta_ref


def _apply_at_nodes(nx, ny, nz, E, u, nodes):
    """Oracle K*u at sampled nodes on a big grid without building the full mesh arrays."""
    K0 = O.element_stiffness()
    out = np.zeros((len(nodes), 3))
    NX, NY = nx + 1, ny + 1
    for t, n in enumerate(nodes):
        i, j, k = n % NX, (n // NX) % NY, n // (NX * NY)
        if i == 0:
            continue
        acc = np.zeros(3)
        for a, (ox, oy, oz) in enumerate(O.LOCAL_NODES):
            ex, ey, ez = i - ox, j - oy, k - oz
            if not (0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz):
                continue
            e = ex + nx * (ey + ny * ez)
            ue = np.zeros(24)
            for b, (bx, by, bz) in enumerate(O.LOCAL_NODES):
                ni = ex + bx
                if ni == 0:
                    continue
                node = ni + NX * ((ey + by) + NY * (ez + bz))
                ue[3 * b:3 * b + 3] = u[3 * node:3 * node + 3]
            acc += E[e] * (K0[3 * a:3 * a + 3] @ ue)
        out[t] = acc
    return out


# ------------------------------------------------------------- fused probe, graphs --
@pytest.mark.parametrize("seed,q,rho0,kmax", [(43, 0.35, 1e-9, 60), (47, 0.30, 1e-9, 60), (1, 0.30, 1e-6, 200),
                                              (5, 0.20, 1e-9, 40)])
def test_fused_probe_bit_identical(gf, seed, q, rho0, kmax):
    """Reading r50/r100 off the running rho0 solve gives exactly the separate probe's
    decisions and the independent rho0 solve's iterate (Algorithm 1 unchanged)."""
    nx, ny, nz, L = 16, 8, 8, 3
    rho = dev(synth.bernoulli_density(nx, ny, nz, seed, q))
    f = dev(O.cantilever_load(O.Mesh(nx, ny, nz)))
    outs, us = [], []
    for fuse in (1, 0):
        g = gf.create_grid(nx, ny, nz, levels=L)
        g.set_density(rho, 3.0)
        pol = gf.policy_defaults(rho0=rho0, ladder=[1e-5, 1e-4, 1e-3], kmax=kmax, fuse_probe=fuse)
        u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        outs.append(g.select_floor(f, u, pol))
        us.append(u.clone())
    a, b = outs
    for key in ("status", "floor_index", "escalated", "r50", "r100", "eta"):
        assert a[key] == b[key] or (np.isnan(a[key]) and np.isnan(b[key])), key
    assert a["attempts"] == b["attempts"]
    assert torch.equal(us[0], us[1])


def test_graph_replay_bit_identical(gf, monkeypatch):
    nx, ny, nz, L = 16, 8, 8, 3
    rho = dev(synth.uniform_density(nx, ny, nz, 2))
    f = dev(O.cantilever_load(O.Mesh(nx, ny, nz)))
    res = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("GF_GRAPHS", graphs)
        g = gf.create_grid(nx, ny, nz, levels=L)
        g.set_density(rho, 3.0)
        g.set_floor(1e-3)
        u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        out = g.solve(f, u, restart=7, prec=gf.GF_MIXED)
        res.append((out, u.clone(), g.stats()))
    assert res[0][0] == res[1][0] and torch.equal(res[0][1], res[1][1])
    assert res[0][2]["kernel_launches"] == res[1][2]["kernel_launches"]


# ------------------------------------------------------------- split-integer K*u --
# tc = "1": element products on the tensor cores (default); "0": the CUDA-core kernel
@pytest.mark.parametrize("tc", ["1", "0"])
@pytest.mark.parametrize("nx,ny,nz,L", GRIDS)
def test_apply_K_split_parity(gf, nx, ny, nz, L, tc, monkeypatch):
    monkeypatch.setenv("GF_SPLIT_TC", tc)
    g, m, rho = make(gf, nx, ny, nz, L, seed=nx + 1, rho_min=1e-6)
    E = O.young_modulus(rho, 1e-6, 3.0)
    K0 = O.element_stiffness()
    for seed, wide in ((3, False), (4, True)):
        u = synth.random_vector(m.n_dof, seed)
        if wide:   # values spread over 16 orders of magnitude
            u = u * 10.0 ** (16.0 * synth.random_vector(m.n_dof, seed + 10))
        y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
        g.apply_K_split(dev(u), y)
        ref = O.apply_K(m, E, K0, u)
        got = host(y)
        absref = O.apply_K(m, E, np.abs(K0), np.abs(u))      # |K| |u|, the rounding scale
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(absref)
        if not wide:
            assert relerr(got, ref) <= 1e-12
        assert np.all(got[m.fixed] == 0.0)
        y64 = torch.zeros_like(y)
        g.apply_K(dev(u), y64)
        assert np.linalg.norm(got - host(y64)) <= 1e-12 * np.linalg.norm(absref)


def test_solve_with_split_outer_operator(gf):
    nx, ny, nz, L = 16, 8, 8, 3
    g, m, rho = make(gf, nx, ny, nz, L, seed=4, rho_min=1e-6, kind="uniform")
    f = O.cantilever_load(m)
    outs = []
    for outer in (0, 1, 2):
        u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        out = g.solve(dev(f), u, prec=gf.GF_MIXED, outer=outer)
        outs.append((out, host(u)))
    a, ua = outs[0]
    E = O.young_modulus(rho, 1e-6, 3.0)
    for b, ub in outs[1:]:
        assert abs(a["iters"] - b["iters"]) <= 1 and a["flag"] == b["flag"] == gf.GF_FLAG_CONVERGED
        h = min(a["iters"], b["iters"])
        assert np.allclose(a["history"][:h], b["history"][:h], rtol=1e-6)
        assert O.true_residual(m, E, O.element_stiffness(), f, ub) <= 1.5e-6


# ------------------------------------------------------------- full-size decision --
@pytest.mark.parametrize("prec,outer", [("mixed", 0), ("mixed", 2), ("fp64", 0)])
def test_full_size_select_floor_matches_oracle_record(gf, prec, outer):
    """Algorithm 1 on the 96x48x48 smoothed-Gaussian state (seed 0, 40% at floor, 5
    levels, probe at 1e-6, ladder {1e-5, 1e-4, 1e-3}, FGMRES(30), tau 1e-6, kmax 200)
    against the oracle's own full-size record (tests/golden/policy_c2_seed0.json,
    written by tests/golden/make_policy_records.py from oracle/ alone): the same status,
    floor and escalation, the same attempted floors, iterations within +-2 of the
    oracle's, and r50 / r100 within 1e-4 relative. Run in the native FP64 form and in
    the mixed form with native FP64 Krylov (outer 0) and with the FP64-class one (2)."""
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "policy_c2_seed0.json")))
    w = rec["workload"]
    rho = synth.smoothed_gaussian_density(w["nx"], w["ny"], w["nz"], rec["seed"], w["sigma"], w["floor_frac"])
    g = gf.create_grid(w["nx"], w["ny"], w["nz"], levels=w["levels"])
    g.set_density(dev(rho), w["p"])
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    u = torch.zeros_like(f)
    pol = gf.policy_defaults(rho0=w["rho0"], ladder=w["ladder"], tau=w["tau"], kmax=w["kmax"],
                             probe_iters=w["probe_iters"], solve_restart=w["restart"],
                             solve_prec=gf.GF_MIXED if prec == "mixed" else gf.GF_FP64, solve_outer=outer)
    out = g.select_floor(f, u, pol)
    assert out["status"] == rec["status"] and out["floor_index"] == rec["floor_index"]
    assert out["escalated"] == rec["escalated"]
    assert abs(out["r50"] - rec["r50"]) <= 1e-4 * rec["r50"]
    assert abs(out["r100"] - rec["r100"]) <= 1e-4 * rec["r100"]
    assert len(out["attempts"]) == len(rec["attempts"])
    for a, b in zip(out["attempts"], rec["attempts"]):
        assert a["rho_min"] == b["rho_min"] and abs(a["iters"] - b["iters"]) <= 2
        assert a["accepted"] == b["accepted"]
    assert out["eta"] <= w["tau"]


def _check_against_record(out, rec):
    w = rec["workload"]
    assert out["status"] == rec["status"] and out["floor_index"] == rec["floor_index"]
    assert out["escalated"] == rec["escalated"]
    assert abs(out["r50"] - rec["r50"]) <= 1e-4 * rec["r50"]
    assert abs(out["r100"] - rec["r100"]) <= 1e-4 * rec["r100"]
    assert len(out["attempts"]) == len(rec["attempts"])
    for a, b in zip(out["attempts"], rec["attempts"]):
        assert a["rho_min"] == b["rho_min"] and abs(a["iters"] - b["iters"]) <= 2
        assert a["accepted"] == b["accepted"]
    assert out["eta"] <= w["tau"]


@pytest.mark.parametrize("form", ["single", "batch"])
def test_192x96x96_select_floor_matches_oracle_record(gf, form):
    """Algorithm 1 at the large workload's size (192x96x96, 5 levels) on the
    smoothed-Gaussian state of seed 0 against the oracle's record
    (tests/golden/policy_c3_seed0.json, written by tests/golden/make_policy_records.py
    --size c3 from oracle/ alone), in the form the benchmark times: mixed V-cycle, native
    FP64 Krylov, one grid ("single") or two copies of the state solved together by the
    batch ("batch"). The same checks as the 96x48x48 record."""
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "policy_c3_seed0.json")))
    w = rec["workload"]
    dims = (w["nx"], w["ny"], w["nz"])
    rho = dev(synth.smoothed_gaussian_density(*dims, rec["seed"], w["sigma"], w["floor_frac"]))
    pol = gf.policy_defaults(rho0=w["rho0"], ladder=w["ladder"], tau=w["tau"], kmax=w["kmax"],
                             probe_iters=w["probe_iters"], solve_restart=w["restart"], solve_prec=gf.GF_MIXED,
                             solve_outer=0)
    if form == "single":
        g = gf.create_grid(*dims, levels=w["levels"])
        g.set_density(rho, w["p"])
        f = g.cantilever_load(torch.zeros(g.n_dof, dtype=torch.float64, device="cuda"))
        outs = [g.select_floor(f, torch.zeros_like(f), pol)]
        g.close()
    else:
        b = gf.Batch([dims] * 2, levels=w["levels"])
        for i in range(2):
            b.set_state(i, rho, b.cantilever_load(i, torch.zeros(b.n_dof[i], dtype=torch.float64, device="cuda")),
                        w["p"])
        outs = b.select_floor(pol)
        b.close()
    for out in outs:
        _check_against_record(out, rec)


# ------------------------------------------------------------- modal FP64 K*u -----
@pytest.mark.parametrize("chunk", ["0", "1", "3", "7"])
@pytest.mark.parametrize("dims", [(40, 20, 10, 2), (34, 18, 10, 2), (1, 2, 2, 1), (60, 28, 12, 3), (31, 14, 4, 1)])
def test_modal_apply_matches_oracle_and_dense(gf, dims, chunk, monkeypatch):
    """The FP64 K*u through the sum/difference factorisation of K0 (the default operator of
    gf_apply_K) against the oracle's element-by-element product to 1e-10, on grids whose
    extents leave ragged CTA tiles (31 x 15 nodes per tile) and for forced chunks of 1, 3
    and 7 node planes per CTA (0: the library's own choice); and against the dense node
    stencil (GF_MODAL=0) to the same bound."""
    nx, ny, nz, L = dims
    monkeypatch.setenv("GF_MODAL_CHUNK", chunk)
    g, m, rho = make(gf, nx, ny, nz, L, seed=nx + ny, rho_min=1e-6, kind="uniform")
    E = O.young_modulus(rho, 1e-6, 3.0)
    for seed in (5, 6):
        u = synth.random_vector(m.n_dof, seed)
        y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
        g.apply_K(dev(u), y)
        got = host(y)
        ref = O.apply_K(m, E, O.element_stiffness(), u)
        assert not np.isnan(got).any()
        assert relerr(got, ref) <= 1e-10
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
        assert np.all(got[m.fixed] == 0.0)
    monkeypatch.setenv("GF_MODAL", "0")
    gd, _, _ = make(gf, nx, ny, nz, L, seed=nx + ny, rho_min=1e-6, kind="uniform")
    yd = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    gd.apply_K(dev(u), yd)
    assert relerr(got, host(yd)) <= 1e-10


@pytest.mark.parametrize("dims", [(40, 20, 10, 2), (34, 18, 6, 2), (1, 2, 2, 1)])
def test_modal_apply_is_independent_of_the_launch_plan(gf, dims, monkeypatch):
    """Each node of the modal K*u sums the same four column corners in one order wherever the
    tiles fall: inside a tile in the kernel, on a tile boundary in the fix-up from the side
    buffer (which for the FP32 fine level also forms the node's smoothing update). Forced
    tile shapes (32 x 16, 16 x 32, and the half-SM 16 x 16 of gf_set_sm_share) and run
    lengths (1, 4 node planes, the cost model's choice) give bit-identical FP64 K*u, FP32
    K*u and mixed V-cycles, on ragged tiles."""
    nx, ny, nz, L = dims
    outs = []
    for share, bx in ((0, "32"), (0, "16"), (1, "16")):
        for chunk in ("1", "4", "0"):
            monkeypatch.setenv("GF_MODAL_BX", bx)
            monkeypatch.setenv("GF_MODAL_CHUNK", chunk)
            g, m, rho = make(gf, nx, ny, nz, L, seed=11, rho_min=1e-6, kind="uniform")
            if share:
                g.set_sm_share(1)   # clears the floor
                g.set_floor(1e-6)
            u = synth.random_vector(m.n_dof, 3)
            y = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
            g.apply_K(dev(u), y)
            y32 = torch.full((g.n_dof,), np.nan, dtype=torch.float32, device="cuda")
            g.apply_K_f32(dev(u, torch.float32), y32)
            z = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
            g.vcycle(dev(u * m.free), z, gf.GF_MIXED)
            outs.append((host(y), host(y32), host(z)))
            g.close()
    for a in outs[0]:
        assert not np.isnan(a).any()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
    ref = O.apply_K(m, O.young_modulus(rho, 1e-6, 3.0), O.element_stiffness(), u)
    assert relerr(outs[0][0], ref) <= 1e-10


@pytest.mark.parametrize("maxn", ["10000", "2000"])
def test_cluster_coarse_vcycle_matches_level_launches(gf, maxn, monkeypatch):
    """GF_VC_CLUSTER=<max nodes> (opt-in): the mixed V-cycle's levels from the first one with
    at most that many nodes run in one cluster launch (its own n x n coarsest GEMV; the sweep's
    inverse, GF_COARSE_LDL=0, so that it exists). The V-cycle agrees with the per-level
    launches to FP32 rounding, 1e-5 relative (not bit for bit: the per-level path's FP32
    kernels and the cluster's scalar node loops round differently), on 64x32x32 with 4
    levels, levels 1-3 or 2-3 in the cluster."""
    nx, ny, nz, L = 64, 32, 32, 4
    monkeypatch.setenv("GF_COARSE_LDL", "0")
    outs = []
    for env in (None, maxn):
        if env is None:
            monkeypatch.delenv("GF_VC_CLUSTER", raising=False)
        else:
            monkeypatch.setenv("GF_VC_CLUSTER", env)
        g, m, rho = make(gf, nx, ny, nz, L, seed=21, rho_min=1e-4, kind="bernoulli")
        v = synth.random_vector(m.n_dof, 4) * m.free
        z = torch.full((g.n_dof,), np.nan, dtype=torch.float64, device="cuda")
        g.vcycle(dev(v), z, gf.GF_MIXED)
        outs.append(host(z))
        g.close()
    assert not np.isnan(outs[0]).any() and not np.isnan(outs[1]).any()
    assert relerr(outs[1], outs[0]) <= 1e-5


# ------------------------------------------------------------- coarsest inverse -----
@pytest.mark.parametrize("dims", [(16, 8, 8, 3), (24, 10, 6, 2), (2, 2, 2, 1), (8, 4, 4, 1), (12, 6, 6, 2),
                                  (48, 24, 24, 3), (6, 4, 4, 2), (3, 2, 2, 1)])
def test_coarsest_inverses_agree(gf, dims, monkeypatch):
    """The coarsest level's dense FP64 inverse three ways: the banded LDL^T factorisation and
    the block-by-block inverse from it (default), the blocked symmetric sweep (8 pivots per
    launch on the upper triangle of the free-DOF matrix, each launch over the band ahead of
    its pivots; GF_COARSE_LDL=0), and the two-pivot full-matrix Gauss-Jordan (GF_SYM_GJ=0).
    FP64 V-cycles agree to 1e-10 relative, on coarsest levels whose size is not always a
    multiple of the pivot blocks (135 / 936 / 81 / 675 / 336 / 1,911 DOFs; at 936 and 675
    the band leaves the early sweeps a leading block of the matrix; at 1,911, the size of
    the 192x96x96 hierarchy's coarsest level, 56 LDL^T blocks each have 173 band rows below
    them; at 6x4x4 and 3x2x2 the 81 free DOFs are an odd count, which the coarsest GEMV reads
    one column at a time instead of in pairs); on one-level grids the inverse is the whole
    operator's, and its direct solution meets the oracle's guard."""
    nx, ny, nz, L = dims
    outs = []
    for ldl, sym in (("1", "1"), ("0", "1"), ("1", "0")):
        monkeypatch.setenv("GF_COARSE_LDL", ldl)
        monkeypatch.setenv("GF_SYM_GJ", sym)
        g, m, rho = make(gf, nx, ny, nz, L, seed=3, rho_min=1e-4, kind="bernoulli")
        v = synth.random_vector(m.n_dof, 9)
        z = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.vcycle(dev(v), z, gf.GF_FP64)
        outs.append(host(z))
        if L == 1 and ldl == "1" and sym == "1":
            f = O.cantilever_load(m)
            res = g.conditioning(dev(f), iters=20)
            E = O.young_modulus(rho, 1e-4, 3.0)
            # the direct solution's recomputed residual is at rounding level
            assert res["eta_direct"] <= 1e-9
            ref = O.vcycle(O.build_hierarchy(m, E, 1), v * m.free)
            assert relerr(outs[-1], ref) <= 1e-8
        g.close()
    assert relerr(outs[0], outs[2]) <= 1e-10
    assert relerr(outs[1], outs[2]) <= 1e-10
