"""Batched frozen states: every state's Algorithm-1 result from the batch equals the
single-state path bit for bit (same kernels, same reduction order), and the
accepted solutions pass the oracle's own FP64 guard."""
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


STATES = [((16, 8, 8), "bern", 43, 0.35), ((24, 12, 12), "smooth", 1, 0.4), ((32, 16, 16), "bern", 47, 0.30),
          ((16, 8, 8), "smooth", 5, 0.3), ((20, 12, 8), "bern", 3, 0.25)]


def _rho(dims, kind, seed, q):
    nx, ny, nz = dims
    if kind == "bern":
        return synth.bernoulli_density(nx, ny, nz, seed, q)
    return synth.smoothed_gaussian_density(nx, ny, nz, seed, 2.0, q)


# restart 45: past 32 basis vectors the Gram-Schmidt passes run over 32-vector slices
@pytest.mark.parametrize("selector,prec,outer,smoother,restart", [("rule", 0, 0, 0, 30), ("full", 1, 0, 0, 30),
                                                                  ("rule", 1, 2, 0, 30), ("rule", 1, 2, 1, 30),
                                                                  ("rule", 1, 2, 0, 45), ("full", 0, 0, 0, 45)])
def test_batch_matches_single_state(gf, selector, prec, outer, smoother, restart):
    L = 3
    sel = gf.GF_SEL_RULE if selector == "rule" else gf.GF_SEL_FULL
    pol = gf.policy_defaults(rho0=1e-8, ladder=[1e-5, 1e-4, 1e-3], kmax=120, selector=sel, solve_prec=prec,
                             solve_outer=outer, solve_smoother=smoother, solve_restart=restart)
    batch = gf.Batch([s[0] for s in STATES], levels=L)
    tuned = batch.autotune()
    assert all(t[0] in (64, 128, 256) and t[1] in (0, 64, 128, 256, -64, -128, -256) for t in tuned)
    rhos, fs = [], []
    for i, (dims, kind, seed, q) in enumerate(STATES):
        rho = dev(_rho(dims, kind, seed, q))
        f = dev(O.cantilever_load(O.Mesh(*dims)))
        rhos.append(rho)
        fs.append(f)
        batch.set_state(i, rho, f, 3.0)
    res = batch.select_floor(pol)
    assert batch.kernel_launches() > 0
    for i, (dims, kind, seed, q) in enumerate(STATES):
        g = gf.create_grid(*dims, levels=L)
        g.set_stencil_blocks(*tuned[i])      # same launch choice as the batch's autotuned state
        g.set_density(rhos[i], 3.0)
        u1 = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        ref = g.select_floor(fs[i], u1, pol)
        got = res[i]
        for key in ("status", "floor_index", "escalated", "eta", "r50", "r100"):
            a, b = got[key], ref[key]
            assert a == b or (isinstance(a, float) and np.isnan(a) and np.isnan(b)), (i, key, a, b)
        assert got["attempts"] == ref["attempts"], i
        u2 = torch.zeros_like(u1)
        batch.solution(i, u2)
        if got["status"] == gf.GF_ACCEPTED:
            assert torch.equal(u1, u2), i
            m = O.Mesh(*dims)
            E = O.young_modulus(_rho(dims, kind, seed, q), got["rho_min"], 3.0)
            eta = O.true_residual(m, E, O.element_stiffness(), O.cantilever_load(m), u2.cpu().numpy())
            assert eta <= 1e-6 * (1 + 1e-9)
        g.close()
    # a second run on the same batch (graphs reused) reproduces the first
    res2 = batch.select_floor(pol)
    strip = lambda r: {k: (None if isinstance(v, float) and np.isnan(v) else v) for k, v in r.items()}
    assert [strip(r) for r in res2] == [strip(r) for r in res]
    batch.close()


def test_batch_half_sm_matches_single_state(gf):
    """gf_batch_set_sm_share(1), called after the states are set: every state's result and
    solution equal those of its single grid with the same half-SM launch shapes, bit for bit
    (the same kernels and Gram-Schmidt block partition), and the accepted solutions pass
    the oracle's guard."""
    L = 3
    pol = gf.policy_defaults(rho0=1e-8, ladder=[1e-5, 1e-4, 1e-3], kmax=120, solve_prec=1, solve_outer=0)
    batch = gf.Batch([s[0] for s in STATES], levels=L)
    tuned = batch.autotune()
    rhos, fs = [], []
    for i, (dims, kind, seed, q) in enumerate(STATES):
        rhos.append(dev(_rho(dims, kind, seed, q)))
        fs.append(dev(O.cantilever_load(O.Mesh(*dims))))
        batch.set_state(i, rhos[i], fs[i], 3.0)
    batch.set_sm_share(1)
    with pytest.raises(gf.GFError):
        batch.set_sm_share(-1)
    res = batch.select_floor(pol)
    for i, (dims, kind, seed, q) in enumerate(STATES):
        g = gf.create_grid(*dims, levels=L)
        g.set_stencil_blocks(*tuned[i])
        g.set_sm_share(1)
        g.set_density(rhos[i], 3.0)
        u1 = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        ref = g.select_floor(fs[i], u1, pol)
        assert res[i]["attempts"] == ref["attempts"], i
        assert res[i]["status"] == ref["status"] and res[i]["floor_index"] == ref["floor_index"], i
        u2 = torch.zeros_like(u1)
        batch.solution(i, u2)
        assert torch.equal(u1, u2), i
        if res[i]["status"] == gf.GF_ACCEPTED:
            m = O.Mesh(*dims)
            E = O.young_modulus(_rho(dims, kind, seed, q), res[i]["rho_min"], 3.0)
            eta = O.true_residual(m, E, O.element_stiffness(), O.cantilever_load(m), u2.cpu().numpy())
            assert eta <= 1e-6 * (1 + 1e-9)
        g.close()
    batch.close()


def test_batch_sweep_inverse_matches_single_state(gf, monkeypatch):
    """With the coarsest inverse by the blocked symmetric sweep (GF_COARSE_LDL=0) the batch
    runs the sweep in lockstep over its states: every state's result and solution still
    equal its single grid's, bit for bit."""
    monkeypatch.setenv("GF_COARSE_LDL", "0")
    L = 3
    pol = gf.policy_defaults(rho0=1e-8, ladder=[1e-5, 1e-4, 1e-3], kmax=120, solve_prec=1, solve_outer=0)
    batch = gf.Batch([s[0] for s in STATES], levels=L)
    tuned = batch.autotune()
    rhos, fs = [], []
    for i, (dims, kind, seed, q) in enumerate(STATES):
        rhos.append(dev(_rho(dims, kind, seed, q)))
        fs.append(dev(O.cantilever_load(O.Mesh(*dims))))
        batch.set_state(i, rhos[i], fs[i], 3.0)
    res = batch.select_floor(pol)
    for i, (dims, kind, seed, q) in enumerate(STATES):
        g = gf.create_grid(*dims, levels=L)
        g.set_stencil_blocks(*tuned[i])
        g.set_density(rhos[i], 3.0)
        u1 = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        ref = g.select_floor(fs[i], u1, pol)
        assert res[i]["attempts"] == ref["attempts"], i
        u2 = torch.zeros_like(u1)
        batch.solution(i, u2)
        assert torch.equal(u1, u2), i
        g.close()
    batch.close()


def test_batch_rejects_single_grid_options(gf):
    """The reuse selector, true-residual checks, the line-searched coarse correction, the
    fine-level correction and the coarse-level Krylov solve are single-grid options; the batch
    refuses them."""
    dims, kind, seed, q = STATES[0]
    batch = gf.Batch([dims], levels=3)
    batch.set_state(0, dev(_rho(dims, kind, seed, q)), dev(O.cantilever_load(O.Mesh(*dims))), 3.0)
    for kw in (dict(selector=gf.GF_SEL_REUSE), dict(true_check_every=10), dict(solve_ls_ratio=0.1),
               dict(solve_fine_steps=5), dict(solve_coarse_steps=10)):
        with pytest.raises(gf.GFError):
            batch.select_floor(gf.policy_defaults(**kw))
    assert batch.select_floor(gf.policy_defaults())[0]["status"] in (gf.GF_ACCEPTED, gf.GF_NO_ADMISSIBLE_FLOOR)
    batch.close()


@pytest.mark.parametrize("prec,outer", [(0, 0), (1, 2), (1, 0)])
def test_batch_galerkin_matches_single_state(gf, prec, outer):
    """Galerkin coarse operators in the batch (gf_batch_set_coarse_operator): every state's
    Algorithm-1 result and solution equal its single grid's with the same coarse operator,
    bit for bit (the lockstep coarsest inverses assemble the Galerkin coarsest matrices)."""
    L = 3
    pol = gf.policy_defaults(rho0=1e-8, ladder=[1e-5, 1e-4, 1e-3], kmax=120, solve_prec=prec, solve_outer=outer)
    batch = gf.Batch([s[0] for s in STATES], levels=L)
    batch.set_coarse_operator(gf.GF_COARSE_GALERKIN)
    rhos, fs = [], []
    for i, (dims, kind, seed, q) in enumerate(STATES):
        rho = dev(_rho(dims, kind, seed, q))
        f = dev(O.cantilever_load(O.Mesh(*dims)))
        rhos.append(rho)
        fs.append(f)
        batch.set_state(i, rho, f, 3.0)
    tuned = batch.autotune()
    res = batch.select_floor(pol)
    for i, (dims, kind, seed, q) in enumerate(STATES):
        g = gf.create_grid(*dims, levels=L)
        g.set_coarse_operator(gf.GF_COARSE_GALERKIN)
        g.set_stencil_blocks(*tuned[i])
        g.set_density(rhos[i], 3.0)
        u1 = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        ref = g.select_floor(fs[i], u1, pol)
        got = res[i]
        for key in ("status", "floor_index", "escalated", "eta", "r50", "r100"):
            a, b = got[key], ref[key]
            assert a == b or (isinstance(a, float) and np.isnan(a) and np.isnan(b)), (i, key, a, b)
        assert got["attempts"] == ref["attempts"], i
        u2 = torch.zeros_like(u1)
        batch.solution(i, u2)
        if got["status"] == gf.GF_ACCEPTED:
            assert torch.equal(u1, u2), i
            m = O.Mesh(*dims)
            E = O.young_modulus(_rho(dims, kind, seed, q), got["rho_min"], 3.0)
            eta = O.true_residual(m, E, O.element_stiffness(), O.cantilever_load(m), u2.cpu().numpy())
            assert eta <= 1e-6 * (1 + 1e-9)
        g.close()
    batch.close()


def test_batch_cantilever_load_matches_grid_and_oracle(gf):
    # Batch.cantilever_load writes each state's tip load on its own grid: the same vector
    # as a single grid of that size, and the oracle's load
    dims = [(16, 8, 8), (20, 12, 8)]
    b = gf.Batch(dims, levels=2)
    for i, d in enumerate(dims):
        fb = b.cantilever_load(i, torch.empty(b.n_dof[i], dtype=torch.float64, device="cuda"))
        g = gf.create_grid(*d, levels=2)
        fg = g.cantilever_load(torch.empty(g.n_dof, dtype=torch.float64, device="cuda"))
        assert torch.equal(fb, fg)
        assert np.array_equal(fb.cpu().numpy(), O.cantilever_load(O.Mesh(*d)))
        g.close()
    b.close()


def test_select_floor_many_matches_each_grid_alone(gf):
    # gf_select_floor_many runs one host thread per grid; grids on distinct streams run
    # concurrently, and every state's result is bit-identical to its grid run alone
    pol = gf.policy_defaults(rho0=1e-6, ladder=[1e-5, 1e-4, 1e-3], tau=1e-6, kmax=200, probe_iters=100,
                             solve_prec=gf.GF_MIXED, solve_outer=0)

    def grids_for(streams):
        gs, fs = [], []
        for (dims, kind, seed, q), st in zip(STATES[:3], streams):
            g = gf.create_grid(*dims, levels=3, stream=st)
            g.set_density(dev(_rho(dims, kind, seed, q)), 3.0)
            fs.append(g.cantilever_load(torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")))
            gs.append(g)
        return gs, fs

    streams = [torch.cuda.Stream() for _ in range(3)]
    alone, u_alone = [], []
    gs, fs = grids_for(streams)
    for g, f in zip(gs, fs):
        u = torch.zeros_like(f)
        alone.append(g.select_floor(f, u, pol))
        u_alone.append(u)
    gs2, fs2 = grids_for(streams)
    us2 = [torch.zeros_like(f) for f in fs2]
    many = gf.select_floor_many(gs2, fs2, us2, pol)
    torch.cuda.synchronize()
    for a, b, ua, ub in zip(alone, many, u_alone, us2):
        assert a == b and torch.equal(ua, ub) and b["status"] == gf.GF_ACCEPTED
    # the half-SM launch shapes (gf_set_sm_share): the same operator bit for bit and the
    # Gram-Schmidt sums over another block partition, so the same decisions and FGMRES
    # iterations; the sums' rounding, amplified by the operator's conditioning over the
    # iterations, moves the solutions apart by ~5e-9 here, inside the solve tolerance tau
    gs3, fs3 = grids_for(streams)
    for g in gs3:
        g.set_sm_share(1)
    with pytest.raises(gf.GFError):
        gs3[0].set_sm_share(2)
    us3 = [torch.zeros_like(f) for f in fs3]
    shared = gf.select_floor_many(gs3, fs3, us3, pol)
    torch.cuda.synchronize()
    for a, c, ua, uc in zip(alone, shared, u_alone, us3):
        assert c["status"] == gf.GF_ACCEPTED and c["floor_index"] == a["floor_index"]
        assert [t["iters"] for t in c["attempts"]] == [t["iters"] for t in a["attempts"]]
        assert float((uc - ua).norm() / ua.norm()) <= 1e-6
    for g in gs3:
        g.close()
    with pytest.raises(gf.GFError):
        gf.select_floor_many([gs2[0], gs2[0]], [fs2[0], fs2[0]], [us2[0], torch.zeros_like(us2[0])], pol)
    # a grid that cannot run (no density stored) fails the call with its own error, named by
    # its position; the other grids still run to completion
    dims = STATES[0][0]
    bad = gf.create_grid(*dims, levels=3)
    fb = bad.cantilever_load(torch.zeros(bad.n_dof, dtype=torch.float64, device="cuda"))
    with pytest.raises(gf.GFError) as e:
        gf.select_floor_many([gs2[0], bad], [fs2[0], fb], [us2[0], torch.zeros_like(fb)], pol)
    assert "grid 1" in str(e.value) and "set_density" in str(e.value)
    torch.cuda.synchronize()
    bad.close()
    for g in gs + gs2:
        g.close()
