"""CPU checks of the CUDA library: it builds, loads, exports every symbol declared in
include/gf.h, and its host-only policy logic makes the same decisions as the oracle
on identical residuals (bit-exact integer decisions)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import gf_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gflib():
    from paper_2607_26382_b300 import build
    build.build()
    from paper_2607_26382_b300 import _lib
    return _lib


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gf.h")).read()
    return sorted(set(re.findall(r"\b(gf_[A-Za-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(gflib):
    L = gflib.lib()
    declared = _declared_symbols()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(L, name), name
    assert set(gflib.EXPORTED) <= set(declared)


def test_trigger_rule_matches_oracle_bit_exact(gflib):
    rng = np.random.default_rng(0)
    pol = gflib.policy_defaults()
    # random pairs over the decision-relevant range plus exact threshold hits
    r50 = 10.0 ** rng.uniform(-8, 0, 4000)
    r100 = r50 * 10.0 ** rng.uniform(-4, 0.5, 4000)
    extra = [(1e-2, 1e-9), (1e-3, 1e-4), (1e-4 / 0.6, 1e-4), (1.6e-4, 1e-4), (2e-4, 9.99e-5)]
    pairs = list(zip(r50, r100)) + extra
    for a, b in pairs:
        assert gflib.trigger_rule(a, b, pol) == O.trigger_rule(a, b), (a, b)


def test_trigger_rule_golden_rows(gflib):
    here = os.path.join(ROOT, "tests", "golden")
    for fname, cols in (("false_keep_rows.txt", (2, 3, 4)), ("trigger_boundaries.txt", (0, 1, 2))):
        for line in open(os.path.join(here, fname)):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            f = line.split()
            r50, r100, out = float(f[cols[0]]), float(f[cols[1]]), f[cols[2]]
            assert gflib.trigger_rule(r50, r100) == (out == "escalate")


def test_probe_features_match_oracle(gflib):
    hist = list(np.geomspace(1.0, 1e-7, 140))
    for k_stop in (0, 10, 49, 50, 51, 99, 100, 139):
        assert gflib.probe_features(hist, k_stop) == O.probe_features(np.array(hist), k_stop)


def test_policy_defaults(gflib):
    p = gflib.policy_defaults()
    assert (p.rho0, p.tau, p.kmax, p.probe_iters) == (1e-6, 1e-6, 200, 100)
    assert [p.ladder[i] for i in range(p.n_ladder)] == [1e-5, 1e-4, 1e-3]
    assert (p.r50_escalate, p.r100_stall, p.plateau_ratio) == (1e-2, 1e-4, 0.6)
    assert (p.solve.restart, p.solve.nu1, p.solve.nu2, p.solve.omega) == (30, 2, 2, 0.6)
    assert (p.true_check_every, p.true_check_ratio) == (0, 10.0)    # the struct's last fields line up
    assert (p.solve.ls_ratio, p.solve.fine_steps, p.solve.coarse_steps) == (0.0, 0, 0)   # adaptive parts off
    p2 = gflib.policy_defaults(ladder=[1e-3, 1e-2], rho0=1e-12, solve_prec=gflib.GF_MIXED)
    assert p2.n_ladder == 2 and p2.rho0 == 1e-12 and p2.solve.prec == gflib.GF_MIXED


def test_missing_library_fails_loudly(gflib, monkeypatch):
    monkeypatch.setattr(gflib, "_LIB", None)
    monkeypatch.setattr(gflib, "LIB_PATH", "/nonexistent/libgf_b300.so")
    with pytest.raises(RuntimeError):
        gflib.lib()


def test_conditioning_screen_matches_oracle(gflib):
    from oracle import gf_oracle as O
    for args in ((1e-8, 2.5, 1e-6, 1e-6), (3e-15, 4.0, 1e-12, 1e-6), (0.5, 0.5, 1e-2, 1e-8)):
        assert gflib.conditioning_screen(*args) == O.conditioning_screen(*args)
    for bad in ((0.0, 1.0, 1e-6, 1e-6), (2.0, 1.0, 1e-6, 1e-6), (1e-3, 1.0, 0.0, 1e-6), (1e-3, 1.0, 1e-6, 0.0)):
        with pytest.raises(gflib.GFError):
            gflib.conditioning_screen(*bad)


@pytest.mark.parametrize("dims,bridge", [((12, 6, 6), False), ((12, 5, 3), False), ((8, 4, 4), False),
                                         ((12, 6, 6), True), ((16, 4, 8), True), ((4, 10, 6), False)])
def test_coarsest_band_bound_holds_for_the_free_dof_matrix(dims, bridge):
    """The coarsest inverse's sweep launches only the tiles inside the band ahead of its
    pivots. It orders the free DOFs with nodes running along the axis with the fewest nodes
    first and the most nodes last (ties in x, y, z order), a node's three components
    together, and assumes no non-zero with |p - q| > 3 (1 + N_a + N_a N_b) + 2 (N_a <= N_b
    the two smallest node counts). The oracle's assembled operator, with random moduli and
    permuted into that order here, stays inside that band for the cantilever and for the
    bridge's supports, and reaches within one node layer of it (the bound is not loose by a
    layer); in x-fastest order it would not fit when x is not the shortest axis."""
    nx, ny, nz = dims
    mesh = O.BridgeMesh(nx, ny, nz) if bridge else O.Mesh(nx, ny, nz)
    E = np.random.default_rng(nx * ny + nz).uniform(0.01, 1.0, mesh.n_elem)
    K = O.assemble_sparse(mesh, E, O.element_stiffness(), constrained=False).tocsr()
    N = [nx + 1, ny + 1, nz + 1]
    ax = sorted(range(3), key=lambda a: N[a])          # stable: ties keep x, y, z order
    # DOF q = 3 (i + NX (j + NY k)) + c listed in the compact order
    order = []
    for u2 in range(N[ax[2]]):
        for u1 in range(N[ax[1]]):
            for u0 in range(N[ax[0]]):
                v = [0, 0, 0]
                v[ax[0]], v[ax[1]], v[ax[2]] = u0, u1, u2
                node = v[0] + N[0] * (v[1] + N[1] * v[2])
                order.extend(3 * node + c for c in range(3))
    order = np.array(order)
    assert np.array_equal(np.sort(order), np.arange(3 * N[0] * N[1] * N[2]))
    free = order[mesh.free[order]]
    rows, cols = K[free][:, free].nonzero()
    band = 3 * (1 + N[ax[0]] + N[ax[0]] * N[ax[1]]) + 2
    width = int(np.max(np.abs(rows - cols)))
    assert width <= band
    assert width > band - 3 * N[ax[0]] * N[ax[1]]
    if ax[0] != 0:   # the x-fastest bound is wider than the permuted one
        assert band < 3 * (1 + N[0] + N[0] * N[1]) + 2
