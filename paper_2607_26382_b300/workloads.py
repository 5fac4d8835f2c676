"""Inputs of the benchmark workloads, built with the library itself.

Every workload is seeded and synthetic. The random parts (noise fields, the voxels
forced to the floor) come from ``synth``; the SIMP-optimised designs come from
this library's own guarded SIMP-OC loop (``gf_oc_iteration``: linear-hat filter,
Algorithm 1 as the state solve, sensitivity through the filter adjoint, OC update
with move limit; Sec. 3.1), because the paper does not publish its optimised
fields. These inputs feed the GPU path only; no parity test takes them as oracle
inputs.

* ``simp_oc_design`` -- the physical density filter(x) after ``iters`` guarded
  SIMP-OC iterations from x = volfrac on the cantilever (tip load), each state solve
  at rho_min = 1e-3 (1e-2 as the guarded fallback), mixed V-cycle.
* ``large_states`` -- the 192x96x96 optimised-like states: the 40-iteration design
  (vol 0.3, r_min 1.5, p 3), then a seeded 30 % of voxels forced to 0.
* ``batch_states`` -- 102 frozen states of uneven size (nx in {32, 48, 64, 80},
  ny = nz = nx/2, round-robin): indices i with i % 10 < 7 are smoothed-Gaussian
  (sigma 2, 40 % at floor, seed 100 + i), the others optimised-like (the size's
  40-iteration SIMP-OC design with a seeded 30 % forced to 0, seed 200 + i).
* ``selector_designs`` -- SIMP-OC designs at 48x24x24 (vol 0.2, 0.3, 0.4) for the
  optimised-like third of the selector's training mix.
"""
from __future__ import annotations

from . import _lib as L

LARGE_DIMS = (192, 96, 96)
LARGE_LEVELS = 5
BATCH_LEVELS = 4


def _design_policy():
    return L.policy_defaults(rho0=1e-3, ladder=[1e-2], tau=1e-6, kmax=200, probe_iters=100,
                             selector=L.GF_SEL_GIVEN, first_index=0, solve_prec=L.GF_MIXED, solve_outer=2)


def simp_oc_design(nx, ny, nz, levels, iters=40, volfrac=0.3, r_min=1.5, p=3.0, move=0.2):
    """filter(x) after `iters` guarded SIMP-OC iterations (host float64, element order)."""
    import torch
    g = L.create_grid(nx, ny, nz, levels=levels)
    try:
        f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.cantilever_load(f)
        u = torch.zeros_like(f)
        x = torch.full((g.n_elem,), float(volfrac), dtype=torch.float64, device="cuda")
        pol = _design_policy()
        for _ in range(iters):
            g.oc_iteration(x, f, u, pol, p=p, volfrac=volfrac, r_min=r_min, move=move)
        rho = torch.empty_like(x)
        g.filter(x, rho, r_min)
        torch.cuda.synchronize()
        return rho.cpu().numpy().clip(0.0, 1.0)
    finally:
        g.close()


def large_states(seeds, iters=40):
    """192x96x96 optimised-like states: one SIMP-OC design, a seeded 30 % forced to 0 per seed."""
    import synth
    base = simp_oc_design(*LARGE_DIMS, LARGE_LEVELS, iters=iters)
    return [synth.force_to_floor(base, 0.3, s) for s in seeds]


def batch_states(n=102, seed0=100, iters=40):
    """(dims, densities, kinds) of the batched frozen-state workload."""
    import synth
    dims = synth.batch_grid_sizes(n)
    designs = {}
    rhos, kinds = [], []
    for i, (nx, ny, nz) in enumerate(dims):
        if i % 10 < 7:
            rhos.append(synth.smoothed_gaussian_density(nx, ny, nz, seed0 + i, 2.0, 0.4))
            kinds.append("random")
        else:
            if (nx, ny, nz) not in designs:
                designs[(nx, ny, nz)] = simp_oc_design(nx, ny, nz, BATCH_LEVELS, iters=iters)
            rhos.append(synth.force_to_floor(designs[(nx, ny, nz)], 0.3, seed0 + 100 + i))
            kinds.append("optimised")
    return dims, rhos, kinds


def selector_designs(dims=(48, 24, 24), volumes=(0.2, 0.3, 0.4), iters=40):
    return [simp_oc_design(*dims, BATCH_LEVELS, iters=iters, volfrac=v) for v in volumes]


def n_dof(dims):
    nx, ny, nz = dims
    return 3 * (nx + 1) * (ny + 1) * (nz + 1)
