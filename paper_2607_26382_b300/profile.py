"""Run one operation of the library a few times on a synthetic state (a profiling target).

    python -m paper_2607_26382_b300.profile apply_k64 --grid 96 48 48 --levels 5 --reps 3
    ops: apply_k64, apply_split, apply_k32, vcycle_mixed, vcycle_fp64, solve_mixed, select_mixed, set_floor
    (--galerkin: the V-cycles on Galerkin coarse operators)

The state is the smoothed-Gaussian density (sigma 2, 40% at floor) at rho_min 1e-6,
p = 3, with the cantilever tip load. Used as the command under ncu so that a
capture covers a known, small number of launches. The repeated operation runs
between cudaProfilerStart and cudaProfilerStop, so `ncu --profile-from-start off`
captures it without the set-up (density, floor, coarsest inverse).
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["apply_k64", "apply_split", "apply_k32", "vcycle_mixed", "vcycle_fp64",
                                   "solve_mixed", "select_mixed", "set_floor"])
    ap.add_argument("--grid", type=int, nargs=3, default=[96, 48, 48])
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--outer", type=int, default=1,
                    help="Krylov arithmetic: 0 native FP64, 1 split-integer K*u, 2 split K*u + double-float CGS2")
    ap.add_argument("--kmax", type=int, default=200, help="iteration budget of solve_mixed")
    ap.add_argument("--fine", type=int, default=0, help="fine-level adaptive correction steps (solve_mixed)")
    ap.add_argument("--galerkin", action="store_true", help="Galerkin coarse operators (gf_set_coarse_operator)")
    ap.add_argument("--sm-share", type=int, default=0, help="gf_set_sm_share: 1 = half-SM launch shapes")
    a = ap.parse_args(argv)

    import torch

    import synth
    from . import _lib as gf

    nx, ny, nz = a.grid
    g = gf.create_grid(nx, ny, nz, levels=a.levels)
    g.set_sm_share(a.sm_share)
    g.set_density(torch.as_tensor(synth.smoothed_gaussian_density(nx, ny, nz, a.seed), device="cuda"), 3.0)
    if a.galerkin:
        g.set_coarse_operator(gf.GF_COARSE_GALERKIN)
    g.set_floor(1e-6)
    gen = torch.Generator(device="cuda").manual_seed(a.seed)
    x = torch.randn(g.n_dof, dtype=torch.float64, device="cuda", generator=gen)
    y = torch.empty_like(x)
    f = torch.zeros_like(x)
    g.cantilever_load(f)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(a.reps):
        if a.op == "apply_k64":
            g.apply_K(x, y)
        elif a.op == "apply_split":
            g.apply_K_split(x, y)
        elif a.op == "apply_k32":
            g.apply_K_f32(x.float(), y.float())
        elif a.op == "vcycle_mixed":
            g.vcycle(x, y, gf.GF_MIXED)
        elif a.op == "vcycle_fp64":
            g.vcycle(x, y, gf.GF_FP64)
        elif a.op == "set_floor":
            g.set_floor(1e-6)
        elif a.op == "solve_mixed":
            y.zero_()
            g.solve(f, y, prec=gf.GF_MIXED, outer=a.outer, kmax=a.kmax, fine_steps=a.fine)
        else:
            g.set_density(torch.as_tensor(synth.smoothed_gaussian_density(nx, ny, nz, a.seed), device="cuda"), 3.0)
            g.select_floor(f, y, gf.policy_defaults(solve_prec=gf.GF_MIXED, solve_outer=a.outer))
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(f"{a.op} x{a.reps} on {nx}x{ny}x{nz}: ok", flush=True)
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
