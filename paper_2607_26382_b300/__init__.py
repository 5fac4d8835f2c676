"""B300-native guarded floor selection for matrix-free 3D SIMP state solves.

Hot path (arXiv 2607.26382): matrix-free hex8 K*u, GMG V-cycle, right-preconditioned
FGMRES, the FP64 recomputed-residual guard and the probe -> ladder -> guard policy
(Algorithm 1), all in hand-written CUDA (libgf_b300.so, C ABI in include/gf.h).
This package is the thin Python binding over that library.
"""
from ._lib import (  # noqa: F401
    GF_ACCEPTED, GF_COARSE_GALERKIN, GF_COARSE_REDISCRETISED, GF_FLAG_BREAKDOWN, GF_FLAG_CONVERGED, GF_FLAG_MAX_ITERS,
    GF_FP64, GF_GEOM_BRIDGE, GF_GEOM_CANTILEVER, GF_MIXED,
    GF_NO_ADMISSIBLE_FLOOR, GF_SEL_FULL, GF_SEL_GIVEN, GF_SEL_MLP, GF_SEL_REUSE, GF_SEL_RULE, Batch, GFError, Grid, MLP, create_grid, lib,
    conditioning_screen, policy_defaults, probe_features, round_to_f32, select_floor_many, trigger_rule,
    true_residual_noalloc, widen_to_f64,
)
