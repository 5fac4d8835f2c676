"""ctypes binding of the C ABI in include/gf.h (argument marshalling only).

Every computation runs in libgf_b300.so; this module checks tensor shapes, dtypes
and devices, passes raw pointers and the current CUDA stream, and converts the
info structs. It never computes anything itself and has no CPU fallback: if the
shared library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_longlong, c_uint8, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgf_b300.so")

GF_OK = 0
GF_FP64, GF_MIXED = 0, 1
GF_FLAG_CONVERGED, GF_FLAG_MAX_ITERS, GF_FLAG_BREAKDOWN = 0, 1, 2
GF_ACCEPTED, GF_NO_ADMISSIBLE_FLOOR = 0, 1
GF_SEL_RULE, GF_SEL_FULL, GF_SEL_GIVEN, GF_SEL_MLP, GF_SEL_REUSE = 0, 1, 2, 3, 4
MLP_PARAMS = 1412
GF_MAX_LADDER = 8
GF_MAX_TRUE_CHECKS = 16
GF_COARSE_REDISCRETISED, GF_COARSE_GALERKIN = 0, 1
GF_GEOM_CANTILEVER, GF_GEOM_BRIDGE = 0, 1

ERRORS = {-1: "GF_ERR_ARG", -2: "GF_ERR_OOM", -3: "GF_ERR_CUDA", -4: "GF_ERR_NONFINITE",
          -5: "GF_ERR_TIMEOUT", -6: "GF_ERR_STATE"}

EXPORTED = [
    "gf_create_grid", "gf_destroy_grid", "gf_grid_sizes", "gf_set_density", "gf_set_floor",
    "gf_cantilever_load", "gf_free_mask", "gf_apply_K", "gf_apply_K_f32", "gf_vcycle", "gf_vcycle_ex", "gf_chebyshev_lambda", "gf_conditioning", "gf_conditioning_screen", "gf_solve",
    "gf_true_residual", "gf_select_floor", "gf_select_floor_many", "gf_policy_defaults", "gf_trigger_rule",
    "gf_probe_features", "gf_sensitivity", "gf_get_stats", "gf_reset_stats", "gf_last_error",
    "gf_true_residual_noalloc", "gf_filter", "gf_filter_adjoint", "gf_oc_update", "gf_compliance",
    "gf_oc_iteration", "gf_create_batch", "gf_destroy_batch", "gf_batch_grid", "gf_batch_set_state",
    "gf_batch_solution", "gf_batch_autotune", "gf_batch_select_floor", "gf_batch_stats",
    "gf_mlp_create", "gf_mlp_destroy", "gf_mlp_set_norm", "gf_mlp_get_params", "gf_mlp_forward",
    "gf_mlp_loss_grad", "gf_mlp_train", "gf_mlp_predict", "gf_select_features", "gf_apply_K_split",
    "gf_set_coarse_operator", "gf_set_sm_share", "gf_batch_set_sm_share", "gf_round_to_f32", "gf_widen_to_f64", "gf_set_geometry", "gf_bridge_load", "gf_batch_set_coarse_operator",
]


class GFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SolveOpts(ctypes.Structure):
    _fields_ = [("restart", c_int), ("kmax", c_int), ("tol", c_double), ("prec", c_int),
                ("nu1", c_int), ("nu2", c_int), ("omega", c_double), ("history", POINTER(c_double)),
                ("outer", c_int), ("smoother", c_int), ("ls_ratio", c_double), ("fine_steps", c_int),
                ("coarse_steps", c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", c_int), ("flag", c_int), ("stop_estimate", c_double)]


class Policy(ctypes.Structure):
    _fields_ = [("rho0", c_double), ("ladder", c_double * GF_MAX_LADDER), ("n_ladder", c_int),
                ("tau", c_double), ("kmax", c_int), ("probe_iters", c_int),
                ("r50_escalate", c_double), ("r100_stall", c_double), ("plateau_ratio", c_double),
                ("checkpoint_a", c_int), ("checkpoint_b", c_int), ("selector", c_int),
                ("first_index", c_int), ("fuse_probe", c_int), ("solve", SolveOpts), ("mlp", c_void_p),
                ("mlp_confidence", c_double), ("true_check_every", c_int), ("true_check_ratio", c_double)]


class Attempt(ctypes.Structure):
    _fields_ = [("rho_min", c_double), ("iters", c_int), ("flag", c_int),
                ("stop_estimate", c_double), ("eta", c_double), ("accepted", c_int)]


class SelectInfo(ctypes.Structure):
    _fields_ = [("status", c_int), ("floor_index", c_int), ("rho_min", c_double), ("eta", c_double),
                ("r50", c_double), ("r100", c_double), ("escalated", c_int), ("probe_iters_run", c_int),
                ("n_attempts", c_int), ("attempts", Attempt * (GF_MAX_LADDER + 1)),
                ("n_true_checks", c_int), ("true_check_k", c_int * GF_MAX_TRUE_CHECKS),
                ("true_check_est", c_double * GF_MAX_TRUE_CHECKS), ("true_check_eta", c_double * GF_MAX_TRUE_CHECKS),
                ("true_check_fired", c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", c_longlong), ("apply_K_fp64", c_longlong), ("vcycles", c_longlong)]


_LIB = None


def lib():
    """Load libgf_b300.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run python -m paper_2607_26382_b300.build)")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "gf_create_grid": [c_int, c_int, c_int, c_double, c_double, c_double, c_int, P, POINTER(P)],
        "gf_destroy_grid": [P],
        "gf_grid_sizes": [P, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)],
        "gf_set_density": [P, P, c_double],
        "gf_set_floor": [P, c_double],
        "gf_set_coarse_operator": [P, c_int],
        "gf_set_sm_share": [P, c_int],
        "gf_batch_set_sm_share": [P, c_int],
        "gf_round_to_f32": [P, P, c_longlong, P],
        "gf_widen_to_f64": [P, P, c_longlong, P],
        "gf_cantilever_load": [P, P],
        "gf_set_geometry": [P, c_int],
        "gf_bridge_load": [P, P],
        "gf_free_mask": [P, P],
        "gf_apply_K": [P, P, P],
        "gf_apply_K_f32": [P, P, P],
        "gf_conditioning": [P, P, c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double)],
        "gf_conditioning_screen": [c_double, c_double, c_double, c_double, POINTER(c_double)],
        "gf_vcycle": [P, P, P, c_int, c_int, c_int, c_double],
        "gf_vcycle_ex": [P, P, P, P],
        "gf_chebyshev_lambda": [P, c_int, P, c_int],
        "gf_solve": [P, P, P, POINTER(SolveOpts), POINTER(SolveInfo)],
        "gf_true_residual": [P, P, P, POINTER(c_double)],
        "gf_select_floor": [P, P, P, POINTER(Policy), POINTER(SelectInfo)],
        "gf_select_floor_many": [c_int, POINTER(P), POINTER(P), POINTER(P), POINTER(Policy), POINTER(SelectInfo)],
        "gf_trigger_rule": [c_double, c_double, POINTER(Policy)],
        "gf_probe_features": [POINTER(c_double), c_int, POINTER(Policy), POINTER(c_double), POINTER(c_double)],
        "gf_sensitivity": [P, P, P],
        "gf_get_stats": [P, POINTER(Stats)],
        "gf_reset_stats": [P],
        "gf_true_residual_noalloc": [c_int, c_int, c_int, c_double, c_double, c_double, P, c_double, c_double,
                                     P, P, P, P],
        "gf_filter": [P, P, P, c_double],
        "gf_filter_adjoint": [P, P, P, c_double],
        "gf_oc_update": [P, P, P, P, c_double, c_double, P],
        "gf_compliance": [P, P, P, POINTER(c_double)],
        "gf_oc_iteration": [P, P, P, P, POINTER(Policy), c_double, c_double, c_double, c_double,
                            POINTER(SelectInfo), POINTER(c_double)],
        "gf_create_batch": [c_int, POINTER(c_int), c_int, c_double, c_double, c_double, P, POINTER(P)],
        "gf_destroy_batch": [P],
        "gf_batch_grid": [P, c_int, POINTER(P)],
        "gf_batch_set_state": [P, c_int, P, c_double, P],
        "gf_batch_solution": [P, c_int, P],
        "gf_batch_autotune": [P, POINTER(c_int)],
        "gf_batch_set_coarse_operator": [P, c_int],
        "gf_batch_select_floor": [P, POINTER(Policy), POINTER(SelectInfo)],
        "gf_batch_stats": [P, POINTER(c_longlong)],
        "gf_mlp_create": [POINTER(ctypes.c_float), P, POINTER(P)],
        "gf_mlp_destroy": [P],
        "gf_mlp_set_norm": [P, POINTER(ctypes.c_float), POINTER(ctypes.c_float)],
        "gf_mlp_get_params": [P, POINTER(ctypes.c_float)],
        "gf_mlp_forward": [P, P, c_int, P],
        "gf_mlp_loss_grad": [P, P, P, c_int, POINTER(ctypes.c_float), POINTER(ctypes.c_float)],
        "gf_mlp_train": [P, P, P, c_int, POINTER(c_int), c_int, c_int, ctypes.c_float, POINTER(ctypes.c_float)],
        "gf_mlp_predict": [P, POINTER(c_double), c_int, POINTER(c_int)],
        "gf_select_features": [P, c_double, c_double, POINTER(c_double)],
        "gf_apply_K_split": [P, P, P],
        "gf_set_stencil_blocks": [P, c_int, c_int],
        "gf_mlp_probs": [P, POINTER(c_double), c_int, POINTER(c_double)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = c_int
    L.gf_policy_defaults.argtypes = [POINTER(Policy)]
    L.gf_policy_defaults.restype = None
    L.gf_last_error.argtypes = []
    L.gf_last_error.restype = c_char_p
    _LIB = L
    return L


def _check(code):
    if code < 0:
        raise GFError(code, lib().gf_last_error().decode())
    return code


# ------------------------------------------------------------- host-only logic --
def policy_defaults(**kw) -> Policy:
    """gf_policy_defaults, then overrides: ladder=[...], solve_* fields, or any Policy field."""
    p = Policy()
    lib().gf_policy_defaults(ctypes.byref(p))
    ladder = kw.pop("ladder", None)
    if ladder is not None:
        if len(ladder) > GF_MAX_LADDER:
            raise ValueError("ladder too long")
        for i, v in enumerate(ladder):
            p.ladder[i] = float(v)
        p.n_ladder = len(ladder)
    for k, v in kw.items():
        if k.startswith("solve_"):
            setattr(p.solve, k[6:], v)
        else:
            setattr(p, k, v)
    return p


def conditioning_screen(lambda_min: float, lambda_max: float, rho_min: float, tau: float = 1e-6) -> float:
    """gf_conditioning_screen: the floor below which kappa * eps exceeds tau (c = kappa rho_min)."""
    out = c_double()
    _check(lib().gf_conditioning_screen(float(lambda_min), float(lambda_max), float(rho_min), float(tau),
                                        ctypes.byref(out)))
    return out.value


def trigger_rule(r50: float, r100: float, policy: Policy | None = None) -> bool:
    p = policy or policy_defaults()
    return bool(_check(lib().gf_trigger_rule(float(r50), float(r100), ctypes.byref(p))))


def probe_features(history, k_stop: int, policy: Policy | None = None):
    p = policy or policy_defaults()
    arr = (c_double * len(history))(*[float(h) for h in history])
    r50, r100 = c_double(), c_double()
    _check(lib().gf_probe_features(arr, int(k_stop), ctypes.byref(p), ctypes.byref(r50), ctypes.byref(r100)))
    return r50.value, r100.value


# ------------------------------------------------------------- device objects ---
def _torch():
    import torch
    return torch


def _ptr(t, dtype, n, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return c_void_p(t.data_ptr())


class Grid:
    """A structured hex8 grid with its level hierarchy and solver workspace (gf_grid)."""

    def __init__(self, nx, ny, nz, h=1.0, E0=1.0, nu=0.3, levels=3, stream=None):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = c_void_p()
        _check(lib().gf_create_grid(int(nx), int(ny), int(nz), float(h), float(E0), float(nu), int(levels),
                                    c_void_p(stream.cuda_stream), ctypes.byref(handle)))
        self._h = handle
        nd, ne, nn, nl = c_int(), c_int(), c_int(), c_int()
        _check(lib().gf_grid_sizes(handle, ctypes.byref(nd), ctypes.byref(ne), ctypes.byref(nn), ctypes.byref(nl)))
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n_dof, self.n_elem, self.n_nodes, self.levels = nd.value, ne.value, nn.value, nl.value
        self.rho_min = None

    def close(self):
        if getattr(self, "_h", None):
            lib().gf_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # state
    def set_density(self, rho_hat, p=3.0):
        _check(lib().gf_set_density(self._h, _ptr(rho_hat, _torch().float64, self.n_elem, "rho_hat"), float(p)))

    def set_floor(self, rho_min):
        _check(lib().gf_set_floor(self._h, float(rho_min)))
        self.rho_min = float(rho_min)

    def set_coarse_operator(self, kind):
        """gf_set_coarse_operator: GF_COARSE_REDISCRETISED or GF_COARSE_GALERKIN, used from
        the next set_floor on (switching clears the floor)."""
        _check(lib().gf_set_coarse_operator(self._h, int(kind)))

    def set_sm_share(self, share):
        """gf_set_sm_share: 1 = launch shapes that leave half of each SM to other grids' solves
        running at once (select_floor_many), 0 = shapes that fill the SMs (default).
        Switching clears the floor."""
        _check(lib().gf_set_sm_share(self._h, int(share)))

    def cantilever_load(self, f):
        _check(lib().gf_cantilever_load(self._h, _ptr(f, _torch().float64, self.n_dof, "f")))
        return f

    def set_geometry(self, kind):
        """gf_set_geometry: GF_GEOM_CANTILEVER (clamped face x = 0) or GF_GEOM_BRIDGE (the
        bridge's point supports and rollers), used from the next set_floor on."""
        _check(lib().gf_set_geometry(self._h, int(kind)))
        self.rho_min = None

    def bridge_load(self, f):
        """gf_bridge_load: the bridge's unit top-face pressure as consistent nodal forces."""
        _check(lib().gf_bridge_load(self._h, _ptr(f, _torch().float64, self.n_dof, "f")))
        return f

    def free_mask(self, mask):
        _check(lib().gf_free_mask(self._h, _ptr(mask, _torch().uint8, self.n_dof, "mask")))
        return mask

    # operator / preconditioner
    def apply_K(self, u, y):
        t = _torch().float64
        _check(lib().gf_apply_K(self._h, _ptr(u, t, self.n_dof, "u"), _ptr(y, t, self.n_dof, "y")))
        return y

    def apply_K_split(self, u, y):
        t = _torch().float64
        _check(lib().gf_apply_K_split(self._h, _ptr(u, t, self.n_dof, "u"), _ptr(y, t, self.n_dof, "y")))
        return y

    def apply_K_f32(self, u, y):
        t = _torch().float32
        _check(lib().gf_apply_K_f32(self._h, _ptr(u, t, self.n_dof, "u"), _ptr(y, t, self.n_dof, "y")))
        return y

    def vcycle(self, v, z, prec=GF_FP64, nu1=2, nu2=2, omega=0.6, smoother=0, ls_ratio=0.0, fine_steps=0,
               coarse_steps=0):
        t = _torch().float64
        if smoother or ls_ratio or fine_steps or coarse_steps:
            o = SolveOpts(30, 0, 0.0, int(prec), int(nu1), int(nu2), float(omega), None, 0, int(smoother),
                          float(ls_ratio), int(fine_steps), int(coarse_steps))
            _check(lib().gf_vcycle_ex(self._h, _ptr(v, t, self.n_dof, "v"), _ptr(z, t, self.n_dof, "z"),
                                      ctypes.byref(o)))
            return z
        _check(lib().gf_vcycle(self._h, _ptr(v, t, self.n_dof, "v"), _ptr(z, t, self.n_dof, "z"), int(prec),
                               int(nu1), int(nu2), float(omega)))
        return z

    def chebyshev_lambda(self, prec=GF_FP64):
        """The Chebyshev smoother's lambda_max estimates of levels 0 .. levels-2."""
        n = max(1, self.levels - 1)
        lam = (c_double * n)()
        _check(lib().gf_chebyshev_lambda(self._h, int(prec), lam, n))
        return [lam[i] for i in range(self.levels - 1)]

    # solve / guard / policy
    def solve(self, f, u, restart=30, kmax=200, tol=1e-6, prec=GF_FP64, nu1=2, nu2=2, omega=0.6,
              want_history=True, outer=0, smoother=0, ls_ratio=0.0, fine_steps=0, coarse_steps=0):
        """gf_solve: FGMRES(restart <= 300) on K(rho_min) u = f from the given u, preconditioned
        by the V-cycle (prec GF_FP64 or GF_MIXED; outer 0/1/2 the Krylov arithmetic; smoother 0
        node-block Jacobi, 1 Chebyshev) and, when set, the adaptive components: ls_ratio (the
        line-searched coarse correction), fine_steps (fine-level inner FGMRES), coarse_steps
        (coarse-level inner Krylov solve). Returns iters, flag, stop_estimate and the history."""
        t = _torch().float64
        hist = (c_double * (kmax + 1))() if want_history else None
        o = SolveOpts(int(restart), int(kmax), float(tol), int(prec), int(nu1), int(nu2), float(omega),
                      ctypes.cast(hist, POINTER(c_double)) if hist is not None else None, int(outer),
                      int(smoother), float(ls_ratio), int(fine_steps), int(coarse_steps))
        info = SolveInfo()
        _check(lib().gf_solve(self._h, _ptr(f, t, self.n_dof, "f"), _ptr(u, t, self.n_dof, "u"),
                              ctypes.byref(o), ctypes.byref(info)))
        out = {"iters": info.iters, "flag": info.flag, "stop_estimate": info.stop_estimate}
        if hist is not None:
            out["history"] = [hist[i] for i in range(info.iters + 1)]
        return out

    def true_residual(self, f, u):
        t = _torch().float64
        eta = c_double()
        _check(lib().gf_true_residual(self._h, _ptr(f, t, self.n_dof, "f"), _ptr(u, t, self.n_dof, "u"),
                                      ctypes.byref(eta)))
        return eta.value

    def select_floor(self, f, u, policy: Policy):
        t = _torch().float64
        info = SelectInfo()
        _check(lib().gf_select_floor(self._h, _ptr(f, t, self.n_dof, "f"), _ptr(u, t, self.n_dof, "u"),
                                     ctypes.byref(policy), ctypes.byref(info)))
        if info.status == GF_ACCEPTED:
            self.rho_min = info.rho_min
        return _select_dict(info)

    def sensitivity(self, u, dc):
        t = _torch().float64
        _check(lib().gf_sensitivity(self._h, _ptr(u, t, self.n_dof, "u"), _ptr(dc, t, self.n_elem, "dc")))
        return dc

    # optimisation loop
    def filter(self, x, xt, r_min=1.5):
        t = _torch().float64
        _check(lib().gf_filter(self._h, _ptr(x, t, self.n_elem, "x"), _ptr(xt, t, self.n_elem, "xt"), float(r_min)))
        return xt

    def filter_adjoint(self, gs, out, r_min=1.5):
        t = _torch().float64
        _check(lib().gf_filter_adjoint(self._h, _ptr(gs, t, self.n_elem, "gs"), _ptr(out, t, self.n_elem, "out"),
                                       float(r_min)))
        return out

    def oc_update(self, x, dc, dv, xnew, volfrac=0.3, move=0.2):
        t = _torch().float64
        n = self.n_elem
        _check(lib().gf_oc_update(self._h, _ptr(x, t, n, "x"), _ptr(dc, t, n, "dc"), _ptr(dv, t, n, "dv"),
                                  float(volfrac), float(move), _ptr(xnew, t, n, "xnew")))
        return xnew

    def compliance(self, f, u):
        t = _torch().float64
        c = c_double()
        _check(lib().gf_compliance(self._h, _ptr(f, t, self.n_dof, "f"), _ptr(u, t, self.n_dof, "u"),
                                   ctypes.byref(c)))
        return c.value

    def oc_iteration(self, x, f, u, policy: Policy, p=3.0, volfrac=0.3, r_min=1.5, move=0.2):
        t = _torch().float64
        info = SelectInfo()
        c = c_double()
        _check(lib().gf_oc_iteration(self._h, _ptr(x, t, self.n_elem, "x"), _ptr(f, t, self.n_dof, "f"),
                                     _ptr(u, t, self.n_dof, "u"), ctypes.byref(policy), float(p), float(volfrac),
                                     float(r_min), float(move), ctypes.byref(info), ctypes.byref(c)))
        atts = [dict(rho_min=a.rho_min, iters=a.iters, flag=a.flag, stop_estimate=a.stop_estimate,
                     eta=a.eta, accepted=bool(a.accepted)) for a in info.attempts[:info.n_attempts]]
        return dict(status=info.status, floor_index=info.floor_index, rho_min=info.rho_min, eta=info.eta,
                    escalated=bool(info.escalated), probe_iters_run=info.probe_iters_run, attempts=atts,
                    compliance=c.value)

    def conditioning(self, f=None, iters=60):
        """gf_conditioning on a one-level grid: extreme eigenvalues of K(rho_min), kappa, and
        (with f) the guard residual of the direct solution."""
        t = _torch().float64
        lo, hi, eta = c_double(), c_double(), c_double()
        fp = _ptr(f, t, self.n_dof, "f") if f is not None else None
        _check(lib().gf_conditioning(self._h, fp, int(iters), ctypes.byref(lo), ctypes.byref(hi),
                                     ctypes.byref(eta) if f is not None else None))
        return dict(lambda_min=lo.value, lambda_max=hi.value, kappa=hi.value / lo.value,
                    eta_direct=eta.value if f is not None else None)

    def features(self, r50, r100):
        return select_features(self._h, r50, r100)

    def set_stencil_blocks(self, tpb64, tpb32):
        _check(lib().gf_set_stencil_blocks(self._h, int(tpb64), int(tpb32)))

    def stats(self):
        s = Stats()
        _check(lib().gf_get_stats(self._h, ctypes.byref(s)))
        return {"kernel_launches": s.kernel_launches, "apply_K_fp64": s.apply_K_fp64, "vcycles": s.vcycles}

    def reset_stats(self):
        _check(lib().gf_reset_stats(self._h))


def true_residual_noalloc(nx, ny, nz, rho_hat, p, rho_min, f, u, eta, h=1.0, E0=1.0, nu=0.3, stream=None):
    """gf_true_residual_noalloc: the FP64 acceptance residual with no device allocation.

    For callers that cannot allocate (graph capture, fixed memory budgets). eta is a
    1-element float64 CUDA tensor that receives the result on the current stream."""
    torch = _torch()
    t = torch.float64
    n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().gf_true_residual_noalloc(
        int(nx), int(ny), int(nz), float(h), float(E0), float(nu),
        _ptr(rho_hat, t, nx * ny * nz, "rho_hat"), float(p), float(rho_min),
        _ptr(f, t, 3 * n_nodes, "f"), _ptr(u, t, 3 * n_nodes, "u"), _ptr(eta, t, 1, "eta"),
        c_void_p(stream.cuda_stream)))
    return eta


def round_to_f32(x, out=None, stream=None):
    """gf_round_to_f32: x (CUDA float64) rounded to float32 by the library's integer routine."""
    torch = _torch()
    n = x.numel()
    out = torch.empty(n, dtype=torch.float32, device=x.device) if out is None else out
    stream = torch.cuda.current_stream() if stream is None else stream
    _check(lib().gf_round_to_f32(_ptr(x, torch.float64, n, "x"), _ptr(out, torch.float32, n, "out"), int(n),
                                 c_void_p(stream.cuda_stream)))
    return out


def widen_to_f64(x, out=None, stream=None):
    """gf_widen_to_f64: x (CUDA float32) widened to float64 by the library's integer routine."""
    torch = _torch()
    n = x.numel()
    out = torch.empty(n, dtype=torch.float64, device=x.device) if out is None else out
    stream = torch.cuda.current_stream() if stream is None else stream
    _check(lib().gf_widen_to_f64(_ptr(x, torch.float32, n, "x"), _ptr(out, torch.float64, n, "out"), int(n),
                                 c_void_p(stream.cuda_stream)))
    return out


def _select_dict(info):
    atts = [dict(rho_min=a.rho_min, iters=a.iters, flag=a.flag, stop_estimate=a.stop_estimate,
                 eta=a.eta, accepted=bool(a.accepted)) for a in info.attempts[:info.n_attempts]]
    checks = [(info.true_check_k[q], info.true_check_est[q], info.true_check_eta[q])
              for q in range(info.n_true_checks)]
    return dict(status=info.status, floor_index=info.floor_index, rho_min=info.rho_min, eta=info.eta,
                r50=info.r50, r100=info.r100, escalated=bool(info.escalated),
                probe_iters_run=info.probe_iters_run, attempts=atts, true_checks=checks,
                true_check_fired=bool(info.true_check_fired))


class Batch:
    """Many frozen states of uneven size solved together (gf_batch)."""

    def __init__(self, dims, levels=3, h=1.0, E0=1.0, nu=0.3, stream=None):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        flat = (c_int * (3 * len(dims)))(*[int(v) for d in dims for v in d])
        handle = c_void_p()
        _check(lib().gf_create_batch(len(dims), flat, int(levels), float(h), float(E0), float(nu),
                                     c_void_p(stream.cuda_stream), ctypes.byref(handle)))
        self._h = handle
        self.dims = [tuple(d) for d in dims]
        self.n_dof = [3 * (d[0] + 1) * (d[1] + 1) * (d[2] + 1) for d in dims]
        self.n_elem = [d[0] * d[1] * d[2] for d in dims]

    def __len__(self):
        return len(self.dims)

    def close(self):
        if getattr(self, "_h", None):
            lib().gf_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, i, rho_hat, f, p=3.0):
        t = _torch().float64
        _check(lib().gf_batch_set_state(self._h, int(i), _ptr(rho_hat, t, self.n_elem[i], "rho_hat"), float(p),
                                        _ptr(f, t, self.n_dof[i], "f")))

    def solution(self, i, u):
        _check(lib().gf_batch_solution(self._h, int(i), _ptr(u, _torch().float64, self.n_dof[i], "u")))
        return u

    def cantilever_load(self, i, f):
        """The cantilever tip load of state i's grid into f (gf_cantilever_load)."""
        gh = c_void_p()
        _check(lib().gf_batch_grid(self._h, int(i), ctypes.byref(gh)))
        _check(lib().gf_cantilever_load(gh, _ptr(f, _torch().float64, self.n_dof[i], "f")))
        return f

    def set_coarse_operator(self, kind):
        """gf_batch_set_coarse_operator: GF_COARSE_REDISCRETISED or GF_COARSE_GALERKIN for every state."""
        _check(lib().gf_batch_set_coarse_operator(self._h, int(kind)))

    def set_sm_share(self, share):
        """gf_batch_set_sm_share: half-SM launch shapes (1) or full-SM ones (0) for every state."""
        _check(lib().gf_batch_set_sm_share(self._h, int(share)))

    def autotune(self):
        out = (c_int * (2 * len(self)))()
        _check(lib().gf_batch_autotune(self._h, out))
        return [(out[2 * i], out[2 * i + 1]) for i in range(len(self))]

    def select_floor(self, policy: Policy):
        infos = (SelectInfo * len(self))()
        _check(lib().gf_batch_select_floor(self._h, ctypes.byref(policy), infos))
        return [_select_dict(infos[i]) for i in range(len(self))]

    def kernel_launches(self):
        n = c_longlong()
        _check(lib().gf_batch_stats(self._h, ctypes.byref(n)))
        return n.value

    def features(self, i, r50, r100):
        gh = c_void_p()
        _check(lib().gf_batch_grid(self._h, int(i), ctypes.byref(gh)))
        return select_features(gh, r50, r100)


class MLP:
    """The learned first-floor selector (gf_mlp): 6 -> 32 -> 32 -> 4, FP32, on the device."""

    def __init__(self, theta0, stream=None):
        import numpy as np
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        th = np.ascontiguousarray(theta0, dtype=np.float32)
        if th.size != MLP_PARAMS:
            raise ValueError(f"theta0 must have {MLP_PARAMS} entries")
        handle = c_void_p()
        _check(lib().gf_mlp_create(th.ctypes.data_as(POINTER(ctypes.c_float)), c_void_p(stream.cuda_stream),
                                   ctypes.byref(handle)))
        self._h = handle

    def close(self):
        if getattr(self, "_h", None):
            lib().gf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_norm(self, mu, sd):
        mu = (ctypes.c_float * 6)(*[float(v) for v in mu])
        sd = (ctypes.c_float * 6)(*[float(v) for v in sd])
        _check(lib().gf_mlp_set_norm(self._h, mu, sd))

    def params(self):
        import numpy as np
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(lib().gf_mlp_get_params(self._h, out.ctypes.data_as(POINTER(ctypes.c_float))))
        return out

    def forward(self, X, logits):
        torch = _torch()
        n = X.shape[0]
        _check(lib().gf_mlp_forward(self._h, _ptr(X, torch.float32, 6 * n, "X"), int(n),
                                    _ptr(logits, torch.float32, 4 * n, "logits")))
        return logits

    def loss_grad(self, X, y):
        import numpy as np
        torch = _torch()
        n = X.shape[0]
        loss = ctypes.c_float()
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(lib().gf_mlp_loss_grad(self._h, _ptr(X, torch.float32, 6 * n, "X"), _ptr(y, torch.int32, n, "y"),
                                      int(n), ctypes.byref(loss), g.ctypes.data_as(POINTER(ctypes.c_float))))
        return loss.value, g

    def train(self, X, y, epochs, batch, lr=1e-3, perm=None):
        import numpy as np
        torch = _torch()
        n = X.shape[0]
        p = None
        if perm is not None:
            perm = np.ascontiguousarray(perm, dtype=np.int32)
            if perm.size != epochs * n:
                raise ValueError("perm must hold epochs * n indices")
            p = perm.ctypes.data_as(POINTER(c_int))
        loss = ctypes.c_float()
        _check(lib().gf_mlp_train(self._h, _ptr(X, torch.float32, 6 * n, "X"), _ptr(y, torch.int32, n, "y"), int(n),
                                  p, int(epochs), int(batch), float(lr), ctypes.byref(loss)))
        return loss.value

    def predict(self, feats):
        import numpy as np
        f = np.ascontiguousarray(feats, dtype=np.float64).reshape(-1, 6)
        cls = np.zeros(f.shape[0], dtype=np.int32)
        _check(lib().gf_mlp_predict(self._h, f.ctypes.data_as(POINTER(c_double)), int(f.shape[0]),
                                    cls.ctypes.data_as(POINTER(c_int))))
        return cls


def _mlp_probs(self, feats):
    import numpy as np
    f = np.ascontiguousarray(feats, dtype=np.float64).reshape(-1, 6)
    p = np.zeros((f.shape[0], 4), dtype=np.float64)
    _check(lib().gf_mlp_probs(self._h, f.ctypes.data_as(POINTER(c_double)), int(f.shape[0]),
                              p.ctypes.data_as(POINTER(c_double))))
    return p


MLP.probs = _mlp_probs


def select_features(grid_handle, r50, r100):
    x = (c_double * 6)()
    _check(lib().gf_select_features(grid_handle, float(r50), float(r100), x))
    return [x[i] for i in range(6)]


def select_floor_many(grids, fs, us, policy: Policy):
    """gf_select_floor_many: Algorithm 1 on several grids at once, one host thread per grid
    (grids created on distinct streams run concurrently); a list of result dicts."""
    t = _torch().float64
    n = len(grids)
    if not (len(fs) == len(us) == n):
        raise ValueError("one f and one u per grid")
    hs = (c_void_p * n)(*[g._h for g in grids])
    fp = (c_void_p * n)(*[_ptr(f, t, g.n_dof, "f") for g, f in zip(grids, fs)])
    up = (c_void_p * n)(*[_ptr(u, t, g.n_dof, "u") for g, u in zip(grids, us)])
    infos = (SelectInfo * n)()
    _check(lib().gf_select_floor_many(n, hs, fp, up, ctypes.byref(policy), infos))
    for g, inf in zip(grids, infos):
        if inf.status == GF_ACCEPTED:
            g.rho_min = inf.rho_min
    return [_select_dict(infos[i]) for i in range(n)]


def create_grid(nx, ny, nz, h=1.0, E0=1.0, nu=0.3, levels=3, stream=None) -> Grid:
    return Grid(nx, ny, nz, h, E0, nu, levels, stream)
