"""Measurement modes of bench.py beyond the headline (every solve runs in libgf_b300.so).

    python bench.py --mode batch102 [--train 0]
    python bench.py --mode oc_loop [--iters 40]
    python bench.py --mode oc_reuse [--iters 40]
    python bench.py --mode true_checks
    python bench.py --mode conditioning
    python bench.py --mode adaptive
    python bench.py --mode false_accept
    python bench.py --mode galerkin
    python bench.py --mode coarse_krylov

Each prints one JSON line of its own (not the headline's contract line).

batch102: 102 frozen states of uneven size (nx in {32,48,64,80}, ny = nz = nx/2,
  round-robin; 72 smoothed-Gaussian states with 40% of voxels at floor, 30
  optimised-like states: SIMP-OC designs with 30% forced to floor), probe at rho0 = 1e-6, ladder
  {1e-5, 1e-4, 1e-3}, tau = 1e-6, kmax = 200, 4-level GMG. Three forms, all with the
  FP64 recomputed-residual guard as the only acceptance test:
    plain   - FP64 V-cycle and Krylov, one state at a time, full ladder from rho0;
    batched - mixed V-cycle, split-integer Krylov operator and double-float CGS2
              (outer = 2), all states in one batch,
              Eq. (trigger) picks the first floor;
    learned - as batched, with an MLP (trained on full-ladder outcomes of 48x24x24
              states; the package's selector_weights.json unless --train N retrains on
              N states) picking the first floor: its most probable floor, and (c0.9)
              the highest floor it is 90% sure the search must reach.
oc_loop: a guarded SIMP-OC loop (vol 0.3, filter radius 1.5, p = 3, move 0.2) on the
  96x48x48 cantilever, Algorithm 1 at every iteration, compared across selectors: the
  plain FP64 full ladder, the mixed form with Eq. (trigger) and with the learned selector
  (native FP64 Krylov), and the latter two with the FP64-class Krylov.
oc_reuse: the in-loop settings of Section 4.1.2 (rho0 = 1e-12, ladder {1e-3, 1e-2},
  kmax = 300, tau = 1e-6) on the same loop with the p continuation 1.5 -> 3.5 after
  iteration 15 (no Heaviside projection), mixed solves. Three guarded selectors:
    rule  - Algorithm 1 at every iteration;
    reuse - Algorithm 1 at iteration 0, then the previous decision without a probe,
            Algorithm 1 again only when the guard rejects it (GF_SEL_REUSE);
    fixed - 1e-3 at every iteration (GF_SEL_GIVEN), still guarded.
true_checks: the 102 batch102 states one at a time (mixed, outer = 2), Algorithm 1 with
  and without true-residual checks every 25 probe steps (detector ratio 10), at the
  workload's floors (rho0 1e-6, ladder {1e-5, 1e-4, 1e-3}) and at the paper's
  (rho0 1e-12, ladder {1e-3, 1e-2}, kmax 300): detector firings, the largest
  eta / estimate ratio seen, decisions that change, and the cost.
conditioning: the reduced floor-conditioning diagnostic of Sec. 4.1.3 on the 24x12x6
  cantilever (6,825 DOF, one level: dense FP64 inverse by Gauss-Jordan), 18 fields
  (9 Bernoulli, q in {0.08..0.35}, 9 smoothed-Gaussian) x 8 floors (1e-12 .. 1e-2),
  p = 4.5: kappa from Lanczos (60 steps on K and on the inverse), the direct
  solution's guard residual, the log-log fit of residual against kappa * eps, the
  split at kappa * eps = tau, and c = kappa * rho_min per field.
adaptive: the paper's adaptive preconditioner components (Table solver-config) against
  the plain V-cycle, Algorithm 1 in the mixed form: the line-searched coarse
  correction (ls_ratio 0.1) and the fine-level correction (fine_steps 20) on the four
  96x48x48 bench states (outer 2) and on the 102 batch102 states one at a time
  (outer 0) at rho0 1e-6 and 1e-12: FGMRES iterations, floors, accepted states, time.
false_accept: the projected-versus-true stopping mismatch of Sec. 4.1.1 on regenerated
  Bernoulli states: the 80x40x20 cantilever (3 levels), seeds 41..71 with the void
  fraction q cycling over {0.08 .. 0.35}, p = 4.5, rho0 = 1e-12, tau = 1e-6,
  k_max = restart = 300 (one Arnoldi cycle). Per solver form: the rho0 solve's flag,
  steps, final projected estimate and FP64 recomputed residual (a false acceptance is a
  converged flag with eta > tau), then Algorithm 1 with Eq. (trigger) and the ladder
  {1e-3, 1e-2}. Forms: FP64 with the fixed V-cycle (the paper's fixed-preconditioner
  control), FP64 with the adaptive preconditioner (line search 0.1, fine correction 20),
  the mixed V-cycle with the split-integer Krylov operator and FP64 CGS2 (outer 1), and
  FP64 with all three adaptive components (plus the coarse Krylov solve, 10 steps).
galerkin: rediscretised against Galerkin coarse operators (gf_set_coarse_operator) on
  the four 96x48x48 bench states at rho_min 1e-6 and 1e-3, 5 levels, FGMRES(30) to
  1e-6: steps, time per step and per V-cycle, mixed (outer 2) and FP64; plus the
  Galerkin hierarchy's set-up time (gf_set_floor).
coarse_krylov: the coarsest level solved exactly against 10 inner FGMRES steps
  (coarse_steps, Table solver-config's coarse level), and the paper's whole adaptive
  preconditioner (line search 0.1, fine correction 20, coarse Krylov 10), on the four
  96x48x48 bench states at rho_min 1e-6 and 1e-3: steps, time per step, accepted
  (FP64 recomputed residual <= 1e-6), mixed (outer 2) and FP64.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from paper_2607_26382_b300 import _lib as L
from paper_2607_26382_b300 import selector as S
from paper_2607_26382_b300 import workloads as W

LADDER = [1e-5, 1e-4, 1e-3]


def _policy(**kw):
    base = dict(rho0=1e-6, ladder=LADDER, tau=1e-6, kmax=200, probe_iters=100)
    base.update(kw)
    return L.policy_defaults(**base)


def batch_states(n=102, seed0=100):
    return W.batch_states(n, seed0)


def batch_states_tapered(n=102, seed0=100):
    """The earlier batch102 mix whose optimised-like states are synth's tapered-bar fields
    (the true_checks and adaptive measurements were recorded on it)."""
    import synth
    dims = synth.batch_grid_sizes(n)
    rhos, kinds = [], []
    for i, (nx, ny, nz) in enumerate(dims):
        if i % 10 < 7:
            rhos.append(synth.smoothed_gaussian_density(nx, ny, nz, seed0 + i, 2.0, 0.4))
            kinds.append("random")
        else:
            rhos.append(synth.optimised_like_density(nx, ny, nz, seed0 + 100 + i, 0.3, 0.3))
            kinds.append("optimised")
    return dims, rhos, kinds


def _summary(recs, seconds):
    acc = sum(r["status"] == L.GF_ACCEPTED for r in recs)
    return {"states": len(recs), "accepted": acc, "seconds": seconds, "guarded_solves_per_s": acc / seconds,
            "arnoldi_steps": int(sum(S.work_of(r) for r in recs)),
            "floors": [r["floor_index"] for r in recs]}


def run_plain(dims, rhos):
    import torch
    pol = _policy(selector=L.GF_SEL_FULL, solve_prec=L.GF_FP64, solve_outer=0)
    recs = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d, rho in zip(dims, rhos):
        g = L.create_grid(*d, levels=4)
        f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.cantilever_load(f)
        g.set_density(torch.as_tensor(rho, device="cuda"), 3.0)
        u = torch.zeros_like(f)
        recs.append(g.select_floor(f, u, pol))
        g.close()
    torch.cuda.synchronize()
    return recs, time.perf_counter() - t0


def run_batched(dims, rhos, pol, reps=1):
    import torch
    b = S._batch_for(dims, 4, rhos)
    b.autotune()
    b.select_floor(pol)                      # warm-up: graphs captured, buffers sized
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        recs = b.select_floor(pol)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    launches = b.kernel_launches()
    b.close()
    return recs, dt, launches


def train_mlp(n_train, seed=7):
    """The selector: the committed weights (n_train == 0), or one trained here on n_train
    full-ladder outcomes at 48x24x24 (the mix of train_selector)."""
    import synth
    if n_train <= 0:
        net, meta = S.load_trained()
        return net, meta
    dims = (48, 24, 24)
    rh = synth.selector_training_states(n_train, dims, seed, designs=W.selector_designs(dims))
    pol = _policy(solve_prec=L.GF_MIXED, solve_outer=0)
    t0 = time.perf_counter()
    X, y, _ = S.ladder_dataset(dims, rh, 4, pol, chunk=100)
    t_data = time.perf_counter() - t0
    ntr = int(0.8 * len(y))
    perm = synth.epoch_permutations(ntr, 200, seed + 1)
    net, loss = S.train_selector(X[:ntr], y[:ntr], synth.mlp_init(seed + 2), perm, 200, 128, 3e-3)
    acc = float((net.predict(X[ntr:]) == y[ntr:]).mean())
    return net, {"train_states": ntr, "held_out": len(y) - ntr, "label_counts": np.bincount(y, minlength=4).tolist(),
                 "held_out_accuracy": acc, "final_loss": loss, "data_seconds": t_data}


def batch102(args):
    dims, rhos, kinds = batch_states()
    out = {"workload": "batch102", "n_dof_total": int(sum(3 * (a + 1) * (b + 1) * (c + 1) for a, b, c in dims))}
    recs, dt = run_plain(dims, rhos)
    out["plain_fp64_single_state_full_ladder"] = _summary(recs, dt)
    recs, dt, launches = run_batched(dims, rhos, _policy(solve_prec=L.GF_MIXED, solve_outer=2))
    out["batched_mixed_rule"] = _summary(recs, dt)
    out["batched_mixed_rule"]["kernel_launches_total"] = launches
    net, info = train_mlp(args.train)
    out["selector_training"] = info
    for name, conf in (("batched_mixed_learned", 0.0), ("batched_mixed_learned_c0.9", 0.9)):
        pol = _policy(solve_prec=L.GF_MIXED, solve_outer=2, selector=L.GF_SEL_MLP, mlp_confidence=conf)
        pol.mlp = net.handle
        recs, dt, _ = run_batched(dims, rhos, pol)
        out[name] = _summary(recs, dt)
    full = out["plain_fp64_single_state_full_ladder"]["floors"]
    for k in ("batched_mixed_rule", "batched_mixed_learned", "batched_mixed_learned_c0.9"):
        fl = out[k]["floors"]
        out[k]["floors_higher_than_full_ladder"] = int(sum(a > b >= 0 for a, b in zip(fl, full)))
    out["speedup_learned_vs_plain"] = (out["batched_mixed_learned"]["guarded_solves_per_s"] /
                                       out["plain_fp64_single_state_full_ladder"]["guarded_solves_per_s"])
    return out


def oc_loop(args):
    import torch
    nx, ny, nz = 96, 48, 48
    out = {"workload": f"guarded SIMP-OC {nx}x{ny}x{nz}, {args.iters} iterations, vol 0.3, r_min 1.5, p 3"}
    modes = [("plain_fp64_full", _policy(selector=L.GF_SEL_FULL, solve_prec=L.GF_FP64, solve_outer=0)),
             ("mixed_rule", _policy(solve_prec=L.GF_MIXED, solve_outer=0)),
             ("mixed_rule_fp64class", _policy(solve_prec=L.GF_MIXED, solve_outer=2))]
    net = None
    if args.train >= 0:
        net, info = train_mlp(args.train)
        out["selector_training"] = {k: v for k, v in info.items() if k in ("states", "train_states", "held_out_accuracy",
                                                                            "label_counts", "label_form")}
        for name, outer in (("mixed_learned", 0), ("mixed_learned_fp64class", 2)):
            pol = _policy(solve_prec=L.GF_MIXED, solve_outer=outer, selector=L.GF_SEL_MLP)
            pol.mlp = net.handle
            modes.append((name, pol))
    for name, pol in modes:
        g = L.create_grid(nx, ny, nz, levels=5)
        f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.cantilever_load(f)
        x = torch.full((g.n_elem,), 0.3, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        hist = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(args.iters):
            r = g.oc_iteration(x, f, u, pol, p=3.0, volfrac=0.3, r_min=1.5, move=0.2)
            hist.append(r)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        acc = sum(r["status"] == L.GF_ACCEPTED for r in hist)
        out[name] = {"seconds": dt, "accepted": acc, "guarded_solves_per_s": acc / dt,
                     "arnoldi_steps": int(sum(sum(a["iters"] for a in r["attempts"]) for r in hist)),
                     "floors": [r["floor_index"] for r in hist],
                     "compliance_first_last": [hist[0]["compliance"], hist[-1]["compliance"]]}
        g.close()
    return out


def oc_reuse(args):
    import torch
    nx, ny, nz = 96, 48, 48
    cont = 15
    out = {"workload": f"guarded SIMP-OC {nx}x{ny}x{nz}, {args.iters} iterations, vol 0.3, r_min 1.5, "
                       f"p 1.5 -> 3.5 after iteration {cont}, rho0 1e-12, ladder [1e-3, 1e-2], kmax 300"}
    base = dict(rho0=1e-12, ladder=[1e-3, 1e-2], tau=1e-6, kmax=300, probe_iters=100,
                solve_prec=L.GF_MIXED, solve_outer=2)
    for name in ("rule", "reuse", "fixed"):
        g = L.create_grid(nx, ny, nz, levels=5)
        f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.cantilever_load(f)
        x = torch.full((g.n_elem,), 0.3, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        hist = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(args.iters):
            if name == "fixed":
                pol = L.policy_defaults(selector=L.GF_SEL_GIVEN, first_index=1, **base)
            elif name == "reuse" and hist:
                pol = L.policy_defaults(selector=L.GF_SEL_REUSE, first_index=max(hist[-1]["floor_index"], 0),
                                        **base)
            else:
                pol = L.policy_defaults(selector=L.GF_SEL_RULE, **base)
            p = 1.5 if it < cont else 3.5
            hist.append(g.oc_iteration(x, f, u, pol, p=p, volfrac=0.3, r_min=1.5, move=0.2))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        acc = [r for r in hist if r["status"] == L.GF_ACCEPTED]
        out[name] = {"seconds": dt, "accepted": len(acc), "guarded_solves_per_s": len(acc) / dt,
                     "arnoldi_steps": int(sum(sum(a["iters"] for a in r["attempts"]) for r in hist)),
                     "probe_steps": int(sum(r["probe_iters_run"] for r in hist)),
                     "attempts": int(sum(len(r["attempts"]) for r in hist)),
                     "max_accepted_eta": max((r["eta"] for r in acc), default=None),
                     "floors": [r["floor_index"] for r in hist],
                     "compliance_last": hist[-1]["compliance"]}
        g.close()
    return out


def true_checks(args):
    import torch
    dims, rhos, kinds = batch_states_tapered()
    out = {"workload": f"{len(dims)} batch102 states one at a time, checks every 25 probe steps, ratio 10"}
    mixed = dict(solve_prec=L.GF_MIXED, solve_outer=2)
    for tag, base in (("workload floors", dict(rho0=1e-6, ladder=LADDER, kmax=200, **mixed)),
                      ("paper floors", dict(rho0=1e-12, ladder=[1e-3, 1e-2], kmax=300, **mixed)),
                      ("paper floors, FP64", dict(rho0=1e-12, ladder=[1e-3, 1e-2], kmax=300,
                                                  solve_prec=L.GF_FP64, solve_outer=0))):
        rec = {}
        for every in (0, 25):
            t_total, fired, changed, worst, floors, n_checks = 0.0, 0, 0, 0.0, [], 0
            steps, rule_esc, rho0_rejected, fired_and_rule, false_acc, visible = 0, 0, 0, 0, 0, 0
            for (nx, ny, nz), rho in zip(dims, rhos):
                g = L.create_grid(nx, ny, nz, levels=4)
                g.set_density(torch.as_tensor(rho, device="cuda"), 3.0)
                f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
                g.cantilever_load(f)
                u = torch.zeros_like(f)
                pol = _policy(true_check_every=every, true_check_ratio=10.0, **base)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = g.select_floor(f, u, pol)
                torch.cuda.synchronize()
                t_total += time.perf_counter() - t0
                floors.append(r["floor_index"])
                fired += int(r["true_check_fired"])
                steps += sum(a["iters"] for a in r["attempts"])
                tr = L.trigger_rule(r["r50"], r["r100"], pol)
                rule_esc += int(tr)
                fired_and_rule += int(tr and r["true_check_fired"])
                rho0_rejected += int(any(a["rho_min"] == base["rho0"] and not a["accepted"] for a in r["attempts"]))
                # a rejected attempt whose stopping flag said converged: a false acceptance by
                # the solver's own estimate (Sec. 4.1.1); else the failure was visible
                false_acc += sum(a["flag"] == L.GF_FLAG_CONVERGED and not a["accepted"] for a in r["attempts"])
                visible += sum(a["flag"] != L.GF_FLAG_CONVERGED and not a["accepted"] for a in r["attempts"])
                n_checks += len(r["true_checks"])
                for _, est, eta in r["true_checks"]:
                    worst = max(worst, eta / est)
                g.close()
            rec[f"every {every}"] = {"seconds": t_total, "guarded_solves_per_s": len(dims) / t_total,
                                     "detector_fired": fired, "rule_escalated": rule_esc,
                                     "fired_where_rule_escalated": fired_and_rule,
                                     "rho0_solved_and_rejected_by_guard": rho0_rejected, "arnoldi_steps": steps,
                                     "false_acceptances": false_acc, "visible_failures": visible,
                                     "checks": n_checks, "max_eta_over_estimate": worst, "floors": floors}
        a, b = rec["every 0"]["floors"], rec["every 25"]["floors"]
        rec["decisions_changed"] = sum(x != y for x, y in zip(a, b))
        rec["overhead"] = rec["every 25"]["seconds"] / rec["every 0"]["seconds"] - 1.0
        out[tag] = rec
    return out


def conditioning(args):
    import torch
    import synth
    nx, ny, nz = 24, 12, 6
    floors = [1e-12, 1e-10, 1e-8, 1e-7, 1e-6, 1e-5, 1e-4, 1e-2]
    qs = [0.08, 0.11, 0.14, 0.17, 0.20, 0.23, 0.26, 0.30, 0.35]
    fields = [("bernoulli", synth.bernoulli_density(nx, ny, nz, 41 + 2 * i, q)) for i, q in enumerate(qs)]
    fields += [("gaussian", synth.smoothed_gaussian_density(nx, ny, nz, 200 + i, 1.5, 0.3 + 0.05 * i)) for i in range(9)]
    eps, tau = 2.0 ** -52, 1e-6
    g = L.create_grid(nx, ny, nz, levels=1)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    rows, t0 = [], time.perf_counter()
    for kind, rho in fields:
        g.set_density(torch.as_tensor(rho, device="cuda"), 4.5)
        for rm in floors:
            g.set_floor(rm)
            o = g.conditioning(f, iters=60)
            rows.append(dict(kind=kind, rho_min=rm, kappa=o["kappa"], eta=o["eta_direct"], c=o["kappa"] * rm))
    secs = time.perf_counter() - t0
    g.close()
    k_eps = np.array([r["kappa"] * eps for r in rows])
    eta = np.array([r["eta"] for r in rows])
    x, y = np.log10(k_eps), np.log10(np.maximum(eta, 1e-300))
    def fit(mask):
        A = np.vstack([x[mask], np.ones(mask.sum())]).T
        slope = float(np.linalg.lstsq(A, y[mask], rcond=None)[0][0])
        return {"n": int(mask.sum()), "slope": slope, "corr": float(np.corrcoef(x[mask], y[mask])[0, 1])}
    floor_ = eta <= 1e-14                        # at the backward-stability floor
    below = k_eps <= tau
    cs = {}
    for i in range(len(fields)):
        c = [r["c"] for r in rows[i * len(floors):(i + 1) * len(floors)]]
        c_small = c[:5]                          # floors 1e-12 .. 1e-6
        cs[i] = max(c_small) / min(c_small)
    return {"workload": f"24x12x6 cantilever, {len(fields)} fields x {len(floors)} floors, p 4.5",
            "seconds": secs, "matrices": len(rows),
            "kappa_range_at_1e-12": [min(r["kappa"] for r in rows if r["rho_min"] == 1e-12),
                                     max(r["kappa"] for r in rows if r["rho_min"] == 1e-12)],
            "fit_all": fit(np.ones(len(rows), bool)), "fit_above_stability_floor": fit(~floor_),
            "fit_bernoulli": fit(np.array([r["kind"] == "bernoulli" for r in rows])),
            "fit_gaussian": fit(np.array([r["kind"] == "gaussian" for r in rows])),
            "at_stability_floor": int(floor_.sum()),
            "kappa_eps_le_tau": {"n": int(below.sum()), "reach_tau": int((eta[below] <= tau).sum())},
            "kappa_eps_gt_tau": {"n": int((~below).sum()), "miss_tau": int((eta[~below] > tau).sum())},
            "upper_envelope_max_eta_over_kappa_eps": float((eta / k_eps).max()),
            "c_spread_1e-12_to_1e-6_per_field_max": float(max(cs.values())),
            "c_spread_median": float(np.median(list(cs.values()))),
            "rows": rows}


def adaptive(args):
    import torch
    import synth
    out = {}
    variants = (("plain", {}), ("line search 0.1", {"solve_ls_ratio": 0.1}), ("fine 20", {"solve_fine_steps": 20}))
    for name, kw in variants:
        t, its, acc, floors = 0.0, 0, 0, []
        for seed in range(4):
            g = L.create_grid(96, 48, 48, levels=5)
            g.set_density(torch.as_tensor(synth.smoothed_gaussian_density(96, 48, 48, seed), device="cuda"), 3.0)
            f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
            g.cantilever_load(f)
            u = torch.zeros_like(f)
            pol = L.policy_defaults(solve_prec=L.GF_MIXED, solve_outer=2, **kw)
            g.select_floor(f, u, pol)                 # warm-up: graphs captured
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = g.select_floor(f, u, pol)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            its += sum(a["iters"] for a in r["attempts"])
            acc += int(r["status"] == L.GF_ACCEPTED)
            floors.append(r["floor_index"])
            g.close()
        out[f"96x48x48 bench states, {name}"] = {"guarded_solves_per_s": 4 / t, "fgmres_iters": its, "accepted": acc,
                                                  "floors": floors, "ms_per_iter": t / its * 1e3}
    dims, rhos, kinds = batch_states_tapered()
    for name, kw in variants:
        for rho0, ladder, kmax in ((1e-6, LADDER, 200), (1e-12, [1e-3, 1e-2], 300)):
            t, its, acc, fl = 0.0, 0, 0, []
            for (nx, ny, nz), rho in zip(dims, rhos):
                g = L.create_grid(nx, ny, nz, levels=4)
                g.set_density(torch.as_tensor(rho, device="cuda"), 3.0)
                f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
                g.cantilever_load(f)
                u = torch.zeros_like(f)
                pol = _policy(rho0=rho0, ladder=ladder, kmax=kmax, solve_prec=L.GF_MIXED, solve_outer=0, **kw)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = g.select_floor(f, u, pol)
                torch.cuda.synchronize()
                t += time.perf_counter() - t0
                its += sum(a["iters"] for a in r["attempts"])
                acc += int(r["status"] == L.GF_ACCEPTED)
                fl.append(r["floor_index"])
                g.close()
            out[f"batch102 single, rho0 {rho0:g}, {name}"] = {
                "seconds": t, "fgmres_iters": its, "accepted": acc,
                "floor_index_counts": [fl.count(i) for i in range(len(ladder) + 1)]}
    return out


def false_accept(args):
    import torch
    import synth
    nx, ny, nz, levels, p, tau, kmax = 80, 40, 20, 3, 4.5, 1e-6, 300
    rho0, ladder = 1e-12, [1e-3, 1e-2]
    qs = [0.08, 0.11, 0.14, 0.17, 0.20, 0.23, 0.26, 0.30, 0.35]
    states = [(seed, qs[i % len(qs)]) for i, seed in enumerate(range(41, 72))]
    forms = (("FP64, fixed V-cycle", dict(prec=L.GF_FP64, outer=0)),
             ("FP64, adaptive (line search 0.1, fine correction 20)",
              dict(prec=L.GF_FP64, outer=0, ls_ratio=0.1, fine_steps=20)),
             ("mixed V-cycle, split-integer K*u, FP64 CGS2", dict(prec=L.GF_MIXED, outer=1)),
             ("FP64, adaptive (line search 0.1, fine correction 20, coarse Krylov 10)",
              dict(prec=L.GF_FP64, outer=0, ls_ratio=0.1, fine_steps=20, coarse_steps=10)))
    if args.forms:
        forms = tuple(forms[int(i)] for i in args.forms.split(","))
    g = L.create_grid(nx, ny, nz, levels=levels)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    out = {"grid": f"{nx}x{ny}x{nz}, {g.n_dof} DOF, {levels} levels", "states": len(states)}
    for name, kw in forms:
        rows, t_solve, t_sel, steps_sel, floors, accepted = [], 0.0, 0.0, 0, [], 0
        for seed, q in states:
            g.set_density(torch.as_tensor(synth.bernoulli_density(nx, ny, nz, seed, q), device="cuda"), p)
            g.set_floor(rho0)
            u = torch.zeros_like(f)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            o = g.solve(f, u, restart=kmax, kmax=kmax, tol=tau, **kw)
            eta = g.true_residual(f, u)
            t_solve += time.perf_counter() - t0
            rows.append((o["flag"], o["iters"], o["history"][o["iters"]], eta))
            pol = L.policy_defaults(rho0=rho0, ladder=ladder, tau=tau, kmax=kmax, probe_iters=100,
                                    selector=L.GF_SEL_RULE, solve_restart=kmax, solve_prec=kw["prec"],
                                    solve_outer=kw["outer"], solve_ls_ratio=kw.get("ls_ratio", 0.0),
                                    solve_fine_steps=kw.get("fine_steps", 0),
                                    solve_coarse_steps=kw.get("coarse_steps", 0))
            u.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = g.select_floor(f, u, pol)
            t_sel += time.perf_counter() - t0
            steps_sel += r["probe_iters_run"] + sum(a["iters"] for a in r["attempts"])
            floors.append(r["floor_index"])
            accepted += int(r["status"] == L.GF_ACCEPTED)
        conv = [(it, est, eta) for fl, it, est, eta in rows if fl == L.GF_FLAG_CONVERGED]
        out[name] = {
            "rho0 solves": {
                "converged_flag": len(conv),
                "false_acceptances": sum(eta > tau for _, _, eta in conv),
                "visible_failures": sum(fl != L.GF_FLAG_CONVERGED for fl, _, _, _ in rows),
                "max_eta_over_estimate": max((eta / est for _, est, eta in conv if est > 0), default=None),
                "steps_mean": float(np.mean([it for _, it, _, _ in rows])),
                "steps_max": max(it for _, it, _, _ in rows),
                "seconds": t_solve},
            "algorithm 1 (Eq. trigger)": {
                "accepted": accepted, "floor_index_counts": [floors.count(i) for i in range(len(ladder) + 1)],
                "arnoldi_steps": steps_sel, "seconds": t_sel}}
        print(name, json.dumps(out[name]), flush=True)
    g.close()
    return out


def galerkin(args):
    import torch
    import synth
    nx, ny, nz, levels = 96, 48, 48, 5
    out = {}
    for kind_name, kind in (("rediscretised", L.GF_COARSE_REDISCRETISED), ("galerkin", L.GF_COARSE_GALERKIN)):
        g = L.create_grid(nx, ny, nz, levels=levels)
        g.set_coarse_operator(kind)
        f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.cantilever_load(f)
        for prec, outer, pname in ((L.GF_MIXED, 2, "mixed"), (L.GF_FP64, 0, "fp64")):
            for rho_min in (1e-6, 1e-3):
                its, t_solve, t_floor, etas = [], 0.0, 0.0, []
                for seed in range(4):
                    g.set_density(torch.as_tensor(synth.smoothed_gaussian_density(nx, ny, nz, seed), device="cuda"), 3.0)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    g.set_floor(rho_min)
                    torch.cuda.synchronize()
                    t_floor += time.perf_counter() - t0
                    u = torch.zeros_like(f)
                    g.solve(f, u, restart=30, kmax=200, prec=prec, outer=outer)    # graphs captured
                    u.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    o = g.solve(f, u, restart=30, kmax=200, prec=prec, outer=outer)
                    torch.cuda.synchronize()
                    t_solve += time.perf_counter() - t0
                    its.append(o["iters"])
                    etas.append(g.true_residual(f, u))
                x = torch.randn(g.n_dof, dtype=torch.float64, device="cuda")
                z = torch.empty_like(x)
                for _ in range(3):
                    g.vcycle(x, z, prec)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(20):
                    g.vcycle(x, z, prec)
                e1.record()
                torch.cuda.synchronize()
                out[f"{kind_name}, {pname}, rho_min {rho_min:g}"] = {
                    "steps": its, "max_eta": max(etas), "ms_per_step": t_solve / sum(its) * 1e3,
                    "vcycle_ms": e0.elapsed_time(e1) / 20, "set_floor_ms": t_floor / 4 * 1e3}
                print(kind_name, pname, rho_min, json.dumps(out[f"{kind_name}, {pname}, rho_min {rho_min:g}"]),
                      flush=True)
        g.close()
    return out


def coarse_krylov(args):
    import torch
    import synth
    nx, ny, nz, levels = 96, 48, 48, 5
    forms = (("exact coarse solve", {}), ("coarse Krylov 10", {"coarse_steps": 10}),
             ("line search 0.1 + fine 20 + coarse Krylov 10", {"coarse_steps": 10, "fine_steps": 20, "ls_ratio": 0.1}))
    g = L.create_grid(nx, ny, nz, levels=levels)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    out = {}
    for prec, outer, pname in ((L.GF_MIXED, 2, "mixed"), (L.GF_FP64, 0, "fp64")):
        for rho_min in (1e-6, 1e-3):
            for name, kw in forms:
                its, t, acc = [], 0.0, 0
                for seed in range(4):
                    g.set_density(torch.as_tensor(synth.smoothed_gaussian_density(nx, ny, nz, seed), device="cuda"), 3.0)
                    g.set_floor(rho_min)
                    u = torch.zeros_like(f)
                    g.solve(f, u, restart=30, kmax=200, prec=prec, outer=outer, **kw)    # graphs captured
                    u.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    o = g.solve(f, u, restart=30, kmax=200, prec=prec, outer=outer, **kw)
                    torch.cuda.synchronize()
                    t += time.perf_counter() - t0
                    its.append(o["iters"])
                    acc += int(g.true_residual(f, u) <= 1e-6)
                key = f"{pname}, rho_min {rho_min:g}, {name}"
                out[key] = {"steps": its, "accepted": acc, "ms_per_step": t / sum(its) * 1e3, "seconds": t}
                print(key, json.dumps(out[key]), flush=True)
    g.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["batch102", "oc_loop", "oc_reuse", "true_checks", "conditioning", "adaptive",
                                     "false_accept", "galerkin", "coarse_krylov"])
    ap.add_argument("--train", type=int, default=0, help="0: the committed selector weights")
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--forms", default="", help="false_accept: comma-separated form indices (default: all)")
    a = ap.parse_args(argv)
    res = {"batch102": batch102, "oc_loop": oc_loop, "oc_reuse": oc_reuse, "true_checks": true_checks,
           "conditioning": conditioning, "adaptive": adaptive, "false_accept": false_accept,
           "galerkin": galerkin, "coarse_krylov": coarse_krylov}[a.what](a)
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

