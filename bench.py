#!/usr/bin/env python
"""Benchmark: guarded solves/s on the 192x96x96 optimised-like cantilever.

One step = one pass of the hot path on one frozen state (Algorithm 1): store the
density, probe at rho0 = 1e-6 for 100 FGMRES iterations, Eq. (trigger), then for
each candidate floor set the floor (moduli, 5-level hierarchy, coarsest inverse),
solve with FGMRES(30) preconditioned by the FP32/BF16 GMG V-cycle with native FP64
Krylov arithmetic (operator, CGS2, Hessenberg, rotations), and accept on the
recomputed FP64 true residual <= 1e-6. value = accepted states / device time.

The states are the 40-iteration SIMP-OC design of this library (vol 0.3, r_min 1.5,
p 3) with a seeded 30 % of voxels forced to the floor; they are made on the device
before the timed region. Beside the headline the line carries the FP64-class
(split-integer, double-float) Krylov form on the same states, the 96x48x48
smoothed-Gaussian workload, and the 102-state comparison of the plain FP64
single-state full ladder with the batched mixed forms (Eq. trigger and the
learned selector).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

N > 1 runs independent replicas (one process per GPU, each on its own states):
states do not exchange data, so the only cross-rank traffic is the barrier and the
max-over-ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF/s of matrix-free K·u; guarded solves/s at true rel. residual ≤1e-6"
UNIT = "guarded solves/s"
LARGE = (192, 96, 96)
LEVELS = 5
MID = (96, 48, 48)
P_SIMP = 3.0
RHO0, LADDER, TAU, KMAX, PROBE, RESTART = 1e-6, [1e-5, 1e-4, 1e-3], 1e-6, 200, 100, 30
FP64_PEAK_NOTE = "derived: 148 SMs x 2 FP64 FMA/clk x 2 flop x sm_max_mhz"
FP32_PEAK_NOTE = "derived: 148 SMs x 128 FP32 FMA/clk x 2 flop x sm_max_mhz"
WORKLOAD = ("cantilever 192x96x96 (5,447,811 DOF), optimised-like density: 40 guarded SIMP-OC iterations "
            "(vol 0.3, linear-hat filter r=1.5, p=3, rho_min 1e-3) then a seeded 30% of voxels forced to "
            "floor; probe at 1e-6, ladder {1e-5,1e-4,1e-3}; FGMRES(30), kmax 200, 5-level GMG (2+2 Jacobi "
            "sweeps, omega 0.6), guard tau=1e-6 on the recomputed FP64 residual")
# the GPU arm's arithmetic (the oracle is FP64 throughout)
GPU_ARITHMETIC = ("FP32/BF16 V-cycle, native FP64 Krylov (K*u, CGS2, Givens), FP64 coarsest solve and guard")
# the oracle's sample: the same recipe at 24x12x12 (3 levels), made by the oracle's own SIMP-OC
CPU_DIMS, CPU_LEVELS = (24, 12, 12), 3
CPU_WORKLOAD = ("cantilever 24x12x12 (12,675 DOF) made by the same recipe with the oracle's own SIMP-OC "
                "(40 iterations, vol 0.3, r=1.5, p=3, rho_min 1e-3) and a seeded 30% forced to floor; "
                "probe at 1e-6, ladder {1e-5,1e-4,1e-3}; FGMRES(30), kmax 200, 3-level GMG; FP64 throughout")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["b300", "reference"], default="b300")
    ap.add_argument("--states", type=int, default=4,
                    help="192x96x96 states per step, solved together through the batch (gf_batch)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-class and 96x48x48 figures")
    ap.add_argument("--no-batch", action="store_true", help="skip the 102-state comparison")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time one complete oracle Algorithm-1 pass on the 96x48x48 state (~2 min)")
    ap.add_argument("--cpu-worker", choices=["passes", "apply", "full_c2"], default=None,
                    help=argparse.SUPPRESS)
    ap.add_argument("--mode", default=None,
                    help="a measurement of bench_modes.py instead of the headline (batch102, oc_loop, oc_reuse, "
                         "true_checks, conditioning, adaptive, false_accept, galerkin, coarse_krylov)")
    args, rest = ap.parse_known_args()
    args.rest = rest
    return args


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def over_ranks(dist, device, maxes, sums):
    """Job-wide figures across ranks: the slowest rank's values (max: times) and the
    totals (sum: units processed, launches). With one process they pass through."""
    if dist is None:
        return [float(v) for v in maxes], [float(v) for v in sums]
    import torch
    t = torch.tensor([float(v) for v in maxes] + [float(v) for v in sums], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    k = len(maxes)
    return [float(v) for v in mx[:k]], [float(v) for v in sm[k:]]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def host_cores():
    """(os.cpu_count(), CPUs this process may run on)."""
    try:
        aff = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = os.cpu_count() or 1
    return os.cpu_count() or 1, aff


def blas_threads():
    """Threads of the BLAS pool this process uses (threadpoolctl where installed, else the
    thread-count environment variables, else every CPU the process may run on)."""
    try:
        from threadpoolctl import threadpool_info
        return max([1] + [int(i.get("num_threads", 1)) for i in threadpool_info()])
    except Exception:
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            if os.environ.get(var, "").isdigit():
                return int(os.environ[var])
        return host_cores()[1]


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def kernel_source_hash(source, start, end):
    """sha1[:16] of the text between two markers of a kernel source file (None if absent)."""
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_2607_26382_b300", "csrc", source)).read()
        a = src.index(start)
        b = src.index(end, a)
    except (OSError, ValueError):
        return None
    return hashlib.sha1(src[a:b].encode()).hexdigest()[:16]


def profiled_traffic(profile, source, start, end):
    """DRAM bytes per launch from a committed ncu summary under profiles/, or None once
    the kernel's source text has changed since the counters were taken."""
    import re
    try:
        prof = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    h = kernel_source_hash(source, start, end)
    m_h = re.search(r"kernel_source_sha1: ([0-9a-f]+)", prof)
    m_t = re.search(r"traffic_bytes_per_launch \| (\d+)", prof)
    if h is None or not m_h or not m_t or m_h.group(1) != h:
        return None
    return int(m_t.group(1))


# kernel text spans hashed for the traffic figures
FP64_KU_SPAN = ("stencil.cuh", "// (i, j, k) of node n", "// First smoothing sweep")
MODAL_SPAN = ("modal.cuh", "// 2D sum/difference transform", "// ---- the FP32 V-cycle's fine-level operator")
MODAL_INSTR, MODAL_FLOPS = 153, 177     # FP64 instructions and flops per element of the modal K*u
FP32_ST_SPAN = FP64_KU_SPAN                # both node-stencil bodies and their shared block update
SPLIT_KU_SPAN = ("split_tc.cuh", "template <bool DD>", "}  // namespace gf")


def emit(d):
    print(json.dumps(d), flush=True)


def state_seeds(rank, n):
    """Seeds of the forced-floor sets of this rank's states: every rank and every state its own."""
    return [1000 * rank + s for s in range(n)]


def pol_of(gf, prec, outer, **kw):
    base = dict(rho0=RHO0, ladder=LADDER, tau=TAU, kmax=KMAX, probe_iters=PROBE, solve_restart=RESTART,
                solve_prec=prec, solve_outer=outer)
    base.update(kw)
    return gf.policy_defaults(**base)


# ----------------------------------------------------------------------------- oracle arm
def oracle_state(seed):
    """The headline's recipe at 24x12x12, made entirely by the oracle (its own guarded
    SIMP-OC loop, then synth's seeded forcing)."""
    import numpy as np
    import synth
    from oracle import gf_oracle as O
    m = O.Mesh(*CPU_DIMS)
    f = O.cantilever_load(m)
    x = np.full(m.n_elem, 0.3)
    kw = dict(rho0=1e-3, ladder=[1e-2], selector="given", first_index=0, tau=TAU, kmax=KMAX)
    for _ in range(40):
        x, _, _ = O.oc_iteration(m, x, f, P_SIMP, 0.3, 1.5, 0.2, kw, CPU_LEVELS)
    rho = np.clip(O.density_filter(O.filter_weights(m, 1.5), x), 0.0, 1.0)
    return m, f, [synth.force_to_floor(rho, 0.3, seed + s) for s in range(2)]


def oracle_pass(m, f, rho):
    """One complete Algorithm-1 pass of the oracle; returns (accepted, seconds, arnoldi steps)."""
    from oracle import gf_oracle as O
    t0 = time.perf_counter()
    setup = O.SolverSetup(m, rho, p=P_SIMP, n_levels=CPU_LEVELS, restart=RESTART)
    r = O.select_floor(setup, f, RHO0, LADDER, tau=TAU, kmax=KMAX, probe_iters=PROBE)
    dt = time.perf_counter() - t0
    steps = sum(a.iters for a in r.attempts) + (r.probe_iters_run if r.escalated else 0)
    return int(r.status == O.ACCEPTED), dt, steps


def oracle_kernel_gdofs(dims):
    """The oracle's FP64 K*u at a full-size grid: one complete application, GDoF/s."""
    import synth
    from oracle import gf_oracle as O
    m = O.Mesh(*dims)
    E = O.young_modulus(synth.uniform_density(*dims, 0), RHO0, P_SIMP)
    u = synth.random_vector(m.n_dof, 1)
    K0 = O.element_stiffness()
    t0 = time.perf_counter()
    O.apply_K(m, E, K0, u)
    return m.n_dof / (time.perf_counter() - t0) / 1e9


def cpu_worker(kind):
    """Runs in a child process whose thread-count variables the parent set: prints one JSON
    line with the timed oracle work of `kind` ("passes", "apply", "full_c2")."""
    if kind == "passes":
        t0 = time.perf_counter()
        m, f, rhos = oracle_state(0)
        t_state = time.perf_counter() - t0
        acc, sec, steps = 0, 0.0, 0
        for rho in rhos * 2:
            a, dt, k = oracle_pass(m, f, rho)
            acc, sec, steps = acc + a, sec + dt, steps + k
        out = {"value": acc / sec, "passes": 2 * len(rhos), "accepted": acc, "seconds": sec,
               "arnoldi_steps": steps, "seconds_state": t_state}
    elif kind == "apply":
        out = {"gdofs": oracle_kernel_gdofs(LARGE)}
    else:
        out = oracle_full_c2()
    out["blas_threads"] = blas_threads()
    print(json.dumps(out), flush=True)


def run_cpu_worker(kind, threads):
    env = dict(os.environ)
    for var in THREAD_VARS:
        env[var] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", kind], env=env,
                       capture_output=True, text=True, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle worker {kind} failed: {r.stderr[-2000:]}")
    return json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])


def cpu_baseline(full_c2=False):
    """Complete oracle Algorithm-1 passes on the 24x12x12 sample in child processes with
    one thread and with every host CPU for BLAS, plus one complete oracle K*u at
    192x96x96. Nothing is extrapolated."""
    ncpu, aff = host_cores()
    runs = {}
    for label, nthreads in (("single_thread", 1), ("all_threads", aff)):
        r = run_cpu_worker("passes", nthreads)
        r["threads"] = nthreads
        runs[label] = r
    gd = run_cpu_worker("apply", 1)["gdofs"]
    best = max(runs.values(), key=lambda r: r["value"])
    out = {"value": best["value"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
           "sample": (f"{best['passes']} complete oracle Algorithm-1 passes (2 states, each twice) on the "
                      f"24x12x12 state of the headline recipe, made by the oracle's own SIMP-OC "
                      f"({best['seconds_state']:.1f} s, untimed); not extrapolated. The bench states are 512x larger"),
           "nproc": ncpu, "affinity_cpus": aff, "runs": runs,
           "apply_K_gdofs_192x96x96": gd,
           "apply_K_note": "one complete oracle FP64 K*u on the 192x96x96 grid, 1 thread"}
    if full_c2:
        out["full_96x48x48"] = run_cpu_worker("full_c2", 1)
    return out


def oracle_full_c2():
    """One complete oracle Algorithm-1 pass on the 96x48x48 smoothed-Gaussian state (seed 0)."""
    import synth
    from oracle import gf_oracle as O
    m = O.Mesh(*MID)
    f = O.cantilever_load(m)
    rho = synth.smoothed_gaussian_density(*MID, 0, 2.0, 0.4)
    t0 = time.perf_counter()
    setup = O.SolverSetup(m, rho, p=P_SIMP, n_levels=5, restart=RESTART)
    r = O.select_floor(setup, f, RHO0, LADDER, tau=TAU, kmax=KMAX, probe_iters=PROBE)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "accepted": int(r.status == O.ACCEPTED), "value": int(r.status == O.ACCEPTED) / dt,
            "unit": UNIT, "iters": [a.iters for a in r.attempts]}


def arm_config(args, world):
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return {"workload": WORKLOAD, "n_dof": 3 * 193 * 97 * 97, "states": args.states,
            "step": (f"one Algorithm-1 pass of each of {args.states} states, solved concurrently by "
                     "gf_select_floor_many (one grid per state, each on its own stream and host thread, "
                     "half-SM launch shapes: gf_set_sm_share)"),
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (Krylov bases V, Z = 2.66 GB per state solve)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
        if rank != 0:
            tdist.destroy_process_group()
            return
    ncpu, aff = host_cores()
    m, f, rhos = oracle_state(0)
    for i in range(args.warmup):
        oracle_pass(m, f, rhos[i % len(rhos)])
    acc, t0 = 0, time.perf_counter()
    for i in range(args.steps):
        a, _, _ = oracle_pass(m, f, rhos[i % len(rhos)])
        acc += a
    dt = time.perf_counter() - t0
    v = acc / dt
    sample = (f"{args.steps} complete oracle Algorithm-1 passes, one per step, on the 24x12x12 state of the "
              f"headline recipe (oracle-made SIMP-OC design, seeded 30% at floor; 512x fewer elements than one "
              f"192x96x96 state); not extrapolated")
    emit({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": arm_config(args, world),
          "sample_config": {"workload": CPU_WORKLOAD, "n_dof": 3 * 25 * 13 * 13},
          "cpu_baseline": {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "sample": sample,
                           "nproc": ncpu, "affinity_cpus": aff},
          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


# ----------------------------------------------------------------------------- GPU arm
def timed_kernel(fn, reps=20):
    """Average duration of fn's launch(es), CUDA events on torch's current stream (the
    grid's stream), after warm-up."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record()
    for _ in range(reps):
        fn()
    k1.record()
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / reps / 1000.0


def large_grids(gf, B):
    """B 192x96x96 grids, each on its own stream with the launch shapes that leave half of
    each SM to the other grids' kernels (set_sm_share), their tip loads and solution vectors."""
    import torch
    streams = [torch.cuda.Stream() for _ in range(B)]
    grids = [gf.create_grid(*LARGE, levels=LEVELS, stream=st) for st in streams]
    for g in grids:
        g.set_sm_share(1)
    fs = [g.cantilever_load(torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")) for g in grids]
    return grids, fs, [torch.zeros_like(f) for f in fs], streams


def concurrent_passes(gf, grids, streams, rhos, fs, us, pol, steps):
    """Algorithm-1 passes of all the states at once, `steps` times: each step sets every
    grid's density (on its own stream) and runs gf_select_floor_many, one host thread per
    grid. CUDA events on the current stream bracket every grid stream's work. (accepted, ms,
    records, Arnoldi steps, FP64 K*u launches)."""
    import torch
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc, iters, recs, kus = 0, 0, [], 0
    torch.cuda.synchronize()
    e0.record(cur)
    for st in streams:
        st.wait_event(e0)
    for _ in range(steps):
        for g, rho in zip(grids, rhos):
            g.set_density(rho, P_SIMP)
        for out in gf.select_floor_many(grids, fs, us, pol):
            acc += int(out["status"] == gf.GF_ACCEPTED)
            iters += sum(a["iters"] for a in out["attempts"]) + (out["probe_iters_run"] if out["escalated"] else 0)
            kus += sum(a["iters"] + 1 for a in out["attempts"])   # Arnoldi K*z, then the guard
            recs.append((out["floor_index"], out["escalated"], [a["iters"] for a in out["attempts"]],
                         [a["accepted"] for a in out["attempts"]]))
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        cur.wait_event(ev)
    e1.record(cur)
    torch.cuda.synchronize()
    return acc, e0.elapsed_time(e1), recs, iters, kus


def large_batch(gf, B):
    """B 192x96x96 cantilever grids in one batch (gf_batch) and their tip loads."""
    import torch
    b = gf.Batch([LARGE] * B, levels=LEVELS)
    b.set_sm_share(1)
    fs = [b.cantilever_load(i, torch.zeros(b.n_dof[i], dtype=torch.float64, device="cuda")) for i in range(B)]
    return b, fs


def batched_passes(gf, b, rhos, fs, pol, steps):
    """Algorithm-1 passes of all the batch's states together, `steps` times (each step sets
    every state's density and load, then gf_batch_select_floor); (accepted, ms, records,
    Arnoldi steps, FP64 K*u launches)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc, iters, recs, kus = 0, 0, [], 0
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        for i in range(len(b)):
            b.set_state(i, rhos[i], fs[i], P_SIMP)
        for out in b.select_floor(pol):
            acc += int(out["status"] == gf.GF_ACCEPTED)
            iters += sum(a["iters"] for a in out["attempts"]) + (out["probe_iters_run"] if out["escalated"] else 0)
            kus += sum(a["iters"] + 1 for a in out["attempts"])   # Arnoldi K*z, then the guard
            recs.append((out["floor_index"], out["escalated"], [a["iters"] for a in out["attempts"]],
                         [a["accepted"] for a in out["attempts"]]))
    e1.record()
    torch.cuda.synchronize()
    return acc, e0.elapsed_time(e1), recs, iters, kus


def single_state_passes(gf, g, rhos, f, u, pol, steps):
    """Algorithm-1 passes over the states in turn; (accepted, ms, records, Arnoldi steps)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc, iters, recs = 0, 0, []
    torch.cuda.synchronize()
    e0.record()
    for i in range(steps):
        g.set_density(rhos[i % len(rhos)], P_SIMP)
        out = g.select_floor(f, u, pol)
        acc += int(out["status"] == gf.GF_ACCEPTED)
        iters += sum(a["iters"] for a in out["attempts"]) + (out["probe_iters_run"] if out["escalated"] else 0)
        recs.append((out["floor_index"], out["escalated"], [a["iters"] for a in out["attempts"]],
                     [a["accepted"] for a in out["attempts"]]))
    e1.record()
    torch.cuda.synchronize()
    return acc, e0.elapsed_time(e1), recs, iters


def comparison_102(gf, dist):
    """The 102 uneven frozen states: plain FP64 single-state full ladder against the
    batched mixed forms with native FP64 Krylov (Eq. trigger; learned selector), and
    the same batched forms with the FP64-class Krylov (outer 2)."""
    import torch
    from paper_2607_26382_b300 import selector as S
    from paper_2607_26382_b300 import workloads as W
    t0 = time.perf_counter()
    dims, rhos_h, kinds = W.batch_states()
    out = {"workload": ("102 frozen cantilever states of uneven size (nx in {32,48,64,80}, ny=nz=nx/2; 72 "
                        "smoothed-Gaussian 40% at floor, 30 SIMP-OC designs with a seeded 30% forced to floor); "
                        "probe at 1e-6, ladder {1e-5,1e-4,1e-3}, FGMRES(30), kmax 200, 4-level GMG, tau 1e-6"),
           "n_dof_total": int(sum(W.n_dof(d) for d in dims)), "states": len(dims),
           "seconds_inputs": time.perf_counter() - t0}
    rhos = [torch.as_tensor(r, device="cuda") for r in rhos_h]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # plain: FP64 V-cycle and Krylov, one state at a time, full ladder from rho0; one grid per size
    grids, loads = {}, {}
    for d in sorted(set(dims)):
        g = gf.create_grid(*d, levels=W.BATCH_LEVELS)
        f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        g.cantilever_load(f)
        grids[d], loads[d] = g, f
    pol_plain = pol_of(gf, gf.GF_FP64, 0, selector=gf.GF_SEL_FULL)
    for d in grids:                                           # warm-up: graphs captured per grid
        i = dims.index(d)
        grids[d].set_density(rhos[i], P_SIMP)
        grids[d].select_floor(loads[d], torch.zeros_like(loads[d]), pol_plain)
    us = {d: torch.zeros_like(loads[d]) for d in grids}
    barrier()
    t0 = time.perf_counter()
    recs = []
    for d, rho in zip(dims, rhos):
        grids[d].set_density(rho, P_SIMP)
        recs.append(grids[d].select_floor(loads[d], us[d], pol_plain))
    barrier()
    dt = time.perf_counter() - t0
    full_floors = [r["floor_index"] for r in recs]

    def summary(recs, dt):
        acc = sum(r["status"] == gf.GF_ACCEPTED for r in recs)
        (dt,), (acc,) = over_ranks(dist, "cuda", [dt], [acc])
        fl = [r["floor_index"] for r in recs]
        return {"value": acc / dt, "unit": UNIT, "accepted": int(acc), "seconds": dt,
                "arnoldi_steps": int(sum(S.work_of(r) for r in recs)),
                "floors_higher_than_full_ladder": int(sum(a > b >= 0 for a, b in zip(fl, full_floors)))}

    out["plain_fp64_single_state_full_ladder"] = summary(recs, dt)
    for g in grids.values():
        g.close()

    net, meta = S.load_trained()
    out["selector"] = {k: meta.get(k) for k in ("states", "train_states", "held_out_accuracy", "label_counts",
                                                "label_form")}
    b = S._batch_for(dims, W.BATCH_LEVELS, rhos_h)
    b.set_sm_share(1)
    b.autotune()
    forms = [("batched_mixed_rule", 0, gf.GF_SEL_RULE), ("batched_mixed_learned", 0, gf.GF_SEL_MLP),
             ("batched_mixed_rule_fp64class", 2, gf.GF_SEL_RULE),
             ("batched_mixed_learned_fp64class", 2, gf.GF_SEL_MLP)]
    for name, outer, sel in forms:
        pol = pol_of(gf, gf.GF_MIXED, outer, selector=sel)
        if sel == gf.GF_SEL_MLP:
            pol.mlp = net.handle
        b.select_floor(pol)                                   # warm-up: graphs captured, buffers sized
        l0 = b.kernel_launches()
        barrier()
        t0 = time.perf_counter()
        recs = b.select_floor(pol)
        barrier()
        out[name] = summary(recs, time.perf_counter() - t0)
        out[name]["gpu_launches"] = b.kernel_launches() - l0
    b.close()
    net.close()
    out["timing"] = "host clock around blocking calls, synchronize on both sides; inputs resident on the device"
    out["speedup_learned_vs_plain"] = (out["batched_mixed_learned"]["value"] /
                                       out["plain_fp64_single_state_full_ladder"]["value"])
    return out


def run_b300(args):
    import torch
    import paper_2607_26382_b300 as gf
    import synth
    from paper_2607_26382_b300 import build as gfbuild
    from paper_2607_26382_b300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    gfbuild.build()

    # ---- inputs (outside the timed region): the SIMP-OC design on the device, then
    # seeded forced floors per state
    t0 = time.perf_counter()
    rhos_h = W.large_states(state_seeds(rank, args.states))
    t_inputs = time.perf_counter() - t0
    rhos = [torch.as_tensor(r, device="cuda") for r in rhos_h]
    B = args.states
    grids, fs, us, streams = large_grids(gf, B)
    pol = pol_of(gf, gf.GF_MIXED, 0)

    concurrent_passes(gf, grids, streams, rhos, fs, us, pol, args.warmup)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clock = ClockSampler(local)
    barrier()
    for g in grids:
        g.reset_stats()
    clock.start()
    accepted, ms, records, iters, kus = concurrent_passes(gf, grids, streams, rhos, fs, us, pol, args.steps)
    barrier()
    clocks = clock.stop()
    launches = sum(g.stats()["kernel_launches"] for g in grids)
    (ms,), (accepted, launches) = over_ranks(dist, "cuda", [ms], [accepted, launches])
    accepted, launches = int(accepted), int(launches)
    value = accepted / (ms / 1000.0)

    # the same states in lockstep through the batch (gf_batch_select_floor)
    b, fs_b = large_batch(gf, B)
    batched_passes(gf, b, rhos, fs_b, pol, 2)
    ab, msb, _, itb, _ = batched_passes(gf, b, rhos, fs_b, pol, args.steps)
    lockstep = {"value": ab / (msb / 1000.0), "unit": UNIT, "steps": args.steps, "accepted": ab,
                "ms_per_step": msb / args.steps, "fgmres_iters_per_step": itb / args.steps,
                "form": (f"the {B} states in lockstep through the batch (gf_batch_select_floor, one CUDA graph per "
                         "FGMRES step)")}
    b.close()

    # the same passes one state at a time through one grid (gf_select_floor)
    g = gf.create_grid(*LARGE, levels=LEVELS)
    f = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    g.cantilever_load(f)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    single_state_passes(gf, g, rhos, f, u, pol, 2)
    a1, ms1, _, it1 = single_state_passes(gf, g, rhos, f, u, pol, args.steps)
    single = {"value": a1 / (ms1 / 1000.0), "unit": UNIT, "passes": args.steps, "accepted": a1,
              "ms_per_pass": ms1 / args.steps, "fgmres_iters_per_pass": it1 / args.steps,
              "form": "one state at a time through one grid (gf_select_floor), same states and policy"}

    # ---- kernels timed alone on the grid's stream (CUDA events, after warm-up)
    g.set_density(rhos[0], P_SIMP)
    g.set_floor(RHO0)
    x = torch.randn(g.n_dof, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    xf, yf = x.float(), torch.empty(g.n_dof, dtype=torch.float32, device="cuda")
    t_kf = timed_kernel(lambda: g.apply_K(x, y))
    t_32f = timed_kernel(lambda: g.apply_K_f32(xf, yf))
    t_s = timed_kernel(lambda: g.apply_K_split(x, y))
    # the headline grids' forms (16x16-column tiles, one CTA per SM), timed alone on grid 0's stream
    g0 = grids[0]
    g0.set_density(rhos[0], P_SIMP)
    g0.set_floor(RHO0)
    with torch.cuda.stream(streams[0]):
        t_k = timed_kernel(lambda: g0.apply_K(x, y))
        t_32 = timed_kernel(lambda: g0.apply_K_f32(xf, yf))
    flops = 1152.0 * g.n_elem                  # 2*24*24 per element and application (dense product)
    sm_max = (clocks or {}).get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2032.0)
    fp64_peak = 148 * 2 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s, FMAs only
    fp32_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12
    hbm = measured_peaks().get("hbm_gbs", 6400.0)
    # the modal K*u executes MODAL_INSTR FP64 instructions per element (45 adds forward,
    # 21 multiplies + 24 FMAs in modal space with the element's scaled coefficients, 54 adds
    # back, 9 adds of the node gather; the constant mode carries no force) = MODAL_FLOPS
    # flops; its ceiling is the FP64 issue rate (2 FP64 instructions per clock and SM) times
    # this mix's flops per instruction. Timed: the kernel and its tile-boundary fix-up.
    modal_flops = MODAL_FLOPS * g.n_elem
    modal_peak = 148 * 2 * sm_max * 1e6 * (MODAL_FLOPS / MODAL_INSTR) / 1e12
    # share of the timed region spent in the native FP64 operator (Arnoldi K*z, cycle-start
    # residuals, guards): its launches in the timed region x its duration timed alone
    share_fp64 = kus * t_k / (ms / 1000.0) if ms > 0 else None
    native = {"bound": "alu", "achieved": modal_flops / t_k / 1e12, "peak": modal_peak, "unit": "TFLOP/s",
              "frac": modal_flops / t_k / 1e12 / modal_peak,
              "traffic": profiled_traffic("apply_modal_kernel_192x96x96.md", *MODAL_SPAN),
              "kernel": ("apply_modal_kernel<16,16> (native FP64 K*u in the sum/difference basis of K0: the "
                         "Krylov operator and the guard; the headline grids' half-SM tiles, timed alone)"),
              "peak_source": ("derived: 148 SMs x 2 FP64 instructions/clk x sm_max_mhz x "
                              f"{MODAL_FLOPS}/{MODAL_INSTR} flop per instruction of this kernel's mix "
                              "(no measured FP64 peak on this pool)"),
              "algorithmic_flops_per_launch": modal_flops, "algorithmic_bytes_per_launch": 18.7 * g.n_dof,
              "dense_equivalent": {"tflops": flops / t_k / 1e12, "fp64_fma_peak": fp64_peak,
                                   "ratio": flops / t_k / 1e12 / fp64_peak,
                                   "note": "1152 flop/element of the dense 24x24 product per launch time"},
              "gdofs": g.n_dof / t_k / 1e9, "ms_per_launch": t_k * 1e3,
              "launches_in_timed_region": kus, "share_of_timed_region_est": share_fp64}
    stencil = {"bound": "alu", "achieved": flops / t_32 / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
               "frac": flops / t_32 / 1e12 / fp32_peak,
               "traffic": None,
               "kernel": ("modal_stencil_f32_kernel<16,16> (the FP32 V-cycle's fine-level operator in the sum/difference "
                          "basis; achieved and frac in dense-equivalent flops, 1152 per element, against the FP32 "
                          "FMA peak: it executes ~171 FP32 instructions per element and is issue-bound)"),
               "peak_source": FP32_PEAK_NOTE, "gdofs": g.n_dof / t_32 / 1e9, "ms_per_launch": t_32 * 1e3}
    split = {"bound": "hbm", "achieved": 7.36e6 * (g.n_dof / 698691.0) / t_s / 1e9, "peak": hbm, "unit": "GB/s",
             "kernel": "apply_split_tc_kernel (split-integer FP64-class K*u, the outer-2 form)",
             "gdofs": g.n_dof / t_s / 1e9, "ms_per_launch": t_s * 1e3,
             "note": "against HBM: its bytes are u, y and the moduli (~10.5 B/DOF); it is issue-bound, far under"}
    split["frac"] = split["achieved"] / hbm
    full_sm = {"ms_per_launch": t_kf * 1e3, "achieved": modal_flops / t_kf / 1e12, "unit": "TFLOP/s",
               "frac": modal_flops / t_kf / 1e12 / modal_peak, "gdofs": g.n_dof / t_kf / 1e9,
               "fp32_stencil_ms_per_launch": t_32f * 1e3,
               "kernel": ("apply_modal_kernel with the full-SM tiles (32x16 or 16x32 columns, one CTA fills an SM): "
                          "the single-state form, same peak")}
    roofline = dict(native)
    roofline["other_kernels"] = {"vcycle_stencil_fp32": stencil, "split_operator": split,
                                 "apply_modal_full_sm": full_sm}

    extras = {"single_state_192x96x96": single, "batched_lockstep_192x96x96": lockstep}
    if not args.no_extras:
        # the FP64-class Krylov form on the same states (split-integer operator, double-float CGS2)
        single_state_passes(gf, g, rhos, f, u, pol_of(gf, gf.GF_MIXED, 2), 1)
        a2, ms2, rec2, it2 = single_state_passes(gf, g, rhos, f, u, pol_of(gf, gf.GF_MIXED, 2), args.states * 2)
        extras["fp64class_krylov_192x96x96"] = {
            "value": a2 / (ms2 / 1000.0), "unit": UNIT, "passes": args.states * 2, "accepted": a2,
            "fgmres_iters_per_pass": it2 / (args.states * 2), "records": rec2,
            "form": ("outer 2: split-integer K*u (~2^-48 of |K||u|) and double-float CGS2 (~2^-47); one state at a "
                     "time"),
            "caution": ("at rho0 = 1e-12 this form stops on a projected estimate the FP64 guard rejects on 27-28 of "
                        "102 states (native FP64: 0); the guard keeps acceptance correct")}
    g.close()
    if not args.no_extras:
        g2 = gf.create_grid(*MID, levels=LEVELS)
        f2 = torch.zeros(g2.n_dof, dtype=torch.float64, device="cuda")
        g2.cantilever_load(f2)
        u2 = torch.zeros_like(f2)
        r2 = [torch.as_tensor(synth.smoothed_gaussian_density(*MID, 1000 * rank + s, 2.0, 0.4), device="cuda")
              for s in range(4)]
        for outer in (0, 2):
            p2 = pol_of(gf, gf.GF_MIXED, outer)
            single_state_passes(gf, g2, r2, f2, u2, p2, 2)
            a, m2, rec, it = single_state_passes(gf, g2, r2, f2, u2, p2, 8)
            extras[f"smoothed_gaussian_96x48x48_outer{outer}"] = {
                "value": a / (m2 / 1000.0), "unit": UNIT, "passes": 8, "accepted": a,
                "fgmres_iters_per_pass": it / 8, "records": rec}
        x2 = torch.randn(g2.n_dof, dtype=torch.float64, device="cuda")
        y2 = torch.empty_like(x2)
        g2.set_density(r2[0], P_SIMP)
        g2.set_floor(RHO0)
        extras["apply_K_fp64_gdofs_96x48x48"] = g2.n_dof / timed_kernel(lambda: g2.apply_K(x2, y2)) / 1e9
        g2.close()

    batch = None
    if not args.no_batch:
        batch = comparison_102(gf, dist)

    # ---- end to end through the public API with host buffers (pinned), 192x96x96: the
    # concurrent passes, every state's density and load uploaded and its solution read back
    e2e = None
    if not args.no_e2e:
        rho_pin = [torch.as_tensor(r).pin_memory() for r in rhos_h]
        f_pin = fs[0].cpu().pin_memory()
        n_dof, n_elem = grids[0].n_dof, grids[0].n_elem
        # double-buffered device inputs and solutions: step s+1's inputs go up and step s's
        # solutions come back on a copy stream while the neighbouring step solves
        rho_d = [[torch.empty(n_elem, dtype=torch.float64, device="cuda") for _ in range(B)] for _ in range(2)]
        f_d = [[torch.empty(n_dof, dtype=torch.float64, device="cuda") for _ in range(B)] for _ in range(2)]
        u_d = [[torch.empty(n_dof, dtype=torch.float64, device="cuda") for _ in range(B)] for _ in range(2)]
        u_pin = [[torch.empty(n_dof, dtype=torch.float64).pin_memory() for _ in range(B)] for _ in range(2)]
        copy_stream = torch.cuda.Stream()
        barrier()
        t0 = time.perf_counter()
        acc_e2e = 0

        def upload(s):
            with torch.cuda.stream(copy_stream):
                for i in range(B):
                    rho_d[s % 2][i].copy_(rho_pin[i], non_blocking=True)
                    f_d[s % 2][i].copy_(f_pin, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            return ev

        ready = upload(0)
        fetched = [None, None]
        for s in range(args.steps):
            ready.synchronize()                      # step s's inputs are on the device
            if fetched[s % 2] is not None:
                fetched[s % 2].synchronize()         # step s-2's solutions have left u_d[s % 2]
            if s + 1 < args.steps:
                ready = upload(s + 1)                # overlaps step s's solve
            for i, gr in enumerate(grids):
                gr.set_density(rho_d[s % 2][i], P_SIMP)
            # returns once every grid's pass is done (each grid synchronises its stream)
            outs = gf.select_floor_many(grids, f_d[s % 2], u_d[s % 2], pol)
            with torch.cuda.stream(copy_stream):     # overlaps step s+1's solve
                for i in range(B):
                    u_pin[s % 2][i].copy_(u_d[s % 2][i], non_blocking=True)
                fetched[s % 2] = torch.cuda.Event()
                fetched[s % 2].record(copy_stream)
            acc_e2e += sum(int(o["status"] == gf.GF_ACCEPTED) for o in outs)
        copy_stream.synchronize()
        torch.cuda.synchronize()
        barrier()
        dt = time.perf_counter() - t0
        (dt,), (acc_e2e,) = over_ranks(dist, "cuda", [dt], [acc_e2e])
        e2e = {"value": int(acc_e2e) / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * B * (n_elem + n_dof),
               "d2h_bytes_per_step": 8 * B * n_dof,
               "note": ("pinned host buffers; every step uploads each state's density and load and reads back "
                        "its solution; step s+1's uploads and step s's downloads run on a copy stream during "
                        "the neighbouring solves (double-buffered device inputs and solutions)")}
    for gr in grids:
        gr.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_full)
    if rank == 0:
        emit({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64 (Krylov, guard, coarsest) / f32+bf16 (V-cycle)",
              "data": "synthetic",
              "config": arm_config(args, world), "arithmetic": GPU_ARITHMETIC, "seconds_inputs": t_inputs,
              "accepted": accepted, "fgmres_iters_per_step": iters / args.steps, "records": records,
              "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e,
              "cpu_baseline": cpu, "apply_K_fp64_gdofs": native["gdofs"], "apply_K_split_gdofs": split["gdofs"],
              "apply_K_fp32_gdofs": stencil["gdofs"], "extras": extras, "comparison_102": batch})
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.mode:
        from paper_2607_26382_b300 import build as gfbuild
        import bench_modes
        gfbuild.build()
        bench_modes.main([args.mode] + args.rest)
    elif args.cpu_worker:
        cpu_worker(args.cpu_worker)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_b300(args)


if __name__ == "__main__":
    main()
