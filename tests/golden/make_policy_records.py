"""Write the oracle's Algorithm-1 record for a smoothed-Gaussian state.

    python tests/golden/make_policy_records.py [--seed 0] [--size c2|c3]

c2: 96x48x48 (policy_c2_seed<seed>.json); c3: 192x96x96 (policy_c3_seed<seed>.json,
about a quarter of an hour of CPU).

Calls only oracle/ (and the seeded generators in synth/). The record (probe
features, candidate floors, per-attempt iterations, flags and recomputed eta) is
a full-size decision fixture for the GPU path (the tests compare the GPU's decision,
floor, iteration counts and features against it).
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import gf_oracle as O  # noqa: E402

WORKLOAD = dict(nx=96, ny=48, nz=48, levels=5, p=3.0, rho0=1e-6, ladder=[1e-5, 1e-4, 1e-3],
                tau=1e-6, kmax=200, probe_iters=100, restart=30, sigma=2.0, floor_frac=0.4)
SIZES = {"c2": dict(nx=96, ny=48, nz=48), "c3": dict(nx=192, ny=96, nz=96)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--size", choices=sorted(SIZES), default="c2")
    args = ap.parse_args()
    w = dict(WORKLOAD, **SIZES[args.size])
    rho = synth.smoothed_gaussian_density(w["nx"], w["ny"], w["nz"], args.seed, w["sigma"], w["floor_frac"])
    m = O.Mesh(w["nx"], w["ny"], w["nz"])
    f = O.cantilever_load(m)
    setup = O.SolverSetup(m, rho, p=w["p"], n_levels=w["levels"], restart=w["restart"])
    t0 = time.time()
    r = O.select_floor(setup, f, w["rho0"], w["ladder"], tau=w["tau"], kmax=w["kmax"],
                       probe_iters=w["probe_iters"])
    rec = dict(workload=w, seed=args.seed, oracle_seconds=time.time() - t0, status=r.status,
               floor_index=r.floor_index, rho_min=r.rho_min, eta=r.eta, r50=r.r50, r100=r.r100,
               escalated=r.escalated, probe_iters_run=r.probe_iters_run,
               attempts=[dict(rho_min=a.rho_min, iters=a.iters, flag=a.flag, stop_estimate=a.stop_estimate,
                              eta=a.eta, accepted=a.accepted) for a in r.attempts])
    out = os.path.join(HERE, f"policy_{args.size}_seed{args.seed}.json")
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
