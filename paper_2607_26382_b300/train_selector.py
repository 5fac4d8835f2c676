"""Train the learned first-floor selector and write its weights.

    python -m paper_2607_26382_b300.train_selector [--states 5000] [--out PATH]

Training mix (48x24x24 cantilevers, 4-level GMG): in turn Bernoulli hard fields,
smoothed-Gaussian fields (floor fraction 0.1-0.6, sigma 1-3) and optimised-like
fields (one of three SIMP-OC designs of this library, volume 0.2 / 0.3 / 0.4, with
a seeded 10-50 % of voxels forced to the floor). Each state runs the full ladder
(rho0 = 1e-6, then 1e-5, 1e-4, 1e-3; FGMRES(30), kmax 200, tau 1e-6) in the batched
solver, in the form the selector is deployed with (mixed V-cycle, native FP64
Krylov); the label is the first floor whose guarded solve is accepted, the
features are the rho0 attempt's r50 / r100 plus density statistics. 80 % of the
states train the network with Adam (200 epochs, minibatch 128, lr 3e-3) in the
library's own forward/backward kernels; 20 % are held out. The default output is
the package's selector_weights.json, which the benchmark loads.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import _lib as L
from . import selector as S
from . import workloads as W

DIMS = (48, 24, 24)
LEVELS = 4


def policy():
    return L.policy_defaults(rho0=1e-6, ladder=[1e-5, 1e-4, 1e-3], tau=1e-6, kmax=200, probe_iters=100,
                             solve_restart=30, solve_prec=L.GF_MIXED, solve_outer=0)


def main(argv=None):
    import synth
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--states", type=int, default=5000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--out", default=S.WEIGHTS)
    args = ap.parse_args(argv)
    build.build()
    t0 = time.perf_counter()
    designs = W.selector_designs(DIMS)
    t_designs = time.perf_counter() - t0
    rhos = synth.selector_training_states(args.states, DIMS, args.seed, designs=designs)
    t0 = time.perf_counter()
    X, y, _ = S.ladder_dataset(DIMS, rhos, LEVELS, policy(), chunk=128)
    t_data = time.perf_counter() - t0
    ntr = int(0.8 * len(y))
    perm = synth.epoch_permutations(ntr, args.epochs, args.seed + 1)
    t0 = time.perf_counter()
    net, loss = S.train_selector(X[:ntr], y[:ntr], synth.mlp_init(args.seed + 2), perm, args.epochs, 128, 3e-3)
    t_train = time.perf_counter() - t0
    pred = net.predict(X[ntr:])
    info = {"states": len(y), "train_states": ntr, "held_out": len(y) - ntr, "dims": list(DIMS),
            "label_counts": np.bincount(y, minlength=4).tolist(),
            "held_out_accuracy": float((pred == y[ntr:]).mean()),
            "held_out_predicted_above_label": int((pred > y[ntr:]).sum()),
            "final_loss": float(loss), "seconds_designs": t_designs, "seconds_labels": t_data,
            "seconds_training": t_train, "seed": args.seed, "epochs": args.epochs,
            "label_form": "batched full ladder, mixed V-cycle, native FP64 Krylov (outer 0)"}
    S.save_trained(net, net.mu, net.sd, info, args.out)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
