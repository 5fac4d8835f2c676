"""Learned first-floor selector: labels from ladder outcomes, training, comparison.

Workflow (every solve, feature and network step runs in libgf_b300.so):
  1. ``ladder_dataset``: run the full ladder (rho0, then every floor in order) on
     batched states; features are the rho0 attempt's r50/r100 (what the probe
     records) plus density statistics, the label is the first accepted floor
     (the top floor when none is accepted).
  2. ``train_selector``: standardise, then Adam on the device MLP.
  3. ``compare_selectors``: Algorithm 1 with the rule of Eq. (trigger) against the
     same policy with the MLP picking the first floor; the guard and the rest of
     the ladder remain the fallback in both.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import _lib as L

# weights written by ``python -m paper_2607_26382_b300.train_selector``
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")


def _batch_for(dims_list, levels, rhos, p=3.0):
    import torch
    b = L.Batch(dims_list, levels=levels)
    for i, (d, rho) in enumerate(zip(dims_list, rhos)):
        f = torch.zeros(b.n_dof[i], dtype=torch.float64, device="cuda")
        gh = L.c_void_p()
        L._check(L.lib().gf_batch_grid(b._h, i, L.ctypes.byref(gh)))
        L._check(L.lib().gf_cantilever_load(gh, L.c_void_p(f.data_ptr())))
        b.set_state(i, torch.as_tensor(np.ascontiguousarray(rho), device="cuda"), f, p)
    return b


def ladder_dataset(dims, rhos, levels, policy: L.Policy, chunk=64):
    """Features X (n x 6), labels y (n), and the full-ladder records."""
    pol = L.policy_defaults()
    L.ctypes.memmove(L.ctypes.byref(pol), L.ctypes.byref(policy), L.ctypes.sizeof(L.Policy))
    pol.selector = L.GF_SEL_FULL
    n_floors = pol.n_ladder + 1
    X, y, recs = [], [], []
    for c0 in range(0, len(rhos), chunk):
        part = rhos[c0:c0 + chunk]
        b = _batch_for([dims] * len(part), levels, part)
        res = b.select_floor(pol)
        for i, r in enumerate(res):
            X.append(b.features(i, r["r50"], r["r100"]))
            y.append(r["floor_index"] if r["status"] == L.GF_ACCEPTED else n_floors - 1)
            recs.append(r)
        b.close()
    return np.array(X), np.array(y, dtype=np.int32), recs


def feature_norm(X):
    """Standardisation of the selector's inputs: per-feature mean and std (+1e-6), from
    the training rows; the device MLP applies it (gf_mlp_set_norm)."""
    return X.mean(axis=0), X.std(axis=0) + 1e-6


def train_selector(X, y, theta0, perm, epochs, batch=128, lr=3e-3):
    import torch
    mu, sd = feature_norm(X)
    net = L.MLP(theta0)
    net.set_norm(mu, sd)
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda").contiguous()
    yd = torch.as_tensor(y, dtype=torch.int32, device="cuda").contiguous()
    loss = net.train(Xd, yd, epochs, batch, lr, perm)
    net.mu, net.sd = mu, sd
    return net, loss


def work_of(r):
    """Arnoldi steps one Algorithm-1 run spent: attempts, plus the probe when it was
    abandoned (a fused probe that continues is counted inside the rho0 attempt)."""
    w = sum(a["iters"] for a in r["attempts"])
    if r["escalated"]:
        w += r["probe_iters_run"]
    return w


def compare_selectors(dims, rhos, levels, policy: L.Policy, net: L.MLP, chunk=64):
    """Per-state records under the rule and under the MLP, plus the full ladder's
    minimal accepted floor (to count floors chosen higher than needed)."""
    out = {}
    for name, sel in (("full", L.GF_SEL_FULL), ("rule", L.GF_SEL_RULE), ("mlp", L.GF_SEL_MLP)):
        pol = L.policy_defaults()
        L.ctypes.memmove(L.ctypes.byref(pol), L.ctypes.byref(policy), L.ctypes.sizeof(L.Policy))
        pol.selector = sel
        pol.mlp = net.handle if sel == L.GF_SEL_MLP else None
        recs = []
        for c0 in range(0, len(rhos), chunk):
            part = rhos[c0:c0 + chunk]
            b = _batch_for([dims] * len(part), levels, part)
            recs += b.select_floor(pol)
            b.close()
        out[name] = recs
    return out


def save_trained(net: L.MLP, mu, sd, info, path=WEIGHTS):
    rec = dict(info, theta=[float(v) for v in net.params()], mu=[float(v) for v in mu],
               sd=[float(v) for v in sd])
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=0)


def load_trained(path=WEIGHTS):
    """(MLP on the device, metadata) from a weights file written by train_selector."""
    rec = json.load(open(path))
    net = L.MLP(np.asarray(rec["theta"], dtype=np.float32))
    net.set_norm(rec["mu"], rec["sd"])
    meta = {k: v for k, v in rec.items() if k not in ("theta", "mu", "sd")}
    return net, meta
