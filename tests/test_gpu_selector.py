"""The learned first-floor selector: device MLP kernels against the FP64 oracle
(forward, loss gradient, Adam training), and what the trained network gains over
the rule of Eq. (trigger) on held-out states, with the guard and the ladder as the
fallback in both."""
import numpy as np
import pytest

import synth
from oracle import gf_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    from paper_2607_26382_b300 import build
    build.build()
    import paper_2607_26382_b300 as gf
    return gf


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, 6)) * np.array([1, 2, 0.3, 0.2, 0.3, 0.1]) + np.array([-3, -5, 0.5, 0.3, 0.6, 0.4])
    y = rng.integers(0, 4, n).astype(np.int32)
    return X, y


def test_mlp_forward_and_gradient_match_oracle(gf):
    X, y = _data(300, 1)
    theta = synth.mlp_init(7)
    mu, sd = X.mean(0), X.std(0) + 1e-6
    net = gf.MLP(theta)
    net.set_norm(mu, sd)
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.as_tensor(y, dtype=torch.int32, device="cuda")
    logits = torch.zeros((300, 4), dtype=torch.float32, device="cuda")
    net.forward(Xd, logits)
    # the oracle sees the same float32 inputs and parameters, in FP64
    X32 = X.astype(np.float32).astype(np.float64)
    mu32, sd32 = mu.astype(np.float32).astype(np.float64), sd.astype(np.float32).astype(np.float64)
    ref = O.mlp_forward(theta.astype(np.float64), X32, mu32, sd32)
    assert np.abs(logits.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    loss, g = net.loss_grad(Xd, yd)
    rl, rg = O.mlp_loss_grad(theta.astype(np.float64), X32, y, mu32, sd32)
    assert abs(loss - rl) <= 1e-5 * rl
    assert np.abs(g - rg).max() <= 1e-5 * np.abs(rg).max()
    # argmax classes agree with the oracle's logits
    assert np.array_equal(net.predict(X), ref.argmax(1))


def test_mlp_training_matches_oracle_adam(gf):
    X, y = _data(256, 2)
    theta = synth.mlp_init(3)
    mu, sd = X.mean(0), X.std(0) + 1e-6
    epochs, batch, lr = 3, 64, 3e-3
    perm = synth.epoch_permutations(256, epochs, 5)
    net = gf.MLP(theta)
    net.set_norm(mu, sd)
    net.train(torch.as_tensor(X, dtype=torch.float32, device="cuda"),
              torch.as_tensor(y, dtype=torch.int32, device="cuda"), epochs, batch, lr, perm)
    X32 = X.astype(np.float32).astype(np.float64)
    mu32, sd32 = mu.astype(np.float32).astype(np.float64), sd.astype(np.float32).astype(np.float64)
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t = 0
    for e in range(epochs):
        for s0 in range(0, 256, batch):
            idx = perm[e * 256 + s0:e * 256 + s0 + batch]
            _, g = O.mlp_loss_grad(th, X32[idx], y[idx], mu32, sd32)
            t += 1
            th, m, v = O.adam_step(th, g, m, v, t, lr=lr)
    got = net.params().astype(np.float64)
    assert np.abs(got - th).max() <= 2e-5, np.abs(got - th).max()


def test_selector_gain_over_rule_on_held_out_states(gf):
    """Train on full-ladder outcomes, then run Algorithm 1 on held-out states with
    the rule and with the network choosing the first floor."""
    from paper_2607_26382_b300 import selector as S
    dims, L = (16, 8, 8), 3
    pol = gf.policy_defaults(rho0=1e-9, ladder=[1e-6, 1e-4, 1e-2], kmax=60, probe_iters=50, checkpoint_a=25,
                             checkpoint_b=50, solve_prec=gf.GF_MIXED)
    rh = synth.selector_training_states(260, dims, 11)
    X, y, recs = S.ladder_dataset(dims, rh, L, pol)
    ntr = 200
    net, loss = S.train_selector(X[:ntr], y[:ntr], synth.mlp_init(3), synth.epoch_permutations(ntr, 300, 2),
                                 300, 100, 3e-3)
    acc = float((net.predict(X[ntr:]) == y[ntr:]).mean())
    majority = float((y[ntr:] == np.bincount(y[:ntr]).argmax()).mean())
    assert acc > majority
    cmp = S.compare_selectors(dims, rh[ntr:], L, pol, net)
    work = {k: sum(S.work_of(r) for r in v) for k, v in cmp.items()}
    accepted = {k: sum(r["status"] == gf.GF_ACCEPTED for r in v) for k, v in cmp.items()}
    print(f"held-out accuracy {acc:.2f} (majority {majority:.2f}); Arnoldi steps {work}; accepted {accepted}")
    assert work["mlp"] < work["rule"]
    assert accepted["mlp"] >= accepted["rule"]
    # every accepted solve passed the FP64 guard, whichever selector chose the floor
    for r in cmp["mlp"]:
        if r["status"] == gf.GF_ACCEPTED:
            assert r["eta"] <= 1e-6
    # the confidence-gated form never starts above the argmax form and picks floors
    # above the full ladder's no more often
    feats = X[ntr:]
    probs = net.probs(feats)
    assert np.allclose(probs.sum(1), 1.0)
    assert np.array_equal(probs.argmax(1), net.predict(feats))
    pol_c = gf.policy_defaults(rho0=1e-9, ladder=[1e-6, 1e-4, 1e-2], kmax=60, probe_iters=50, checkpoint_a=25,
                               checkpoint_b=50, solve_prec=gf.GF_MIXED, mlp_confidence=0.9)
    cmp_c = S.compare_selectors(dims, rh[ntr:], L, pol_c, net)
    higher = lambda name, c: sum(r["floor_index"] > f["floor_index"] >= 0
                                 for r, f in zip(c[name], c["full"]) if r["status"] == gf.GF_ACCEPTED)
    assert higher("mlp", cmp_c) <= higher("mlp", cmp)
