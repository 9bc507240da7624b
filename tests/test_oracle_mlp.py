"""Pins of the MLP oracle: FP64 finite differences of its loss on a reduced
network, its softmax cross-entropy against scipy, its BF16 rounding, and its
stage checks (another accumulation order passes them, planted mistakes do
not)."""
import numpy as np
from scipy.special import log_softmax

from oracle import mlp_oracle as M


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1e-40], np.float32)
    r = M.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0             # tie -> even
    assert r[2] == 1.0 + 2 ** -7                    # representable
    assert r[3] == 1.0 + 2 ** -6                    # tie -> even (up)
    assert r[4] == -2.5 and r[5] == 0.0
    assert (M.bf16(r) == r).all()


def test_loss_matches_scipy():
    rng = np.random.default_rng(0)
    P = M.random_params(rng, 27, 8, 8)
    X = rng.integers(0, 2, (5, 27)).astype(np.float64)
    sg = rng.random((5, 6))
    T = rng.random((5, 8)); T /= T.sum(1, keepdims=True)
    loss, _, f = M.loss_and_grads(P, X, sg, T, rnd=False)
    ref = np.mean(-(T * log_softmax(f["logits"], axis=1)).sum(1))
    assert abs(loss - ref) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    Din, H, Nc, B = 27, 8, 8, 4
    P = M.random_params(rng, Din, H, Nc)
    X = rng.integers(0, 2, (B, Din)).astype(np.float64)
    sg = rng.random((B, 6))
    T = rng.random((B, Nc)); T /= T.sum(1, keepdims=True)
    _, g, _ = M.loss_and_grads(P, X, sg, T, rnd=False)
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = M.loss_and_grads(P, X, sg, T, rnd=False)
            flat[idx] = old - eps
            lm, _, _ = M.loss_and_grads(P, X, sg, T, rnd=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g["g" + name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (name, idx, fd, an)


def _stage_case(seed, Din=512, H=64, Nc=64, B=8):
    rng = np.random.default_rng(seed)
    P = M.random_params(rng, Din, H, Nc)
    P = {k: v.astype(np.float32) for k, v in P.items()}
    X = rng.integers(0, 2, (B, Din)).astype(np.float32)
    sg = rng.random((B, 6)).astype(np.float32)
    T = (rng.random((B, Nc)) ** 8).astype(np.float32)
    T /= T.sum(1, keepdims=True)
    return P, X, sg, T


def _values(P, X, sg, T, acc):
    """The oracle network's stage values with sums accumulated in `acc`, in
    the order of a reversed input axis (another implementation)."""
    perm = np.arange(X.shape[1])[::-1]
    loss, g, f = M.loss_and_grads(dict(P, W1=P["W1"][:, perm]), X[:, perm], sg, T, rnd=True, acc=acc)
    g["gW1"] = g["gW1"][:, np.argsort(perm)]
    V = dict(g, loss=loss, logits=f["logits"], H1=f["H1"], H2=f["H2"], Z=f["Z"], dlog=f["dlog"], dH2=f["dH2"],
             dH1=f["dH1p"], W1b=M.bf16(P["W1"]), W2b=M.bf16(P["W2"]), W3b=M.bf16(P["W3"]))
    return V


def test_stage_checks_accept_another_accumulation_order():
    for seed in range(3):
        P, X, sg, T = _stage_case(seed)
        for acc in (np.float32, np.float64):
            V = _values(P, X, sg, T, acc)
            bad = M.stage_violations(P, X, sg, T, V)
            assert not any(bad.values()), bad
            e2e, _ = M.end_to_end_violations(P, X, sg, T, V)
            assert not any(e2e.values()), e2e


def test_stage_checks_catch_planted_mistakes():
    # one activation two BF16 steps off, a dlog without its 1/B, one gradient
    # element with the wrong sign, a ReLU mask not applied, a 1% scale error,
    # rows of an activation swapped: each makes its stage fail
    P, X, sg, T = _stage_case(5)
    base = _values(P, X, sg, T, np.float64)

    def fails(name, **over):
        bad = M.stage_violations(P, X, sg, T, dict(base, **over))
        assert bad[name] > 0, (name, bad)

    H1 = base["H1"].copy()
    j = tuple(np.argwhere(H1 > 0)[0])
    H1[j] = M.bf16(np.array([H1[j] * (1 + 2 ** -6)], np.float32))[0]
    fails("H1", H1=H1)
    fails("dlog", dlog=M.bf16((base["dlog"] * X.shape[0]).astype(np.float32)))
    gW2 = base["gW2"].copy()
    i = np.unravel_index(np.argmax(np.abs(gW2)), gW2.shape)
    gW2[i] = -gW2[i]
    fails("gW2", gW2=gW2)
    H = base["W2b"].shape[0]
    fails("dH2", dH2=M.bf16((base["dlog"] @ base["W3b"])[:, :H].astype(np.float32)))
    fails("gW1", gW1=base["gW1"] * 1.01)
    fails("H2", H2=base["H2"][::-1].copy())
