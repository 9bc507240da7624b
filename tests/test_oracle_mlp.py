"""Pins of the MLP oracle: FP64 finite differences of its loss on a reduced
network, its softmax cross-entropy against scipy, and its BF16 rounding."""
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
