"""CPU oracle of the learned-proposal MLP -- TEST INFRASTRUCTURE ONLY.

numpy restatement of the network the library trains on the tensor cores:
    H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Z = [H2, start, goal, 0],
    logits = Z W3^T + b3, loss = mean_b( -sum_c T_bc log softmax(logits_b)_c ),
with the gradients of that loss.  With round=True every operand the GPU feeds
to a BF16 GEMM is rounded to BF16 (round to nearest even) at the same point,
and products are accumulated in FP32; with round=False everything is FP64
(used for the finite-difference pin).  Only tests import this module.
"""
import numpy as np


def bf16(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    out = rounded.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def _r(x, rnd):
    return bf16(x) if rnd else x


def forward(P, X, sg, rnd=True):
    dt = np.float32 if rnd else np.float64
    X = np.asarray(X, dt); sg = np.asarray(sg, dt)
    W1, W2, W3 = (_r(np.asarray(P[k], dt), rnd) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.asarray(P[k], dt) for k in ("b1", "b2", "b3"))
    H = W2.shape[0]
    H1 = _r(np.maximum(X @ W1.T + b1, 0), rnd)
    H2 = _r(np.maximum(H1 @ W2.T + b2, 0), rnd)
    Dz = W3.shape[1]
    Z = np.zeros((X.shape[0], Dz), dt)
    Z[:, :H] = H2
    Z[:, H:H + 6] = sg
    Z = _r(Z, rnd)
    logits = Z @ W3.T + b3
    return {"H1": H1, "H2": H2, "Z": Z, "logits": logits, "W1": W1, "W2": W2, "W3": W3}


def loss_and_grads(P, X, sg, T, rnd=True):
    dt = np.float32 if rnd else np.float64
    f = forward(P, X, sg, rnd)
    T = np.asarray(T, dt)
    X = np.asarray(X, dt)
    B = X.shape[0]
    H = f["W2"].shape[0]
    l = f["logits"]
    m = l.max(axis=1, keepdims=True)
    lse = m + np.log(np.exp(l - m).sum(axis=1, keepdims=True))
    p = np.exp(l - lse)
    loss = float(np.mean(-(T * (l - lse)).sum(axis=1)))
    dlog = _r((p - T) / B, rnd)
    g = {"gW3": dlog.T @ f["Z"], "gb3": dlog.sum(axis=0)}
    dZ = dlog @ f["W3"]
    dH2 = _r(np.where(f["H2"] > 0, dZ[:, :H], 0), rnd)
    g["gW2"] = dH2.T @ f["H1"]
    g["gb2"] = dH2.sum(axis=0)
    dH1 = dH2 @ f["W2"]
    dH1p = _r(np.where(f["H1"] > 0, dH1, 0), rnd)
    g["gW1"] = dH1p.T @ X
    g["gb1"] = dH1p.sum(axis=0)
    return loss, g, f


def random_params(rng, Din, H, Nc, dtype=np.float64):
    Dz = H + 16
    return {"W1": rng.normal(0, np.sqrt(2 / Din), (H, Din)).astype(dtype), "b1": rng.normal(0, 0.1, H).astype(dtype),
            "W2": rng.normal(0, np.sqrt(2 / H), (H, H)).astype(dtype), "b2": rng.normal(0, 0.1, H).astype(dtype),
            "W3": rng.normal(0, np.sqrt(1 / Dz), (Nc, Dz)).astype(dtype), "b3": rng.normal(0, 0.1, Nc).astype(dtype)}
