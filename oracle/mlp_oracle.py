"""CPU oracle of the learned-proposal MLP -- TEST INFRASTRUCTURE ONLY.

numpy restatement of the network the library trains on the tensor cores:
    H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Z = [H2, start, goal, 0],
    logits = Z W3^T + b3, loss = mean_b( -sum_c T_bc log softmax(logits_b)_c ),
with the gradients of that loss.  With round=True every operand the GPU feeds
to a BF16 GEMM is rounded to BF16 (round to nearest even) at the same point,
and products are accumulated in FP32; with round=False everything is FP64
(used for the finite-difference pin).  stage_violations() checks another
implementation's values, stage by stage and element by element, against these
definitions applied to that implementation's own stage inputs.  Only tests
import this module.
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


def forward(P, X, sg, rnd=True, acc=None):
    """acc: accumulation dtype of the products (default FP32 when rounding,
    FP64 otherwise)."""
    dt = acc if acc is not None else (np.float32 if rnd else np.float64)
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


def loss_and_grads(P, X, sg, T, rnd=True, acc=None):
    dt = acc if acc is not None else (np.float32 if rnd else np.float64)
    f = forward(P, X, sg, rnd, acc)
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
    f.update(dlog=dlog, dH2=dH2, dH1p=dH1p)
    return loss, g, f


def random_params(rng, Din, H, Nc, dtype=np.float64):
    Dz = H + 16
    return {"W1": rng.normal(0, np.sqrt(2 / Din), (H, Din)).astype(dtype), "b1": rng.normal(0, 0.1, H).astype(dtype),
            "W2": rng.normal(0, np.sqrt(2 / H), (H, H)).astype(dtype), "b2": rng.normal(0, 0.1, H).astype(dtype),
            "W3": rng.normal(0, np.sqrt(1 / Dz), (Nc, Dz)).astype(dtype), "b3": rng.normal(0, 0.1, Nc).astype(dtype)}


# --------------------------------------------------------------------------- stage checks
U_ACC = 2.0 ** -23   # per-step roundoff allowed in an FP32 accumulation (a tensor-core adder may truncate)


def gamma(k):
    """Bound, relative to the sum of the terms' magnitudes, on the error of a
    k-term FP32 sum taken in any order (Higham, Accuracy and Stability of
    Numerical Algorithms, Sec. 3.1: gamma_k = k u / (1 - k u))."""
    return k * U_ACC / (1.0 - k * U_ACC)


def bf16_range(center, err, fn=None):
    """Every BF16 value that rounding fn(a) to nearest even can give for an
    FP32 value a within err of center: [bf16(fn(lo)), bf16(fn(hi))] with lo
    and hi rounded outward to FP32 (fn and the rounding are monotone)."""
    lo = np.asarray(center - err, np.float64)
    hi = np.asarray(center + err, np.float64)
    lo32 = lo.astype(np.float32)
    lo32 = np.where(lo32.astype(np.float64) > lo, np.nextafter(lo32, np.float32(-np.inf)), lo32)
    hi32 = hi.astype(np.float32)
    hi32 = np.where(hi32.astype(np.float64) < hi, np.nextafter(hi32, np.float32(np.inf)), hi32)
    if fn is not None:
        lo32, hi32 = fn(lo32), fn(hi32)
    return bf16(lo32).astype(np.float64), bf16(hi32).astype(np.float64)


def stage_violations(P, X, sg, T, V):
    """Count, per stage, the elements of another implementation's values V that
    the network's definition, applied to V's own inputs of that stage, rules
    out.  V holds the BF16 weight copies W1b, W2b, W3b, the BF16 activations H1,
    H2, Z, dlog, dH2, dH1 (after the ReLU masks), the FP32 logits, the six
    gradients and the mean loss.  A BF16 value must be one that rounding the
    exact result, moved by at most its FP32 sum's accumulation error (gamma_K
    times the sum of the terms' magnitudes), can give; an FP32 value must lie
    within that error of the exact result; the softmax adds the error of its
    exponent sum and a few ulps for exp and log."""
    a = lambda x: np.abs(np.asarray(x, np.float64))
    f64 = lambda x: np.asarray(x, np.float64)
    X, sg, T = f64(X), f64(sg), f64(T)
    B, H = X.shape[0], V["W2b"].shape[0]
    Din, Dz, Nc = X.shape[1], V["W3b"].shape[1], V["W3b"].shape[0]
    W1, W2, W3 = f64(V["W1b"]), f64(V["W2b"]), f64(V["W3b"])
    b1, b2, b3 = f64(P["b1"]), f64(P["b2"]), f64(P["b3"])
    H1, H2, Z, dlog, dH2, dH1 = (f64(V[k]) for k in ("H1", "H2", "Z", "dlog", "dH2", "dH1"))
    logits = f64(V["logits"])
    relu = lambda x: np.maximum(x, np.float32(0))
    out = {}

    def within(name, x, rng):
        out[name] = int(np.count_nonzero(~((x >= rng[0]) & (x <= rng[1]))))

    def close(name, x, ref, bound):
        out[name] = int(np.count_nonzero(np.abs(f64(x) - ref) > bound))

    for k, Wb in (("W1", W1), ("W2", W2), ("W3", W3)):
        out[k + "b"] = int(np.count_nonzero(Wb != bf16(np.asarray(P[k], np.float32))))
    within("H1", H1, bf16_range(X @ W1.T + b1, gamma(Din + 1) * (a(X) @ a(W1).T + a(b1)), relu))
    within("H2", H2, bf16_range(H1 @ W2.T + b2, gamma(H + 1) * (a(H1) @ a(W2).T + a(b2)), relu))
    Zref = np.zeros((B, Dz))
    Zref[:, :H] = H2
    Zref[:, H:H + 6] = bf16(np.asarray(sg, np.float32))
    out["Z"] = int(np.count_nonzero(Z != Zref))
    close("logits", logits, Z @ W3.T + b3, gamma(Dz + 1) * (a(Z) @ a(W3).T + a(b3)))
    mx = logits.max(1, keepdims=True)
    lse = mx + np.log(np.exp(logits - mx).sum(1, keepdims=True))
    p = np.exp(logits - lse)
    ref_loss = float(np.mean(-(T * (logits - lse)).sum(1)))
    out["loss"] = int(abs(V["loss"] - ref_loss) > 2 * gamma(Nc + 2) * abs(ref_loss) + 1e-6)
    perr = p * (gamma(Nc + 1) + 2.0 ** -20 * (1 + a(lse) + a(logits) + a(logits - lse)))
    within("dlog", dlog, bf16_range((p - T) / B, (perr + 2.0 ** -24 * a(p - T)) / B))
    close("gW3", V["gW3"], dlog.T @ Z, gamma(B) * (a(dlog).T @ a(Z)))
    close("gb3", V["gb3"], dlog.sum(0), gamma(B) * a(dlog).sum(0))
    lo, hi = bf16_range((dlog @ W3)[:, :H], gamma(Nc) * (a(dlog) @ a(W3))[:, :H])
    within("dH2", dH2, (np.where(H2 > 0, lo, 0.0), np.where(H2 > 0, hi, 0.0)))
    close("gW2", V["gW2"], dH2.T @ H1, gamma(B) * (a(dH2).T @ a(H1)))
    close("gb2", V["gb2"], dH2.sum(0), gamma(B) * a(dH2).sum(0))
    lo, hi = bf16_range(dH2 @ W2, gamma(H) * (a(dH2) @ a(W2)))
    within("dH1", dH1, (np.where(H1 > 0, lo, 0.0), np.where(H1 > 0, hi, 0.0)))
    close("gW1", V["gW1"], dH1.T @ X, gamma(B) * (a(dH1).T @ a(X)))
    close("gb1", V["gb1"], dH1.sum(0), gamma(B) * a(dH1).sum(0))
    return out


def end_to_end_violations(P, X, sg, T, V):
    """Count the elements of V's logits and gradients that differ from this
    oracle's (run from the true inputs) by more than the BF16 intermediates
    that differ between the two carry through the last product, plus both
    sides' accumulation error.  Returns (counts, fraction of differing BF16
    intermediates per array)."""
    a = lambda x: np.abs(np.asarray(x, np.float64))
    f64 = lambda x: np.asarray(x, np.float64)
    _, rg, f = loss_and_grads(P, X, sg, T, rnd=True)
    X = f64(X)
    B, H = X.shape[0], V["W2b"].shape[0]
    W3 = f64(V["W3b"])
    Z, rZ = f64(V["Z"]), f64(f["Z"])
    out = {"logits": int(np.count_nonzero(
        a(f64(V["logits"]) - f["logits"]) >
        a(Z - rZ) @ a(W3).T + 2 * gamma(Z.shape[1] + 1) * ((a(Z) + a(rZ)) @ a(W3).T + a(P["b3"]))))}
    pairs = {"gW3": ("dlog", "Z", "dlog", "Z"), "gW2": ("dH2", "H1", "dH2", "H1"), "gW1": ("dH1", None, "dH1p", None)}
    for k, (u, w, ru, rw) in pairs.items():
        Ug, Ur = f64(V[u]), f64(f[ru])
        Vg, Vr = (f64(V[w]), f64(f[rw])) if w else (X, X)
        bound = a(Ug - Ur).T @ a(Vg) + a(Ur).T @ a(Vg - Vr) + 2 * gamma(B) * ((a(Ug) + a(Ur)).T @ (a(Vg) + a(Vr)))
        out[k] = int(np.count_nonzero(a(f64(V[k]) - rg[k]) > bound))
    for k, (u, ru) in {"gb3": ("dlog", "dlog"), "gb2": ("dH2", "dH2"), "gb1": ("dH1", "dH1p")}.items():
        Ug, Ur = f64(V[u]), f64(f[ru])
        bound = a(Ug - Ur).sum(0) + 2 * gamma(B) * (a(Ug) + a(Ur)).sum(0)
        out[k] = int(np.count_nonzero(a(f64(V[k]) - rg[k]) > bound))
    frac = {k: float(np.mean(f64(V[k]) != f64(f[rk]))) for k, rk in
            (("H1", "H1"), ("H2", "H2"), ("Z", "Z"), ("dlog", "dlog"), ("dH2", "dH2"), ("dH1", "dH1p"))}
    return out, frac
