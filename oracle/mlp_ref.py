"""FP64 CPU reference of the ranker MLP — TEST INFRASTRUCTURE ONLY.

96 -> 256 (ReLU) -> 256 (ReLU) -> 1, weighted binary cross-entropy on the
logit: loss = sum_i w_i * (max(z,0) - z*y + log(1 + exp(-|z|))) / sum_i w_i.
Parameters are one flat vector in the order W1[256x96], b1, W2[256x256], b2,
W3[256], b3 (W[out][in]).  With bf16=True the operands are rounded to
bfloat16 where the GPU kernels round them (inputs, weights, hidden
activations, activation gradients); products and sums are exact fp64.
Pinned by a central finite-difference check of its own gradients.
"""
import numpy as np

IN, HID = 96, 256
SIZES = [("W1", HID * IN), ("b1", HID), ("W2", HID * HID), ("b2", HID), ("W3", HID), ("b3", 1)]
NPARAM = sum(n for _, n in SIZES)


def bf16(x):
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def split(p):
    out, o = {}, 0
    for name, n in SIZES:
        out[name] = np.asarray(p[o:o + n], dtype=np.float64)
        o += n
    out["W1"] = out["W1"].reshape(HID, IN)
    out["W2"] = out["W2"].reshape(HID, HID)
    return out


def forward(p, x, rnd=True):
    q = split(p)
    r = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    xb = r(x)
    h1 = r(np.maximum(xb @ r(q["W1"]).T + q["b1"], 0))
    h2 = r(np.maximum(h1 @ r(q["W2"]).T + q["b2"], 0))
    z = h2 @ q["W3"] + q["b3"][0]
    return z, (xb, h1, h2)


def loss_and_grad(p, x, y, w=None, rnd=True):
    q = split(p)
    r = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    y = np.asarray(y, np.float64)
    w = np.ones_like(y) if w is None else np.asarray(w, np.float64)
    ws = w.sum()
    z, (xb, h1, h2) = forward(p, x, rnd)
    loss = float(np.sum(w * (np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))) / ws)
    dz = w * (1 / (1 + np.exp(-z)) - y) / ws
    g = {}
    g["W3"] = h2.T @ dz
    g["b3"] = np.array([dz.sum()])
    dh2 = r(np.where(h2 > 0, np.outer(dz, q["W3"]), 0))
    g["b2"] = dh2.sum(0)
    g["W2"] = dh2.T @ h1
    dh1 = r(np.where(h1 > 0, dh2 @ r(q["W2"]), 0))
    g["b1"] = dh1.sum(0)
    g["W1"] = dh1.T @ xb
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, flat
