"""FP64 oracle of the proposal MLP (test infrastructure only).

The learned pivot proposal is a project extension, not part of the paper: a
per-correspondence inlier-scoring MLP 8 -> 64 -> 128 -> 64 -> 1 with ReLU and
a sigmoid output, trained with the mean binary cross-entropy.  This module
states its forward pass, its gradient by manual back-propagation and its
input features in double precision with NumPy, plainly and layer by layer.

With ``bf16=True`` the forward rounds to bfloat16 at the points the GPU
kernels do (input features, weights and biases, and the ReLU outputs h1, h2,
h3), so the GPU's gradients can be compared with it; everything else stays
FP64.  With ``bf16=False`` it is the exact FP64 network, which the tests pin
with finite differences.

Parameter vector layout (row-major [out][in]):
W1[64][8] b1[64] W2[128][64] b2[128] W3[64][128] b3[64] W4[64] b4[1].
"""
from __future__ import annotations

import numpy as np

SIZES = [("W1", (64, 8)), ("b1", (64,)), ("W2", (128, 64)), ("b2", (128,)), ("W3", (64, 128)),
         ("b3", (64,)), ("W4", (64,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)   # 17217


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(a):
    """Round float values to bfloat16 (round to nearest, ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, feat, bf16_round=True):
    """Layer outputs of the network for features [m, 8]: dict with z1..z4, h1..h3, p."""
    P = unpack(theta)
    rnd = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    if bf16_round:
        P = {k: bf16(v) for k, v in P.items()}
    x = rnd(feat)
    z1 = x @ P["W1"].T + P["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = rnd(np.maximum(z2, 0.0))
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = rnd(np.maximum(z3, 0.0))
    z4 = h3 @ P["W4"] + P["b4"][0]
    p = 1.0 / (1.0 + np.exp(-z4))
    return {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "h3": h3, "z4": z4, "p": p, "P": P}


def loss(theta, feat, label, bf16_round=True):
    """Mean binary cross-entropy of the sigmoid output."""
    z = forward(theta, feat, bf16_round)["z4"]
    y = np.asarray(label, dtype=np.float64)
    return float(np.mean(np.log1p(np.exp(-np.abs(z))) + np.maximum(z, 0.0) - y * z))


def grad(theta, feat, label, bf16_round=True):
    """(d mean BCE / d theta, loss) by back-propagation, layer by layer."""
    f = forward(theta, feat, bf16_round)
    P = f["P"]
    y = np.asarray(label, dtype=np.float64)
    m = y.shape[0]
    z4 = f["z4"]
    L = float(np.mean(np.log1p(np.exp(-np.abs(z4))) + np.maximum(z4, 0.0) - y * z4))
    dz4 = (f["p"] - y) / m                           # d L / d z4
    gW4 = f["h3"].T @ dz4
    gb4 = np.array([dz4.sum()])
    dz3 = np.outer(dz4, P["W4"]) * (f["h3"] > 0)     # ReLU mask of layer 3
    gW3 = dz3.T @ f["h2"]
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ P["W3"]) * (f["h2"] > 0)
    gW2 = dz2.T @ f["h1"]
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (f["h1"] > 0)
    gW1 = dz1.T @ f["x"]
    gb1 = dz1.sum(0)
    g = pack({"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3, "W4": gW4, "b4": gb4})
    return g, L


def features(x, y, A, S):
    """Proposal features [n, 8]: centred coordinates scaled by their RMS
    distance to the centroid (source, target), degree / n and SC^2 row score /
    its maximum; A and S are the oracle's compatibility and SC^2 matrices."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    out = np.zeros((n, 8))
    for k, pts in enumerate((x, y)):
        c = pts - pts.mean(0)
        rms = np.sqrt(np.mean(np.sum(c * c, axis=1)))
        out[:, 3 * k:3 * k + 3] = c / rms if rms > 0 else 0.0
    out[:, 6] = A.sum(1) / n
    r = S.sum(1).astype(np.float64)
    out[:, 7] = r / r.max() if r.max() > 0 else 0.0
    return out
