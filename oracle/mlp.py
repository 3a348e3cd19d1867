"""Oracle of the learned warm start (not in the paper): features, forward and backward of the
per-circle MLP in plain numpy.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline); the CUDA library never uses it.

Features: binary32 arithmetic, one correctly rounded operation at a time (numpy float32
element-wise operations are IEEE operations), in the order the library documents:
  e_r = c / |c| (|c| = sqrt(x*x + y*y)), e_t = (-e_r.y, e_r.x); the 12 nearest other centres with
  squared distance (dx*dx + dy*dy) < 4.5^2, ordered by (squared distance, index), as offsets
  (dx*e_r.x + dy*e_r.y, dy*e_r.x - dx*e_r.y), zero-padded; then min((R - |c|) - 1, 4.5).
Network: 25 -> 128 -> 128 -> 128 -> 2 with ReLU; every GEMM input (features, weights,
activations, back-propagated gradients) is rounded to bfloat16 (round to nearest even) after a
binary32 rounding, GEMMs are accumulated in binary64 (the device accumulates in binary32).
"""
from __future__ import annotations

import numpy as np

H, F, KNN = 128, 25, 12
OW1 = 0
OB1 = OW1 + H * F
OW2 = OB1 + H
OB2 = OW2 + H * H
OW3 = OB2 + H
OB3 = OW3 + H * H
OW4 = OB3 + H
OB4 = OW4 + 2 * H
NPAR = OB4 + 2


def bf16(x):
    """Round to bfloat16 (nearest even) through binary32, as float64 values."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    nan = np.isnan(f)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    out = np.where(nan, f, out)
    return out.astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    return dict(W1=p[OW1:OB1].reshape(H, F), b1=p[OB1:OW2], W2=p[OW2:OB2].reshape(H, H), b2=p[OB2:OW3],
                W3=p[OW3:OB3].reshape(H, H), b3=p[OB3:OW4], W4=p[OW4:OB4].reshape(2, H), b4=p[OB4:NPAR])


def pack(d):
    return np.concatenate([d["W1"].ravel(), d["b1"], d["W2"].ravel(), d["b2"], d["W3"].ravel(), d["b3"],
                           d["W4"].ravel(), d["b4"]])


def features(xy32, R):
    """Features [n, 25] of one instance; xy32 float32 [n, 2] (the coordinates the device holds)."""
    x = np.ascontiguousarray(xy32, dtype=np.float32)
    n = x.shape[0]
    out = np.zeros((n, F), dtype=np.float32)
    f32 = np.float32
    for i in range(n):
        dx = x[:, 0] - x[i, 0]
        dy = x[:, 1] - x[i, 1]
        s = dx * dx + dy * dy
        cand = np.nonzero((s < f32(4.5 * 4.5)) & (np.arange(n) != i))[0]
        order = cand[np.lexsort((cand, s[cand]))][:KNN]
        r = np.sqrt(x[i, 0] * x[i, 0] + x[i, 1] * x[i, 1])
        if r > 0:
            erx, ery = x[i, 0] / r, x[i, 1] / r
        else:
            erx, ery = f32(1.0), f32(0.0)
        for u, j in enumerate(order):
            out[i, 2 * u] = dx[j] * erx + dy[j] * ery
            out[i, 2 * u + 1] = dy[j] * erx - dx[j] * ery
        b = (f32(R) - r) - f32(1.0)
        out[i, 24] = min(b, f32(4.5))
    return out


def forward(params, feat, round_bf16=True, keep=False):
    """Outputs [rows, 2]; keep=True also returns the layer inputs for backward."""
    p = unpack(params)
    rnd = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = rnd(np.asarray(feat, dtype=np.float32))
    Ws = [rnd(p["W1"]), rnd(p["W2"]), rnd(p["W3"]), rnd(p["W4"])]
    bs = [p["b1"], p["b2"], p["b3"], p["b4"]]
    acts = [X]
    h = X
    for layer in range(3):
        z = h @ Ws[layer].T + bs[layer]
        h = rnd(np.maximum(z, 0.0).astype(np.float32) if round_bf16 else np.maximum(z, 0.0))
        acts.append(h)
    out = h @ Ws[3].T + bs[3]
    return (out, acts, Ws) if keep else out


def loss_grad(params, feat, target, round_bf16=True):
    """L = mean_r |out_r - target_r|^2 and dL/dparams (float64, layout of the parameter vector)."""
    out, acts, Ws = forward(params, feat, round_bf16, keep=True)
    rnd = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    rows = feat.shape[0]
    diff = out - np.asarray(target, dtype=np.float64)
    L = float(np.sum(diff * diff) / rows)
    dZ = rnd((2.0 * diff / rows).astype(np.float32) if round_bf16 else 2.0 * diff / rows)
    g = {}
    names = ["1", "2", "3", "4"]
    for layer in (3, 2, 1, 0):
        Hin = acts[layer]
        g["W" + names[layer]] = dZ.T @ Hin
        g["b" + names[layer]] = dZ.sum(0)
        if layer > 0:
            dH = dZ @ Ws[layer]
            mask = acts[layer] > 0
            dZ = rnd((dH * mask).astype(np.float32) if round_bf16 else dH * mask)
    return L, pack(g)


# ------------------------------------------------------------------ layer-by-layer restatement
# For element-wise parity of the tensor-core network: each layer recomputed in binary64 from the
# device's own bf16 inputs of that layer (its traced activations), so that an element can differ
# from the device's only by the device's binary32 accumulation of that one layer.

def weights_bf16(params):
    """The bf16 values of W1..W4 (binary64 arrays, [out][in]) and the binary32 biases."""
    p = unpack(params)
    return [bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"]), bf16(p["W4"])], [p["b1"], p["b2"], p["b3"], p["b4"]]


def pre_activation(params, layer, h_in):
    """z = h_in W_layer^T + b_layer in binary64 (layer 0..3; h_in holds bf16 values), and the sum of
    the magnitudes of its terms |h_in| |W|^T + |b| (the scale of a rounding bound)."""
    Ws, bs = weights_bf16(params)
    h = np.asarray(h_in, dtype=np.float64)
    return h @ Ws[layer].T + bs[layer], np.abs(h) @ np.abs(Ws[layer]).T + np.abs(bs[layer])


def output_gradient(out, target, rows):
    """dO = bf16((out - target) * (2 / rows)), every operation in binary32: the output layer's gradient of the
    mean squared loss as the device forms it from its binary32 outputs."""
    d = np.asarray(out, dtype=np.float32) - np.asarray(target, dtype=np.float32)
    return bf16((d * (np.float32(2.0) / np.float32(rows))).astype(np.float32))


def back_pre(params, layer, dz):
    """dZ_layer W_layer (binary64; dz holds bf16 values) and |dZ| |W| (the scale of its rounding bound):
    the gradient with respect to the input of layer `layer` before the ReLU mask of that input."""
    Ws, _ = weights_bf16(params)
    d = np.asarray(dz, dtype=np.float64)
    return d @ Ws[layer], np.abs(d) @ np.abs(Ws[layer])
