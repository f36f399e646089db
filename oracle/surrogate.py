"""FP64 reference of the surrogate EOS: an ensemble of MLPs 2 -> 128 -> 128 -> 128 -> 2
(tanh hidden layers) mapping normalised (rho, e) to normalised (P, T), trained with
Adam on mean-squared error.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the CPU arm of ``bench.py``.
Shares no code with the CUDA path.

Precision reading (BF16 weights, FP32 accumulation): every weight matrix enters the
forward pass rounded to bfloat16 (round to nearest even); the hidden activations that
feed a matrix product (h1, h2, h3) are rounded to bfloat16; biases, pre-activations,
outputs and all gradients stay in full precision.  Backward: the tanh derivative is
1 - h^2 with the rounded h; the error signals dz2, dz3 that feed matrix products are
rounded to bfloat16 (dz1 is not: layer 1 has no product after it).  With
``bf16=False`` every rounding is skipped (plain FP64 network, used for the
finite-difference pins).

Parameter vector of one model (FP32 on the GPU, FP64 here), in this order:
W1[128,2] b1[128] W2[128,128] b2[128] W3[128,128] b3[128] W4[2,128] b4[2]
(W[out, in], row-major): 33,666 values.
"""
from __future__ import annotations

import numpy as np

H = 128
SHAPES = [("W1", (H, 2)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
          ("b3", (H,)), ("W4", (2, H)), ("b4", (2,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (r.astype(np.uint32)).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(x))


def unpack(p):
    d, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        d[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return d


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed, n_models=4):
    """Glorot-uniform weights, zero biases (an input generator, not part of the method)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_models):
        d = {}
        for name, shp in SHAPES:
            if name[0] == "W":
                lim = np.sqrt(6.0 / (shp[0] + shp[1]))
                d[name] = rng.uniform(-lim, lim, shp)
            else:
                d[name] = np.zeros(shp)
        out.append(pack(d))
    return np.array(out, dtype=np.float32).astype(np.float64)


def forward(p, x, bf16_mode=True):
    """x: [B, 2] normalised inputs.  Returns y [B, 2] and the cache for backward."""
    r = bf16 if bf16_mode else (lambda a: np.asarray(a, dtype=np.float64))
    d = unpack(p)
    W1, W2, W3, W4 = r(d["W1"]), r(d["W2"]), r(d["W3"]), r(d["W4"])
    z1 = x @ W1.T + d["b1"]
    h1 = r(np.tanh(z1))
    z2 = h1 @ W2.T + d["b2"]
    h2 = r(np.tanh(z2))
    z3 = h2 @ W3.T + d["b3"]
    h3 = r(np.tanh(z3))
    y = h3 @ W4.T + d["b4"]
    return y, dict(x=x, h1=h1, h2=h2, h3=h3, W2=W2, W3=W3, W4=W4)


def loss_and_grad(p, x, t, bf16_mode=True):
    """Mean-squared error over the batch and both outputs, and its gradient."""
    r = bf16 if bf16_mode else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(p, x, bf16_mode)
    B = x.shape[0]
    diff = y - t
    loss = float(np.mean(diff * diff))
    dy = 2.0 * diff / (B * 2)
    g = {}
    g["W4"] = dy.T @ c["h3"]
    g["b4"] = dy.sum(axis=0)
    dz3 = r((dy @ c["W4"]) * (1.0 - c["h3"] ** 2))
    g["W3"] = dz3.T @ c["h2"]
    g["b3"] = dz3.sum(axis=0)
    dz2 = r((dz3 @ c["W3"]) * (1.0 - c["h2"] ** 2))
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ c["W2"]) * (1.0 - c["h1"] ** 2)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): step t counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def normaliser(a):
    """Mean and standard deviation per column (FP64)."""
    a = np.asarray(a, dtype=np.float64)
    return a.mean(axis=0), a.std(axis=0)


def ensemble_predict(params, x_phys, xs, ys, bf16_mode=True):
    """Ensemble mean and standard deviation of the physical outputs.
    xs, ys: (mean, std) normalisers of inputs and outputs."""
    x = (np.asarray(x_phys, dtype=np.float64) - xs[0]) / xs[1]
    outs = np.array([forward(p, x, bf16_mode)[0] * ys[1] + ys[0] for p in params])
    return outs.mean(axis=0), outs.std(axis=0)
