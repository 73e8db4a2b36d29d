"""FP64 reference of the learned energy-integral surrogate -- TEST INFRASTRUCTURE.

Only the tests may import this module.  The surrogate approximates ln T, the
logarithm of the energy-weighted transmission of a ray (Sec. II.F, I_f
equation), from the per-material path lengths L:

    x      = L * scale                             (8 input features)
    z1     = W1 x + b1,   h1 = SiLU(z1)            (128)
    z2     = W2 h1 + b2,  h2 = SiLU(z2)            (128)
    z3     = W3 h2 + b3,  h3 = SiLU(z3)            (128)
    y_hat  = ln sum_k a_k exp(-mu_k . L) + w4 . h3 + b4   (k = 1..4 groups)
    loss   = mean_b (y_hat - y)^2,    SiLU(z) = z / (1 + exp(-z))

Parameters arrive as the packed vector of the C ABI (W1 [128][8], b1,
W2 [128][128], b2, W3, b3, w4 [128], b4, scale [8], a [4], mu [4][8],
box [8]); (a, mu) is the energy integral with the spectrum lumped into four
groups (its one-group form is the first-order term -mubar . L).
With ``round_weights`` the three weight matrices are rounded to bf16, the
operands the tensor cores multiply (the CUDA path carries inputs and
activations as bf16 hi + lo pairs, i.e. to ~16 bits, which this reference
does not round); everything else is float64, with the exact SiLU.  The backward pass is the chain rule written out layer by layer
(pinned against central finite differences of ``loss`` in the tests).
"""
from __future__ import annotations

import numpy as np

H, NIN = 128, 8
OFF = {}
_o = 0
for _name, _size in (("W1", H * NIN), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * H),
                     ("b3", H), ("w4", H), ("b4", 1)):
    OFF[_name] = (_o, _o + _size)
    _o += _size
N_PARAMS = _o
OFF["scale"] = (_o, _o + 8)
OFF["ga"] = (_o + 8, _o + 12)
OFF["gmu"] = (_o + 12, _o + 44)
OFF["box"] = (_o + 44, _o + 52)
N_PACKED = _o + 52


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    d = {k: P[a:b] for k, (a, b) in OFF.items()}
    d["W1"] = d["W1"].reshape(H, NIN)
    d["W2"] = d["W2"].reshape(H, H)
    d["W3"] = d["W3"].reshape(H, H)
    return d


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s + z * s * (1.0 - s)


def forward(P, L, round_weights=True):
    """y_hat [n] and the intermediates of the forward pass."""
    p = unpack(P)
    L = np.asarray(L, dtype=np.float64)
    n_mat = L.shape[1]
    Lp = np.zeros((L.shape[0], NIN))
    Lp[:, :n_mat] = L
    x = Lp * p["scale"][None, :]
    W1, W2, W3 = p["W1"], p["W2"], p["W3"]
    if round_weights:
        W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
    z1 = x @ W1.T + p["b1"]
    h1 = _silu(z1)
    z2 = h1 @ W2.T + p["b2"]
    h2 = _silu(z2)
    z3 = h2 @ W3.T + p["b3"]
    h3 = _silu(z3)
    base = np.log(np.exp(-(Lp @ p["gmu"].reshape(4, NIN).T)) @ p["ga"])
    y = base + h3 @ p["w4"] + p["b4"][0]
    return y, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, W2=W2, W3=W3)


def loss_and_grad(P, L, y, round_weights=True):
    """Mean squared error and its gradient w.r.t. the N_PARAMS parameters."""
    yh, c = forward(P, L, round_weights)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    e = yh - y
    loss = float(np.mean(e * e))
    g = 2.0 * e / n                                   # dLoss / dy_hat
    p = unpack(P)
    grad = np.zeros(N_PARAMS)

    def put(name, v):
        a, b = OFF[name]
        grad[a:b] = np.ravel(v)

    put("b4", [g.sum()])
    put("w4", c["h3"].T @ g)
    dz3 = np.outer(g, p["w4"]) * _dsilu(c["z3"])
    put("W3", dz3.T @ c["h2"])
    put("b3", dz3.sum(0))
    dz2 = (dz3 @ c["W3"]) * _dsilu(c["z2"])
    put("W2", dz2.T @ c["h1"])
    put("b2", dz2.sum(0))
    dz1 = (dz2 @ c["W2"]) * _dsilu(c["z1"])
    put("W1", dz1.T @ c["x"])
    put("b1", dz1.sum(0))
    return loss, grad


def loss(P, L, y, round_weights=True):
    yh, _ = forward(P, L, round_weights)
    e = yh - np.asarray(y, dtype=np.float64)
    return float(np.mean(e * e))
