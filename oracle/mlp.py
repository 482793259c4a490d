"""Plain FP64 reference of the surrogate network's forward pass, loss and
gradients.

TEST INFRASTRUCTURE ONLY (part of the oracle).  The surrogate is not in the
paper; it replaces the near-field Sommerfeld quadrature of one reaction
component (the I_00 integrals used by Algorithm 1's local direct
interactions) by a small network.  This module states the network's
arithmetic in the most direct form, so that the GPU training kernels'
gradients can be checked against it.

Network: 4 inputs -> 64 -> 64 -> 64 -> 3, SiLU after each hidden layer,
    z1 = W1 x + b1, a1 = silu(z1), ..., out = W4 a3 + b4,
loss = (1/n) sum_samples sum_outputs (out - y)^2.
Parameter vector layout (float32 on the device): W1[64][4], b1[64],
W2[64][64], b2[64], W3[64][64], b3[64], W4[3][64], b4[3].
The forward pass uses the weight matrices rounded to bfloat16 (round to
nearest even), biases in float32 - as the device does.
"""
from __future__ import annotations

import numpy as np

H, NIN, NOUT = 64, 4, 3
SHAPES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (NOUT, H)), ("b4", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, quantize=True):
    p = unpack(theta)
    W = {k: (bf16_round(v) if (quantize and k.startswith("W")) else v) for k, v in p.items()}
    z1 = x @ W["W1"].T + W["b1"]
    a1 = silu(z1)
    z2 = a1 @ W["W2"].T + W["b2"]
    a2 = silu(z2)
    z3 = a2 @ W["W3"].T + W["b3"]
    a3 = silu(z3)
    out = a3 @ W["W4"].T + W["b4"]
    return out, (x, z1, a1, z2, a2, z3, a3, W)


def loss_and_grad(theta, x, y, quantize=True):
    """Loss and its gradient with respect to the parameter vector (the
    gradient of the bfloat16-rounded weights is applied to the master
    weights, i.e. a straight-through estimate)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    out, (x, z1, a1, z2, a2, z3, a3, W) = forward(theta, x, quantize)
    r = out - y
    loss = float(np.sum(r * r) / n)
    d4 = 2.0 * r / n
    g = {}
    g["W4"] = d4.T @ a3
    g["b4"] = d4.sum(0)
    d3 = (d4 @ W["W4"]) * dsilu(z3)
    g["W3"] = d3.T @ a2
    g["b3"] = d3.sum(0)
    d2 = (d3 @ W["W3"]) * dsilu(z2)
    g["W2"] = d2.T @ a1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ W["W2"]) * dsilu(z1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(0)
    grad = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    return loss, grad
