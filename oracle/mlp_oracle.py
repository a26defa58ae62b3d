"""FP64 reference of the learned Newton-start network (test infrastructure).

Only the tests and the smoke check import this module.

The paper has no learned component; this is the per-node multilayer perceptron the
library adds as a Newton initial guess: input 216 features (a 3x3x3 stencil x 4 fields
x 2 time levels), three hidden layers of 128 with the exact GELU x Phi(x) (Phi the
standard normal CDF, written with erf), a linear output of 3, mean-squared-error loss.
Weights are stored input-major: W[l] has shape (fan_in, fan_out) and a layer computes
Z = A W + b.  Everything is plain numpy in float64: matrix products are the library
primitive; the backward pass is the chain rule written out layer by layer.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

LAYERS = (216, 128, 128, 128, 3)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0, layers=LAYERS):
    """He-style normal initialisation (std sqrt(2/fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for fi, fo in zip(layers[:-1], layers[1:]):
        Ws.append(rng.normal(0.0, math.sqrt(2.0 / fi), (fi, fo)))
        bs.append(np.zeros(fo))
    return Ws, bs


def forward(Ws, bs, X):
    """Returns the output and the pre-activations Z_l and activations A_l of every layer."""
    A = [np.asarray(X, dtype=np.float64)]
    Z = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = A[-1] @ W + b
        Z.append(z)
        A.append(gelu(z) if l < len(Ws) - 1 else z)
    return A[-1], Z, A


def loss(Ws, bs, X, Y):
    """Mean over samples and outputs of the squared error."""
    out, _, _ = forward(Ws, bs, X)
    return float(np.mean((out - Y) ** 2))


def backward(Ws, bs, X, Y):
    """Gradients of ``loss`` with respect to every W and b (chain rule, layer by layer)."""
    out, Z, A = forward(Ws, bs, X)
    B, n_out = out.shape
    dA = 2.0 * (out - Y) / (B * n_out)
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        dZ = dA if l == len(Ws) - 1 else dA * gelu_prime(Z[l])
        gW[l] = A[l].T @ dZ
        gb[l] = dZ.sum(axis=0)
        dA = dZ @ Ws[l].T
    return gW, gb, float(np.mean((out - Y) ** 2))


def adam_step(Ws, bs, gW, gb, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; state = dict(t, m, v)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    params = Ws + bs
    grads = gW + gb
    if "m" not in state:
        state["m"] = [np.zeros_like(p) for p in params]
        state["v"] = [np.zeros_like(p) for p in params]
    for i, (p, g) in enumerate(zip(params, grads)):
        state["m"][i] = beta1 * state["m"][i] + (1 - beta1) * g
        state["v"][i] = beta2 * state["v"][i] + (1 - beta2) * g * g
        mh = state["m"][i] / (1 - beta1**t)
        vh = state["v"][i] / (1 - beta2**t)
        p -= lr * mh / (np.sqrt(vh) + eps)
    return Ws, bs


def bf16_round(x):
    """Round-to-nearest-even to bfloat16, returned as float64 (to mirror BF16 operands)."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.view(np.float32).astype(np.float64)
