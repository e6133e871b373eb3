"""FP64 oracle of the warm-start network (test infrastructure only).

A plain multilayer perceptron: inputs (4 features) -> hidden layers of width
256 with the erf form of GELU -> linear outputs (2 Hmax). Loss: mean squared
error over the entries whose mask is 1, divided by the mask sum. Training:
Adam on FP32-representable master weights.

With ``bf16=True`` every operand that the GPU feeds to its tensor-core
products (layer inputs, weights, back-propagated errors) is first rounded to
bfloat16 (round to nearest, ties to even), the products are then accumulated
in FP64. This isolates the accumulation order as the only difference from
the device path, which accumulates in FP32.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def bf16_round(a):
    """Round float64/float32 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    # NaN and infinity pass through unchanged
    bad = ~np.isfinite(f)
    out = np.where(bad, f, out)
    return out.astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def layer_shapes(nin=4, hidden=256, nhidden=3, nout=160):
    dims = [nin] + [hidden] * nhidden + [nout]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unflatten(params, shapes):
    """Flat FP32 layout: for each layer W (out x in, row-major) then b (out)."""
    out, k = [], 0
    for (o, i) in shapes:
        W = np.asarray(params[k:k + o * i], dtype=np.float64).reshape(o, i)
        k += o * i
        b = np.asarray(params[k:k + o], dtype=np.float64)
        k += o
        out.append((W, b))
    assert k == len(params)
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward(params, X, shapes, bf16=False):
    """Returns the outputs and the cache of pre-activations / layer inputs."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unflatten(params, shapes)
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        hin = rnd(h)
        z = hin @ rnd(W).T + b
        cache.append((hin, z))
        h = gelu(z) if li < len(layers) - 1 else z
    return h, cache


def loss_and_grads(params, X, T, mask, shapes, bf16=False):
    """Masked MSE and its gradient with respect to the flat parameters."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unflatten(params, shapes)
    Y, cache = forward(params, X, shapes, bf16)
    M = np.asarray(mask, dtype=np.float64)
    msum = max(M.sum(), 1.0)
    diff = (Y - np.asarray(T, dtype=np.float64)) * M
    loss = float((diff * diff).sum() / msum)
    dz = 2.0 * diff / msum
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        hin, z = cache[li]
        if li < len(layers) - 1:
            dz = dz * gelu_grad(z)
        dzr = rnd(dz)
        dW = dzr.T @ hin
        db = dz.sum(axis=0)
        grads.append((dW, db))
        dz = dzr @ rnd(W)  # d(loss)/d(layer input)
    grads.reverse()
    return loss, flatten(grads)


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), t counted from 1. Returns new (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grads
    v = beta2 * v + (1 - beta2) * grads * grads
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
