"""Plain fp64 reference of the surrogate network's arithmetic (numpy).

TEST INFRASTRUCTURE ONLY: used by tests/ and never by the product path.

The network: layer l maps dims[l] -> dims[l+1] with y = x W^T + b; hidden
layers apply GELU, GELU(z) = z * Phi(z) with Phi the standard normal CDF; the
last layer is linear.  Weights, biases and every layer's input are stored in
BF16 (round to nearest even); all arithmetic here is fp64.  Parameters are one
flat vector, per layer W (row-major [out][in]) then b.

Loss: mean squared error over the used output columns.  Optimiser: AdamW
(Loshchilov and Hutter, "Decoupled weight decay regularization", ICLR 2019):
m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr (m/(1-b1^t) /
(sqrt(v/(1-b2^t)) + eps) + wd p).
"""
from __future__ import annotations

import math

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def layers(dims, params):
    """Views (W, b) of the flat parameter vector."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        n, k = dims[l + 1], dims[l]
        W = params[o:o + n * k].reshape(n, k)
        o += n * k
        b = params[o:o + n]
        o += n
        out.append((W, b))
    return out


def param_count(dims):
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def forward(dims, params, x, bf16=True):
    """Returns the output and the per-layer (input, pre-activation) pairs."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    a = rnd(x)
    cache = []
    L = len(dims) - 1
    for l, (W, b) in enumerate(layers(dims, rnd(params))):
        z = a @ W.T + b
        cache.append((a, z))
        a = z if l == L - 1 else rnd(gelu(z))
    return a, cache


def backward(dims, params, x, dy, bf16=True):
    """Gradient of sum(dy * y) with respect to the flat parameters."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    _, cache = forward(dims, params, x, bf16)
    Ws = layers(dims, rnd(params))
    grads = []
    dz = np.asarray(dy, dtype=np.float64)
    L = len(dims) - 1
    for l in range(L - 1, -1, -1):
        a_in, _ = cache[l]
        W, _ = Ws[l]
        gW = dz.T @ a_in
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        if l == 0:
            break
        da = dz @ W
        dz = da * gelu_grad(cache[l - 1][1])
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return np.concatenate(flat)


def mse(y, t, used):
    """Loss and its gradient over the first `used` columns."""
    y = np.asarray(y, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = y.shape[0]
    d = np.zeros_like(y)
    d[:, :used] = y[:, :used] - t[:, :used]
    loss = (d[:, :used] ** 2).sum() / (B * used)
    return loss, 2.0 * d / (B * used)


def adamw(p, g, m, v, lr, b1, b2, eps, wd, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v
