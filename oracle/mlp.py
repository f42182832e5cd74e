"""Oracle of the per-column MLP closure (an extension of the method: the paper
has no learned component), float64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: L dense layers, y = W_L^T relu(... relu(W_1^T x + b_1) ...) + b_L,
with W_l stored [n_in_l][n_out_l] (row-major, inputs along rows). The GPU
kernels keep float32 master weights and compute with bfloat16 weights and
bfloat16 layer inputs, accumulating in float32; ``bf16`` here reproduces that
rounding (IEEE round-to-nearest-even to 8 significant bits) at the same
points so that the oracle evaluates the same function in float64.

Loss: mean squared error over all outputs of the batch,
L = sum((y - t)^2) / (M N). Optimiser: Adam (Kingma and Ba 2015) with bias
correction, on the float32 master weights.
"""

import numpy as np


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(sizes, rng):
    """He-uniform weights and zero biases: W_l ~ U(-a, a), a = sqrt(6/n_in)."""
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / n_in)
        params.append((rng.uniform(-a, a, (n_in, n_out)), np.zeros(n_out)))
    return params


def forward(params, x, quantize=True):
    """Returns the output and the cache of layer inputs and pre-activations."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        hin = q(h)
        z = hin @ q(W) + b
        cache.append((hin, z))
        h = np.maximum(z, 0.0) if l + 1 < len(params) else z
    return h, cache


def backward(params, cache, dy, quantize=True):
    """Gradients of sum(y * dy) with respect to every (W_l, b_l). The output
    gradient enters the weight-gradient product in bfloat16, as in the
    kernels; the hidden-layer gradients are rounded the same way."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    grads = [None] * len(params)
    g = np.asarray(dy, dtype=np.float64)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        hin, z = cache[l]
        if l + 1 < len(params):
            g = g * (z > 0.0)
        gq = q(g)
        grads[l] = (hin.T @ gq, g.sum(axis=0))
        if l > 0:
            g = gq @ q(W).T
    return grads


def mse(y, t):
    return float(np.sum((y - t) ** 2) / y.size)


def mse_grad(y, t):
    return 2.0 * (y - t) / y.size


def adam(params, grads, state, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in float64 (the kernels do it in float32)."""
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        mW, vW, mb, vb = state[l]
        mW = b1 * mW + (1 - b1) * gW
        vW = b2 * vW + (1 - b2) * gW ** 2
        mb = b1 * mb + (1 - b1) * gb
        vb = b2 * vb + (1 - b2) * gb ** 2
        c1, c2 = 1 - b1 ** step, 1 - b2 ** step
        W = W - lr * (mW / c1) / (np.sqrt(vW / c2) + eps)
        b = b - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)
        state[l] = (mW, vW, mb, vb)
        out.append((W, b))
    return out
