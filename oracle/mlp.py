"""Oracle of the learned warm start (TEST INFRASTRUCTURE ONLY): the per-node
MLP that proposes the initial guess of the elliptic-relaxation solve.

Network: 11 inputs (<U>, <V>, <W>, the six Reynolds stresses, <omega>, wall
distance), three hidden layers of 64 with GELU, 9 outputs (wp_ij); inputs
and outputs standardized with stored means and scales.  The GPU computes
every matrix product from BF16 operands with FP32 accumulation; this oracle
evaluates the same function in FP64 and rounds to BF16 at exactly the points
where the GPU does (weights, the standardized input, each hidden activation,
and in the backward pass each upstream gradient before its product), so the
two differ only by FP32 accumulation order.
The paper has no network; its warm start is the previous step's solution
(sec. 3.2).
"""
import math

import numpy as np

SIZES = (11, 64, 64, 64, 9)


def bf16(x):
    """Round to bfloat16 (round to nearest even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    rnd = ((b >> 16) & 1) + 0x7FFF
    b = ((b + rnd) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))


def gelu_grad(z):
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))
    return cdf + z * phi


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    P = {}
    for l in range(4):
        fan_in, fan_out = SIZES[l], SIZES[l + 1]
        P["W%d" % l] = rng.normal(size=(fan_out, fan_in)) * math.sqrt(2.0 / fan_in)
        P["b%d" % l] = np.zeros(fan_out)
    return P


def _ident(x):
    return np.asarray(x, dtype=np.float64)


def forward(P, Xn, keep=False, rounding=True):
    """Xn: standardized inputs [B, 11].  Returns outputs [B, 9] (standardized).
    rounding=False evaluates the exact FP64 function (for derivative checks)."""
    r = bf16 if rounding else _ident
    a = r(Xn)
    cache = [a]
    zs = []
    for l in range(4):
        z = a @ r(P["W%d" % l]).T + P["b%d" % l]
        zs.append(z)
        if l < 3:
            a = r(gelu(z))
            cache.append(a)
    y = zs[-1]
    if keep:
        return y, cache, zs
    return y


def loss_and_grads(P, Xn, Yn, rounding=True):
    """Mean squared error over the batch and the 9 outputs, and its gradients
    by backpropagation (the GPU's rounding points reproduced unless
    rounding=False)."""
    r = bf16 if rounding else _ident
    B = Xn.shape[0]
    y, acts, zs = forward(P, Xn, keep=True, rounding=rounding)
    diff = y - Yn
    loss = float(np.sum(diff * diff) / (B * 9))
    g = {}
    dz = r(2.0 * diff / (B * 9))
    for l in (3, 2, 1, 0):
        g["W%d" % l] = dz.T @ acts[l]
        g["b%d" % l] = dz.sum(axis=0)
        if l > 0:
            da = dz @ r(P["W%d" % l])
            dz = r(da * gelu_grad(zs[l - 1]))
    return loss, g
