"""CPU oracle of the learned step-size proposer -- TEST INFRASTRUCTURE ONLY.

Plain numpy float64, one formula per line, for checking the library's training and
inference kernels.  Shares no code with them.

The model (the paper has none; this defines the component the library builds):
    a1 = bf16(gelu(W1 bf16(x) + b1))      W1: 64 x 12
    a2 = bf16(gelu(W2 a1 + b2))            W2: 64 x 64
    m  = W3 a2 + b3                        W3: 1 x 64
with W1, W2, W3 rounded to bfloat16 for the forward pass (the master weights stay in
float32), gelu(u) = u Phi(u) = u (1 + erf(u / sqrt 2)) / 2, and bf16() rounding to the
nearest bfloat16 (ties to even).  m estimates log2 of the largest step, relative to the
last attempted one, that the corrector would accept.

Loss of one logged corrector stage with attempted log2 step ratio r and outcome
accepted in {0, 1}: z = m - r,  l = softplus(-kappa z) if accepted else softplus(kappa z),
i.e. the logistic likelihood of the outcome with acceptance probability sigma(kappa z);
the batch loss is the mean.  The backward pass treats bf16() as the identity.

Parameter vector (float32, 5,057 entries): W1 (64x12, row-major) | b1 (64) | W2 (64x64) |
b2 (64) | W3 (64) | b3 (1).
"""
from __future__ import annotations

import math

import numpy as np

NIN, NH = 12, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)),
         ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf)


def gelu(u):
    return 0.5 * u * (1.0 + _erf(u / math.sqrt(2.0)))


def gelu_prime(u):
    return 0.5 * (1.0 + _erf(u / math.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)


def forward(p, X):
    """Returns m [B] and the cache of the backward pass."""
    w = unpack(p)
    W1, W2, W3 = bf16(w["W1"]), bf16(w["W2"]), bf16(w["W3"])
    x = bf16(X)
    u1 = x @ W1.T + w["b1"]
    a1 = bf16(gelu(u1))
    u2 = a1 @ W2.T + w["b2"]
    a2 = bf16(gelu(u2))
    m = a2 @ W3 + w["b3"][0]
    return m, (x, u1, a1, u2, a2, W1, W2, W3)


def softplus(v):
    return np.logaddexp(0.0, v)


def loss(p, X, r, acc, kappa):
    m, _ = forward(p, X)
    z = m - r
    a = np.asarray(acc, dtype=np.float64)
    l = np.where(a > 0, softplus(-kappa * z), softplus(kappa * z))
    return float(np.mean(l))


def grad(p, X, r, acc, kappa):
    """Analytic gradient of the mean loss (bf16() as the identity), and the loss."""
    m, (x, u1, a1, u2, a2, W1, W2, W3) = forward(p, X)
    B = X.shape[0]
    z = m - r
    a = np.asarray(acc, dtype=np.float64)
    sig = 1.0 / (1.0 + np.exp(-kappa * z))
    dm = kappa * (sig - a) / B                      # d mean-loss / d m
    g = {}
    g["W3"] = dm @ a2
    g["b3"] = np.array([dm.sum()])
    da2 = np.outer(dm, W3)
    du2 = da2 * gelu_prime(u2)
    g["W2"] = du2.T @ a1
    g["b2"] = du2.sum(axis=0)
    da1 = du2 @ W2
    du1 = da1 * gelu_prime(u1)
    g["W1"] = du1.T @ x
    g["b1"] = du1.sum(axis=0)
    l = np.where(a > 0, softplus(-kappa * z), softplus(kappa * z))
    return pack(g), float(np.mean(l))


def adamw(p, m1, m2, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (Loshchilov & Hutter): moments, bias correction, decoupled decay."""
    m1 = beta1 * m1 + (1 - beta1) * g
    m2 = beta2 * m2 + (1 - beta2) * g * g
    mh = m1 / (1 - beta1 ** step)
    vh = m2 / (1 - beta2 ** step)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m1, m2


def init(seed=0):
    """He-style initialisation: weights N(0, 2 / fan_in), biases 0 (float32 values)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, math.sqrt(2 / NIN), (NH, NIN)), "b1": np.zeros(NH),
         "W2": rng.normal(0, math.sqrt(2 / NH), (NH, NH)), "b2": np.zeros(NH),
         "W3": rng.normal(0, math.sqrt(1 / NH), NH), "b3": np.zeros(1)}
    return pack(d).astype(np.float32)
