"""FP64 oracle of the learned surrogate's multilayer perceptron.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the GPU library never
imports it.  Plain numpy in float64: the forward pass, the back-propagation of
the mean-squared error and one AdamW step, written from their definitions.

With ``bf16=True`` the values are rounded to bfloat16 exactly where the GPU
kernels store them in BF16 -- the network input, the weights, every hidden
activation, and the gradients that feed the next matrix product -- so the
oracle computes what the GPU path computes up to the order of float
summation.  With ``bf16=False`` it is the exact-arithmetic network, which the
finite-difference pin checks.

Network: a_0 = x; for hidden layer l: z_l = a_{l-1} W_l^T + b_l, a_l = SiLU(z_l);
output y = a_L W_out^T + b_out.  SiLU(z) = z sigmoid(z) (Elfwing et al. 2018).
Loss: mean over valid rows r and valid outputs c of (y_rc - t_rc)^2.
AdamW: decoupled weight decay (Loshchilov & Hutter, ICLR 2019).

Parity status: pinned (tests/test_oracle_mlp.py): bfloat16 rounding against
torch's conversion, SiLU' against a central difference, gradients against
central differences of the loss, AdamW against its closed form.
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to the nearest bfloat16 (ties to even) through float32; returns float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def unflatten(flat, dims):
    """dims: list of (out_pad, in_pad) per layer -> list of (W, b) float64."""
    flat = np.asarray(flat, dtype=np.float64)
    out = []
    off = 0
    for o, i in dims:
        W = flat[off:off + o * i].reshape(o, i)
        off += o * i
        b = flat[off:off + o]
        off += o
        out.append((W.copy(), b.copy()))
    assert off == len(flat)
    return out


def flatten(parts):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in parts])


def forward(layers, X, bf=True):
    """Returns y and the cache (activations a_0..a_L, pre-activations z_1..z_L)."""
    rnd = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    a = [rnd(X)]
    z = []
    for W, b in layers[:-1]:
        zl = a[-1] @ rnd(W).T + b
        z.append(zl)
        a.append(rnd(silu(zl)))
    W, b = layers[-1]
    y = a[-1] @ rnd(W).T + b
    return y, (a, z)


def loss_and_grads(layers, X, T, n_valid, m_valid, bf=True):
    """Mean-squared error over rows < m_valid and columns < n_valid, and its
    gradients with respect to every (W, b)."""
    rnd = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    y, (a, z) = forward(layers, X, bf)
    M, N = y.shape
    mask = np.zeros_like(y)
    mask[:m_valid, :n_valid] = 1.0
    s = 1.0 / (m_valid * n_valid)
    e = (y - T) * mask
    loss = float((e * e).sum() * s)
    dy = 2.0 * e * s
    g = dy                 # gradient wrt the current pre-activation (float)
    gq = rnd(dy)           # the copy that feeds the matrix products
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        gW = gq.T @ a[l]
        gb = g.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            g = (gq @ rnd(W)) * dsilu(z[l - 1])
            gq = rnd(g)
    return loss, grads, y


def adamw(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step; returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    w = w - lr * (mh / (np.sqrt(vh) + eps) + wd * w)
    return w, m, v
