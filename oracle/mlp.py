"""The learned coefficient predictor: features, MLP forward/backward, loss, Adam.

Not in the paper (Algorithm 1 computes y by least squares every step); this is
the learned variant of the guess step.  Definitions shared with the GPU side
(the readings of the workload statement):

Features (160 = 4 M + s for M = 20, s = 80) of system i, computed from the
sketched block W = S [A X | b] and the coefficient vectors of the previous
four systems:
  * y_{i-k}, k = 1..4, each shifted into the current window: entry j of
    y_{i-k} refers to history column x(t_{i-k-M+j}), which is column j - k of
    the current window; entries with j - k < 0 are dropped and the k newest
    columns get 0;
  * (W1 e - wb) / ||wb||, the sketched residual of the linear extrapolation
    2 x(t_{i-1}) - x(t_{i-2}) (e = 2 e_M - e_{M-1}).
Inputs are normalised by per-feature mean and standard deviation of the
training set.

Network: h1 = GELU(W1 z + b1), h2 = GELU(W2 h1 + b2), d = W3 h2 + b3,
  y_hat = shift(y_{i-1}) + sigma_out * d
with z the normalised features, GELU(u) = u Phi(u) (exact, erf form), weights
rounded to bfloat16 (round to nearest even) for the forward and backward
passes, FP32 master weights, FP32 arithmetic.

Loss of a sample (target y, the method's least-squares coefficients, and
G = W1^T W1): (y_hat - y)^T G (y_hat - y) / ||wb||^2 -- the excess of the
sketched residual squared over its least-squares minimum, relative to
||S b||^2.  Batch loss = mean over the batch.

Adam: lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.

Parity: pinned by a float64 finite-difference check of the backward pass and
by the exact minimum of the loss at y_hat = y; the bfloat16 rounding by
comparison with its definition on chosen bit patterns.
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 160, 256, 20     # the sizes used with M = 20, s = 80 (any M, s work)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = a[nan]
    return out


def gelu(u):
    from scipy.special import erf
    return 0.5 * u * (1.0 + erf(u / math.sqrt(2.0)))


def gelu_grad(u):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(u / math.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)


def shift(y: np.ndarray, k: int) -> np.ndarray:
    """Coefficient vector of window i-k expressed in window i's frame."""
    M = y.shape[-1]
    out = np.zeros_like(y)
    if k < M:
        out[..., :M - k] = y[..., k:]
    return out


def features(W: np.ndarray, M: int, prev_y: list) -> np.ndarray:
    """prev_y[k-1] = y_{i-k} (k = 1..4), each of length M.  Returns 4M + s values."""
    W1, wb = W[:, :M], W[:, M]
    e = np.zeros(M)
    e[M - 1] = 2.0
    e[M - 2] = -1.0
    nb = np.linalg.norm(wb)
    parts = [shift(np.asarray(prev_y[k - 1], dtype=np.float64), k) for k in range(1, 5)]
    parts.append((W1 @ e - wb) / nb)
    return np.concatenate(parts)


class Params:
    def __init__(self, W1, b1, W2, b2, W3, b3, mu, sd, sig):
        self.W1, self.b1, self.W2, self.b2, self.W3, self.b3 = W1, b1, W2, b2, W3, b3
        self.mu, self.sd, self.sig = mu, sd, sig

    def arrays(self):
        return [self.W1, self.b1, self.W2, self.b2, self.W3, self.b3]


def forward(p: Params, F: np.ndarray, dtype=np.float32, round_bf16=True):
    """F: B x IN raw features.  Returns (y_hat, cache)."""
    rw = (lambda w: bf16_round(w)) if round_bf16 else (lambda w: w)
    W1, W2, W3 = (rw(p.W1).astype(dtype), rw(p.W2).astype(dtype), rw(p.W3).astype(dtype))
    z = ((F - p.mu) / p.sd).astype(dtype)
    a1 = z @ W1.T + p.b1.astype(dtype)
    h1 = gelu(a1).astype(dtype)
    a2 = h1 @ W2.T + p.b2.astype(dtype)
    h2 = gelu(a2).astype(dtype)
    d = h2 @ W3.T + p.b3.astype(dtype)
    base = F[:, :p.W3.shape[0]].astype(dtype)     # shift(y_{i-1}): the first M features
    y = base + p.sig.astype(dtype) * d
    return y, (z, a1, h1, a2, h2, W1, W2, W3)


def loss_and_grad(p: Params, F, T, G, nb, dtype=np.float32, round_bf16=True):
    """Batch-mean loss and gradients (dW1, db1, dW2, db2, dW3, db3).
    T: B x OUT targets, G: B x OUT x OUT, nb: B."""
    B = F.shape[0]
    y, (z, a1, h1, a2, h2, W1, W2, W3) = forward(p, F, dtype, round_bf16)
    e = (y - T.astype(dtype))
    Ge = np.einsum("bij,bj->bi", G.astype(dtype), e)
    inv = (1.0 / (nb.astype(dtype) ** 2))
    loss = float(np.mean(np.einsum("bi,bi->b", e, Ge) * inv))
    dy = (2.0 / B) * Ge * inv[:, None]
    dd = dy * p.sig.astype(dtype)
    dW3 = dd.T @ h2
    db3 = dd.sum(axis=0)
    dh2 = dd @ W3
    da2 = dh2 * gelu_grad(a2).astype(dtype)
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * gelu_grad(a1).astype(dtype)
    dW1 = da1.T @ z
    db1 = da1.sum(axis=0)
    return loss, [dW1, db1, dW2, db2, dW3, db3]


def adam_update(params: list, grads: list, m: list, v: list, t: int, lr=1e-3, b1=0.9, b2=0.999,
                eps=1e-8):
    """One Adam step (t counts from 1), in place on float32 arrays."""
    for w, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1 - b1) * g
        vv *= b2
        vv += (1 - b2) * g * g
        mhat = mm / (1 - b1 ** t)
        vhat = vv / (1 - b2 ** t)
        w -= (lr * mhat / (np.sqrt(vhat) + eps)).astype(w.dtype)


def he_uniform(seed: int, fan_out: int, fan_in: int, stream_offset: int) -> np.ndarray:
    """He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in)) from SplitMix64
    outputs stream_offset + 1 .. (seeded); row-major fan_out x fan_in."""
    from .sketch import splitmix64_outputs
    k = np.arange(fan_out * fan_in, dtype=np.uint64) + np.uint64(stream_offset + 1)
    u = (splitmix64_outputs(seed, k) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    bound = math.sqrt(6.0 / fan_in)
    return ((2.0 * u - 1.0) * bound).astype(np.float32).reshape(fan_out, fan_in)
