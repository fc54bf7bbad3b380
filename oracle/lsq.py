"""Small dense least squares min_y || W1 y - wb ||_2 (Algorithm 1).

The paper solves the reduced problem with a QR factorisation (Section 2, the
cost paragraph after Algorithm 1, citing Golub and Van Loan).  The
history columns are nearly dependent by design (Theorem 1: their singular
values decay geometrically), so the factorisation is made rank revealing.
Readings, identical on the GPU side:

1. Column scaling: d_k = ||W1[:, k]||_2; a zero column is never pivoted and
   gets y_k = 0.  B = W1 D^-1.
2. Householder QR of B with Businger-Golub column pivoting: at step k the
   remaining column of largest 2-norm (recomputed, not downdated) is swapped
   to position k; ties go to the lowest index.
3. Reflector for x = B[k:, k]: alpha = -sign(x_0) ||x|| with sign(0) = +1,
   v = x - alpha e_1, H = I - 2 v v^T / (v^T v).
4. Rank r = number of leading k with |R_kk| > tau |R_00|.
5. z = R[:r, :r]^-1 (Q^T wb)[:r] by back substitution; y = D^-1 P [z; 0].
6. rho_s = || W1 y - wb ||_2 (the sketched residual).

Parity: pinned against LAPACK least squares on full-rank problems, the M = 1
closed form, exact consistent right-hand sides, the normal equations, and a
rank-deficient case.
"""
from __future__ import annotations

import numpy as np


def pivoted_qr_lstsq(W1: np.ndarray, wb: np.ndarray, tau: float):
    """Return (y, rank, rho_s, perm, Rdiag) for min ||W1 y - wb||_2."""
    W1 = np.asarray(W1, dtype=np.float64)
    wb = np.asarray(wb, dtype=np.float64)
    s, m = W1.shape
    y = np.zeros(m)
    if m == 0:
        return y, 0, float(np.linalg.norm(wb)), np.zeros(0, dtype=np.int64), np.zeros(0)
    d = np.sqrt(np.sum(W1 * W1, axis=0))
    B = np.zeros_like(W1)
    live = d > 0
    B[:, live] = W1[:, live] / d[live]
    c = wb.copy()
    perm = np.arange(m)
    steps = min(s, m)
    rdiag = np.zeros(steps)
    for k in range(steps):
        norms = np.sqrt(np.sum(B[k:, k:] * B[k:, k:], axis=0))
        norms[~live[perm[k:]]] = -1.0            # zero columns are never chosen
        p = k + int(np.argmax(norms))            # first maximum: lowest index
        if p != k:
            B[:, [k, p]] = B[:, [p, k]]
            perm[[k, p]] = perm[[p, k]]
        x = B[k:, k].copy()
        normx = float(np.sqrt(np.dot(x, x)))
        if normx == 0.0 or not live[perm[k]]:
            break
        alpha = -normx if x[0] >= 0.0 else normx
        v = x
        v[0] -= alpha
        vtv = float(np.dot(v, v))
        if vtv > 0.0:
            B[k:, k:] -= np.outer(v, (2.0 / vtv) * (v @ B[k:, k:]))
            c[k:] -= v * ((2.0 / vtv) * float(np.dot(v, c[k:])))
        B[k, k] = alpha
        B[k + 1:, k] = 0.0
        rdiag[k] = alpha
    r = 0
    if steps and rdiag[0] != 0.0:
        lim = tau * abs(rdiag[0])
        while r < steps and abs(rdiag[r]) > lim:
            r += 1
    z = np.zeros(r)
    for i in range(r - 1, -1, -1):               # back substitution
        z[i] = (c[i] - np.dot(B[i, i + 1:r], z[i + 1:r])) / B[i, i]
    ys = np.zeros(m)
    ys[perm[:r]] = z
    y[live] = ys[live] / d[live]
    rho = float(np.linalg.norm(W1 @ y - wb))
    return y, r, rho, perm, rdiag
