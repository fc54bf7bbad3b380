"""Compressed bases of span(X) (Section 2): POD (Algorithm 2) and the
randomised range finder with progressive updates (Algorithm 4).

Test infrastructure only (see oracle/__init__.py).

Both methods replace the whole span of the history X (n x M, oldest column
first) by an m-dimensional subspace S = span(Q) with Q having orthonormal
columns; Algorithm 1 then takes the minimiser of ||A s - b|| over S.  With
the row sketch of the hot path the guess is the sketched least squares over
the chosen basis (method.sketched_guess with the basis in place of X); any
basis of the same span gives the same minimiser, so the basis need not be
orthonormalised for the guess (the functions below return the orthonormal Q
of the paper where it is cheap to form, for the pins).

POD (Algorithm 2): Q_POD = the m leading left singular vectors of X.  Its
optimality (the identity following Algorithm 2): ||(I - Q Q^T) X||_F^2 equals
the sum of the squared trailing singular values, the minimum over all
orthonormal n x m bases.

Randomised range finder (Algorithm 4): Omega = X Z with Z (M x m) Gaussian,
computed from scratch, then from one time step to the next updated in place
(the algorithm's progressive update): the contribution of the column that leaves the
history is removed with the first row of Z, the rows of Z move up by one, a
new Gaussian row is drawn for the newest solution and its contribution is
added.  The update is exact in exact arithmetic (Omega = X Z for the current Z
at all times); to bound the drift from cancellation, Omega is recomputed from
scratch with a newly drawn Z every `refresh` updates (the experiments of
Section 4 use 50).  The reduced QR of Omega gives Q.

Readings (the paper assumes a full history):
  * while the history holds M_i < M columns, Z has M_i rows and a new
    solution adds a row without removing one;
  * Omega is first computed at the first guess with a non-empty history; a
    solution pushed before that only enters the history;
  * the from-scratch recomputation happens at the guess that finds `refresh`
    or more progressive updates since the last one.

Gaussian draws (for Z from scratch and for each new row).  Draw k = 0, 1, 2, ... of a context is the
Box-Muller transform (Box and Muller, 1958) of two outputs of SplitMix64
(Steele, Lea and Flood, 2014) seeded with seed XOR 0x52414E44:
    h1 = output 2k+1,  h2 = output 2k+2,
    u1 = ((h1 >> 11) + 1) 2^-53  in (0, 1],   u2 = (h2 >> 11) 2^-53  in [0, 1),
    g  = sqrt(-2 ln u1) cos(2 pi u2).
A from-scratch Z takes M_i m consecutive draws, row by row, row l belonging
to the l-th oldest history column; a progressive update takes the next m
draws for the new row.

Parity: pinned by the Box-Muller closed forms and the moments of the stream,
progressive update = from-scratch product X Z after every step (the paper's
exactness remark), the expected-error bound of the randomised SVD (the
Halko-Martinsson-Tropp bound quoted in Section 2.2), the POD optimality
identity, and the full-span limit (m >= M_i gives the guess of the whole
span).
"""
from __future__ import annotations

import math

import numpy as np

from . import method, sketch

GAUSS_SEED_XOR = 0x52414E44


def box_muller(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """Standard normal value from u1 in (0, 1] and u2 in [0, 1)."""
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def gaussians(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the context's Gaussian stream (FP64)."""
    k = np.arange(start, start + count, dtype=np.uint64)
    gseed = (seed ^ GAUSS_SEED_XOR) & 0xFFFFFFFFFFFFFFFF
    h1 = sketch.splitmix64_outputs(gseed, 2 * k + 1)
    h2 = sketch.splitmix64_outputs(gseed, 2 * k + 2)
    u1 = ((h1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return box_muller(u1, u2)


def pod_basis(X: np.ndarray, m: int) -> np.ndarray:
    """Algorithm 2: the min(m, M) leading left singular vectors of X."""
    U, _, _ = np.linalg.svd(X, full_matrices=False)
    return U[:, :min(m, X.shape[1])]


def pod_guess(A, b, X: np.ndarray, m: int, S, tau: float = method.RANK_TOL_F64) -> method.Guess:
    """Algorithm 1 over span(Q_POD), sketched least squares."""
    if X.shape[1] == 0:
        return method.sketched_guess(A, b, X, S, tau)
    return method.sketched_guess(A, b, pod_basis(X, m), S, tau)


class RandRangeFinder:
    """State of Algorithm 4 for one sequence: Omega (n x m), the rows of Z
    (oldest history column first), the draw counter and the number of
    progressive updates since the last from-scratch Omega."""

    def __init__(self, m: int, refresh: int, seed: int):
        self.m, self.refresh, self.seed = m, refresh, seed
        self.omega = None
        self.Z: list[np.ndarray] = []
        self.counter = 0
        self.updates = 0

    def _draw(self, count: int) -> np.ndarray:
        g = gaussians(self.seed, self.counter, count)
        self.counter += count
        return g

    def from_scratch(self, X: np.ndarray) -> None:
        """From scratch: Z drawn anew (one row per history column), Omega = X Z."""
        Mi = X.shape[1]
        Z = self._draw(Mi * self.m).reshape(Mi, self.m)
        self.Z = [Z[l].copy() for l in range(Mi)]
        self.omega = X @ Z
        self.updates = 0

    def on_push(self, x_new: np.ndarray, x_leaving) -> None:
        """The progressive update for one new solution x_new; x_leaving is the
        column that leaves the history (None while the history is still
        filling)."""
        if self.omega is None:
            return
        if x_leaving is not None:
            self.omega = self.omega - np.outer(x_leaving, self.Z[0])     # leaving column out
            self.Z = self.Z[1:]                                          # rows of Z move up
        z_new = self._draw(self.m)                                       # new Gaussian row
        self.Z.append(z_new)
        self.omega = self.omega + np.outer(x_new, z_new)                 # new column in
        self.updates += 1

    def basis(self, X: np.ndarray) -> np.ndarray:
        """Omega for the guess with history X (from scratch when due)."""
        if self.omega is None or self.updates >= self.refresh:
            self.from_scratch(X)
        return self.omega

    def Zmat(self) -> np.ndarray:
        return np.stack(self.Z) if self.Z else np.zeros((0, self.m))


def orthonormal_basis(omega: np.ndarray) -> np.ndarray:
    """Reduced QR of Omega (Algorithm 4), Q factor."""
    Q, _ = np.linalg.qr(omega)
    return Q


def rand_guess(A, b, rrf: RandRangeFinder, X: np.ndarray, S,
               tau: float = method.RANK_TOL_F64) -> method.Guess:
    """Algorithm 1 over span(Omega), sketched least squares (x0 = Omega c)."""
    if X.shape[1] == 0:
        return method.sketched_guess(A, b, X, S, tau)
    return method.sketched_guess(A, b, rrf.basis(X), S, tau)
