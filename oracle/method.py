"""Algorithm 1 of the paper with S = span(X) and a row-sketched reduced problem.

Algorithm 1 (Section 2) builds the guess for system i from the history
X = [x(t_{i-M}) | ... | x(t_{i-1})] (oldest first) as the element of a
subspace of span(X) that minimises ||A(t_i) s - b(t_i)||_2, then runs the
Krylov solver from it.  With the whole span (Section 2, cost paragraph after
Algorithm 1) the minimiser is X y* with y* = argmin ||A X y - b||.  The
hot path replaces that n-row problem by its sketch:

    W  = S [A X | b]                    (s x (m+1), S sparse-sign, see sketch.py)
    y  = argmin_y || W[:, :m] y - W[:, m] ||_2      (see lsq.py)
    x0 = X y

Start-up (a reading; Algorithm 1 assumes M solutions exist): system 0 starts
from x0 = 0 and system i < M uses the i columns it has.  The history is
shifted by one column per system: the oldest column leaves and the newest
solution is appended (Section 2.1).

Parity: pinned (S = I equals the dense unsketched projection; exactness when
b lies in A span(X); residual decay in M for analytic data, Theorem 2; dense
LU on tiny systems).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import krylov, lsq, sketch

RANK_TOL_F64 = 1e-12
RANK_TOL_F32 = 1e-5


@dataclasses.dataclass
class Guess:
    x0: np.ndarray
    y: np.ndarray
    W: np.ndarray          # s x (m+1) sketched block (empty for other modes)
    rank: int
    rho_s: float           # sketched residual ||W1 y - wb||


def sketched_guess(A, b, X: np.ndarray, S, tau: float = RANK_TOL_F64) -> Guess:
    """x0 = X y with y = argmin ||S (A X y - b)||_2 (X oldest column first)."""
    n, m = X.shape
    if m == 0:
        return Guess(np.zeros(n), np.zeros(0), np.zeros((S.shape[0], 1)), 0,
                     float(np.linalg.norm(S @ b)))
    W = sketch.sketch_block(S, A, X, b)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(W[:, :m], W[:, m], tau)
    return Guess(X @ y, y, W, rank, rho)


def projected_guess(A, b, X: np.ndarray, tau: float = RANK_TOL_F64) -> Guess:
    """Unsketched projection (S = I): x0 = X y*, y* = argmin ||A X y - b||_2."""
    n, m = X.shape
    if m == 0:
        return Guess(np.zeros(n), np.zeros(0), np.zeros((n, 1)), 0, float(np.linalg.norm(b)))
    AX = np.asarray(A @ X)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(AX, b, tau)
    return Guess(X @ y, y, np.zeros((0, 0)), rank, rho)


def previous_guess(X: np.ndarray) -> np.ndarray:
    """The paper's baseline guess x0 = x(t_{i-1}) (0 with an empty history)."""
    n, m = X.shape
    return X[:, m - 1].copy() if m else np.zeros(n)


class History:
    """The last M solutions, oldest first."""

    def __init__(self, n: int, M: int):
        self.n, self.M = n, M
        self.cols: list[np.ndarray] = []

    def push(self, x: np.ndarray) -> None:
        self.cols.append(np.array(x, dtype=np.float64, copy=True))
        if len(self.cols) > self.M:
            self.cols.pop(0)

    def matrix(self) -> np.ndarray:
        if not self.cols:
            return np.zeros((self.n, 0))
        return np.stack(self.cols, axis=1)


def relres(A, b, x) -> float:
    """||b - A x|| / ||b||; the absolute residual when b = 0 (then undefined
    relative to b; x = 0 solves the system exactly)."""
    rn = float(np.linalg.norm(b - A @ x))
    bn = float(np.linalg.norm(b))
    return rn / bn if bn > 0 else rn


def solve_step(A, b, hist: History, S, tol: float, krylov_kind: str,
               guess: str = "sketch", restart: int = 30, max_iters: int = 30000,
               precond=None):
    """One system of the sequence: guess, Krylov solve, push.  Returns a dict."""
    X = hist.matrix()
    if guess == "sketch":
        g = sketched_guess(A, b, X, S)
        x0 = g.x0
    elif guess == "projected":
        g = projected_guess(A, b, X)
        x0 = g.x0
    else:
        g = None
        x0 = previous_guess(X)
    r0 = relres(A, b, x0)
    if krylov_kind == "cg":
        x, it, rel, st = krylov.cg(A, b, x0, tol, max_iters)
    else:
        minv = krylov.jacobi_sweeps(A, *precond) if precond else None
        x, it, rel, st = krylov.gmres(A, b, x0, tol, restart, max_iters, minv=minv)
    hist.push(x)
    return {"x": x, "x0": x0, "guess_relres": r0, "iters": it, "relres": rel,
            "status": st, "rank": g.rank if g else 0, "rho_s": g.rho_s if g else 0.0,
            "y": g.y if g else None}


def sketched_guess_mixed(A32, b, X32: np.ndarray, S, tau: float = RANK_TOL_F32) -> Guess:
    """Mixed-precision guess: W = S [A32 X32 | b] formed in float32 arithmetic
    (float32 products and sums), the reduced least squares in FP64, and
    x0 = X32 y accumulated in FP64 (the history is stored in float32)."""
    n, m = X32.shape
    if m == 0:
        return Guess(np.zeros(n), np.zeros(0), np.zeros((S.shape[0], 1)), 0,
                     float(np.linalg.norm(S @ b)))
    S32 = S.astype(np.float32)
    Y = np.column_stack([A32 @ X32, b.astype(np.float32)])
    W = np.asarray(S32 @ Y).astype(np.float64)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(W[:, :m], W[:, m], tau)
    return Guess(X32.astype(np.float64) @ y, y, W, rank, rho)


def solve_step_mixed(A64, A32, b, hist: History, S, tol: float, krylov_kind: str,
                     restart: int = 30, max_iters: int = 30000, inner_tol: float = 1e-2):
    """One system in mixed precision: float32 history, float32 sketch, FP64
    least squares and FP64 refinement around float32 inner solves."""
    X32 = hist.matrix().astype(np.float32)
    g = sketched_guess_mixed(A32, b, X32, S)
    r0 = relres(A64, b, g.x0)
    x, it, nref, rel, st = krylov.mixed_refine(A64, A32, b, g.x0, tol, krylov_kind, restart,
                                               max_iters, inner_tol=inner_tol)
    hist.push(x.astype(np.float32).astype(np.float64))
    return {"x": x, "x0": g.x0, "guess_relres": r0, "iters": it, "refinements": nref,
            "relres": rel, "status": st, "rank": g.rank, "rho_s": g.rho_s, "y": g.y}


def batched_step(systems, hists, sketches, tol: float, max_iters: int = 100000,
                 inner_tol: float = 1e-2):
    """One time step of independent SPD sequences: for each sequence, the
    sketched guess from its own history (FP64), then FP64 refinement around
    float32 CG, then the push.  systems: list of (A, b); hists: list of History;
    sketches: list of S.  Returns per-sequence dicts."""
    out = []
    for (A, b), h, S in zip(systems, hists, sketches):
        g = sketched_guess(A, b, h.matrix(), S)
        x, it, nref, rel, st = krylov.mixed_refine(A, A.astype(np.float32), b, g.x0, tol, "cg",
                                                   30, max_iters, inner_tol=inner_tol)
        h.push(x)
        out.append({"x": x, "x0": g.x0, "iters": it, "refinements": nref, "relres": rel,
                    "status": st, "guess_relres": relres(A, b, g.x0), "rank": g.rank,
                    "rho_s": g.rho_s})
    return out
