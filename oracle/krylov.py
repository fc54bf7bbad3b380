"""Krylov solvers started from the subspace guess (the solve of Algorithm 1).

The paper runs GMRES (Saad and Schultz) for general matrices and names CG
(Hestenes and Stiefel) for symmetric positive definite ones (Section 1); both
stop on the residual relative to ||b||.  That reading is the one under which
the paper's observation that many systems need no iteration at all (the guess
already meets the tolerance, Sections 4 and 5) can happen.  Conventions shared with the GPU side:

* an iteration is one product with A inside the loop (one Arnoldi step for
  GMRES, one search direction for CG);
* CG: when the recursive residual passes the test, the true residual b - A x
  is recomputed; if it fails, CG restarts from it (the count continues);
  p^T A p <= 0 is a breakdown;
* GMRES(m): CGS2 Arnoldi (two classical Gram-Schmidt passes, h = h1 + h2),
  Givens rotations with r = hypot(a, b), inner stop when |g_{j+1}| <= tol ||b||,
  happy breakdown when h_{j+1,j} <= 1e-14 ||h_{:,j}||, and the true residual
  recomputed at every restart;
* preconditioned GMRES (optional): right preconditioning, GMRES on A M^{-1}
  with x = x0 + M^{-1} V y, so the minimised residual is the true one and the
  stopping test is unchanged; M^{-1} = a fixed number of damped Jacobi sweeps
  on A z = u from z = 0, or the Chebyshev polynomial of the same degree on an
  interval [lmax / ratio, lmax] of the spectrum of D^{-1} A (lmax from
  Gershgorin's theorem) -- polynomials in D^{-1} A times D^{-1}; Jacobi and
  polynomial preconditioners are the GPU-friendly members of the family the
  paper's runs use, ILU and AMG, Sections 4-5;
* mixed refinement: r = b - A64 x in FP64; the correction d solves
  A32 d = r (r rounded to float32; the same as solving for r / ||r|| and
  scaling back, in exact arithmetic) by the same solver run entirely in
  float32, to a relative residual max(inner_tol, theta * tol ||b|| / ||r||);
  x += d in FP64.
  A GMRES inner solve is a single restart cycle, so every restart begins from
  a residual formed in FP64 (GMRES-based iterative refinement).

Status codes: 0 converged, 1 not converged within max_iters, -4 breakdown.

* direct solve (reference solutions): sparse LU with column approximate
  minimum degree ordering (SuperLU through scipy, the library primitive),
  followed by FP64 iterative refinement with the same factors; used to state
  the error of the iterative solutions against the exact one.

Parity: pinned by dense LU on small systems, finite termination of full
GMRES, CG's k-step termination on k distinct eigenvalues, the Arnoldi
relation and the orthogonality of the Krylov basis; the direct solve by dense
LU and by its refined residual.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse

CONVERGED = 0
NOT_CONVERGED = 1
BREAKDOWN = -4


def csr(rowptr, colind, values, n: int) -> scipy.sparse.csr_matrix:
    """The CSR triple as a scipy matrix (scipy's product is the SpMV primitive)."""
    return scipy.sparse.csr_matrix((values, colind, rowptr), shape=(n, n))


def cg(A, b, x, tol: float, max_iters: int):
    """Conjugate gradients from x.  Returns (x, iterations, relres, status)."""
    dt = b.dtype
    x = x.astype(dt, copy=True)
    bnorm = math.sqrt(float(np.dot(b, b)))
    target = tol * bnorm
    r = b - A @ x
    rr = np.dot(r, r)
    it = 0
    if math.sqrt(float(rr)) <= target:
        return x, 0, math.sqrt(float(rr)) / bnorm, CONVERGED
    p = r.copy()
    while True:
        if it >= max_iters:
            return x, it, math.sqrt(float(np.dot(r, r))) / bnorm, NOT_CONVERGED
        q = A @ p
        pq = np.dot(p, q)
        if not pq > 0:
            return x, it, math.sqrt(float(rr)) / bnorm, BREAKDOWN
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.dot(r, r)
        it += 1
        if math.sqrt(float(rr_new)) <= target:
            r = b - A @ x
            rr = np.dot(r, r)
            if math.sqrt(float(rr)) <= target:
                return x, it, math.sqrt(float(rr)) / bnorm, CONVERGED
            p = r.copy()
            continue
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p


def jacobi_sweeps(A, sweeps: int, omega: float):
    """M^{-1} u = the result of `sweeps` damped Jacobi sweeps on A z = u from
    z = 0:  z_1 = omega D^{-1} u,  z_{k+1} = z_k + omega D^{-1} (u - A z_k),
    with D = diag(A) in A's precision.  Equals sum_{k<sweeps} (I - omega
    D^{-1} A)^k omega D^{-1} (a fixed linear operator).  sweeps = 0: identity."""
    if sweeps <= 0:
        return None
    dinv = 1.0 / A.diagonal()
    om = dinv.dtype.type(omega)

    def minv(u):
        z = (om * dinv) * u
        for _ in range(sweeps - 1):
            z = z + (om * dinv) * (u - A @ z)
        return z
    return minv


def gershgorin_bound(A) -> float:
    """max_i (sum_j |a_ij|) / |a_ii| -- by Gershgorin's theorem every eigenvalue
    of D^{-1} A lies in a disc of that radius about the origin, so it bounds the
    spectrum from above.  Row sums in CSR order, FP64."""
    A = scipy.sparse.csr_matrix(A)
    absrow = np.add.reduceat(np.abs(A.data.astype(np.float64)), A.indptr[:-1]) \
        if A.nnz else np.zeros(A.shape[0])
    absrow[np.diff(A.indptr) == 0] = 0.0
    d = np.abs(A.diagonal().astype(np.float64))
    d[d == 0] = 1.0
    return float(np.max(absrow / d))


def chebyshev_sweeps(A, degree: int, lmin: float, lmax: float, dinv=None):
    """M^{-1} u = p(D^{-1} A) D^{-1} u for the degree-`degree` polynomial whose
    residual polynomial 1 - lam p(lam) is T_d((theta - lam) / delta) / T_d(theta /
    delta) (theta, delta the centre and half-width of [lmin, lmax]): among
    polynomials of that degree it has the smallest maximum of |1 - lam p(lam)|
    on [lmin, lmax] (Chebyshev).  Applied by the three-term recurrence of the
    Chebyshev iteration on A z = u from z = 0, with D^{-1} A as the operator:
        sigma = theta / delta, rho_0 = 1 / sigma,
        d_0 = D^{-1} u / theta, z_1 = d_0,
        for k = 1 .. degree - 1:
            r_k = u - A z_k,  rho_k = 1 / (2 sigma - rho_{k-1}),
            d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^{-1} r_k,
            z_{k+1} = z_k + d_k.
    That is degree applications of D^{-1} and degree - 1 products with A, the
    cost of `degree` damped Jacobi sweeps.  `dinv` replaces 1 / diag(A) (tests
    use it to evaluate the polynomial on a diagonal operator).  degree = 0:
    identity."""
    if degree <= 0:
        return None
    if dinv is None:
        dinv = 1.0 / A.diagonal()
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta

    def minv(u):
        dt = u.dtype.type
        dv = dinv.astype(u.dtype, copy=False)
        d = (dv * u) * dt(1.0 / theta)
        z = d.copy()
        rho_prev = 1.0 / sigma
        for _ in range(degree - 1):
            r = u - A @ z
            rho = 1.0 / (2.0 * sigma - rho_prev)
            d = dt(rho * rho_prev) * d + dt(2.0 * rho / delta) * (dv * r)
            z = z + d
            rho_prev = rho
        return z
    return minv


def gmres(A, b, x, tol: float, restart: int, max_iters: int, record=None, minv=None):
    """Restarted GMRES with CGS2 Arnoldi from x, right-preconditioned by the
    linear operator `minv` when given.  Returns (x, iters, relres, status).

    ``record`` (optional list) receives (V, Hbar) of every cycle, for tests of
    the Arnoldi relation (of A M^{-1} when preconditioned).
    """
    dt = b.dtype
    x = x.astype(dt, copy=True)
    n = b.shape[0]
    bnorm = math.sqrt(float(np.dot(b, b)))
    target = tol * bnorm
    it = 0
    while True:
        r = b - A @ x
        beta = math.sqrt(float(np.dot(r, r)))
        if beta <= target:
            return x, it, beta / bnorm, CONVERGED
        if it >= max_iters:
            return x, it, beta / bnorm, NOT_CONVERGED
        V = np.zeros((n, restart + 1), dtype=dt, order="F")     # columns contiguous
        H = np.zeros((restart + 1, restart))          # Hessenberg, FP64 always
        Hbar = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / dt.type(beta)
        k = 0
        for j in range(restart):
            w = A @ (V[:, j] if minv is None else minv(V[:, j]))
            h1 = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h1
            h2 = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h2
            h = h1.astype(np.float64) + h2.astype(np.float64)
            hn = math.sqrt(float(np.dot(w, w)))
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            Hbar[:j + 2, j] = H[:j + 2, j]
            for i in range(j):                        # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a_, b_ = H[j, j], H[j + 1, j]
            rr = math.hypot(a_, b_)
            if rr == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = a_ / rr, b_ / rr
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if hn > 0.0:
                V[:, j + 1] = w / dt.type(hn)
            happy = hn <= 1e-14 * math.sqrt(float(np.dot(h, h)) + hn * hn)
            if happy or abs(g[j + 1]) <= target or it >= max_iters:
                break
        if any(H[i, i] == 0.0 for i in range(k)):
            return x, it, beta / bnorm, BREAKDOWN
        yk = np.zeros(k)
        for i in range(k - 1, -1, -1):                # back substitution
            yk[i] = (g[i] - np.dot(H[i, i + 1:k], yk[i + 1:k])) / H[i, i]
        if record is not None:
            record.append((V[:, :k + 1].copy(), Hbar[:k + 1, :k].copy()))
        step = V[:, :k] @ yk.astype(dt)
        x = x + (step if minv is None else minv(step))


def mixed_refine(A64, A32, b, x, tol: float, inner: str, restart: int,
                 max_iters: int, inner_tol: float = 1e-2, theta: float = 0.5,
                 max_refinements: int = None, precond=None):
    """FP32-inner / FP64-outer iterative refinement.  Returns
    (x, inner_iterations, refinements, relres, status).

    A GMRES inner solve is one restart cycle (at most `restart` iterations):
    every restart of the restarted GMRES starts from a residual formed in
    FP64 by the refinement.  (Restarting inside the float32 solve would form
    the residual in float32, whose rounding noise, about u32 cond(A) ||r||,
    stalls the inner solve on ill-conditioned systems.)  The number of
    refinements is bounded by max_iters, each costing at least one iteration,
    unless max_refinements is given."""
    x = x.astype(np.float64, copy=True)
    bnorm = math.sqrt(float(np.dot(b, b)))
    target = tol * bnorm
    total = 0
    refinements = 0
    while True:
        r = b - A64 @ x
        rn = math.sqrt(float(np.dot(r, r)))
        if rn <= target:
            return x, total, refinements, rn / bnorm, CONVERGED
        if (max_refinements is not None and refinements >= max_refinements) or total >= max_iters:
            return x, total, refinements, rn / bnorm, NOT_CONVERGED
        # The inner equation A d = r / ||r|| (the correction is ||r|| d): the
        # Krylov iterates scale with the right-hand side and the inner
        # tolerance is relative, so this is the same solve in exact
        # arithmetic, and the float32 right-hand side stays in range whatever
        # the scale of b.
        rhs32 = (r / rn).astype(np.float32)
        itol = max(inner_tol, theta * target / rn)
        d0 = np.zeros_like(rhs32)
        budget = max_iters - total
        if inner == "cg":
            d, it, _, st = cg(A32, rhs32, d0, itol, budget)
        else:
            minv = (precond(A32) if callable(precond) else jacobi_sweeps(A32, *precond)) \
                if precond else None
            d, it, _, st = gmres(A32, rhs32, d0, itol, restart, min(restart, budget), minv=minv)
        total += it
        refinements += 1
        if st == BREAKDOWN:
            return x, total, refinements, rn / bnorm, BREAKDOWN
        x = x + rn * d.astype(np.float64)


def direct_solve(A, b, refinements: int = 2):
    """x = A^{-1} b by sparse LU (SuperLU, COLAMD column ordering) and
    `refinements` steps of FP64 iterative refinement x += LU^{-1}(b - A x).
    Returns (x, relres) with relres = ||b - A x|| / ||b||."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(scipy.sparse.csc_matrix(A), permc_spec="COLAMD")
    x = lu.solve(b)
    for _ in range(refinements):
        x = x + lu.solve(b - A @ x)
    bnorm = math.sqrt(float(np.dot(b, b)))
    r = b - A @ x
    return x, math.sqrt(float(np.dot(r, r))) / bnorm
