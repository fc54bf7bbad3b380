"""Pins of the oracle's Krylov solvers (CPU only)."""
import numpy as np
import pytest
import scipy.sparse

import workloads
from oracle import krylov


def _system(p, i):
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    return krylov.csr(rowptr, colind, vals, p.n), b


def test_cg_matches_dense_lu():
    A, b = _system(workloads.plain_spd(12), 4)
    x_ref = np.linalg.solve(A.toarray(), b)
    x, it, rel, st = krylov.cg(A, b, np.zeros_like(b), 1e-12, 10000)
    assert st == krylov.CONVERGED and rel <= 1e-12
    kappa = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= kappa * 1e-12


def test_cg_terminates_in_k_steps_on_k_distinct_eigenvalues():
    eig = np.repeat([1.0, 2.0, 5.0, 11.0, 30.0], 40)         # 5 distinct values
    A = scipy.sparse.diags(eig).tocsr()
    b = np.random.default_rng(0).standard_normal(eig.size)
    x, it, rel, st = krylov.cg(A, b, np.zeros_like(b), 1e-12, 100)
    assert st == krylov.CONVERGED and it <= 5


def test_cg_breakdown_on_indefinite():
    A = scipy.sparse.diags([1.0, -1.0]).tocsr()
    b = np.array([1.0, 1.0])
    _, _, _, st = krylov.cg(A, b, np.zeros(2), 1e-12, 10)
    assert st == krylov.BREAKDOWN


def test_zero_iterations_from_exact_guess():
    A, b = _system(workloads.plain_nonsym(10), 2)
    x_ref = np.linalg.solve(A.toarray(), b)
    for solver in ("cg", "gmres"):
        if solver == "cg":
            _, it, rel, st = krylov.cg(A, b, x_ref, 1e-10, 100)
        else:
            _, it, rel, st = krylov.gmres(A, b, x_ref, 1e-10, 30, 100)
        assert it == 0 and st == krylov.CONVERGED


def test_gmres_matches_dense_lu():
    A, b = _system(workloads.plain_nonsym(14), 7)
    x_ref = np.linalg.solve(A.toarray(), b)
    x, it, rel, st = krylov.gmres(A, b, np.zeros_like(b), 1e-11, 30, 20000)
    assert st == krylov.CONVERGED and rel <= 1e-11
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    kappa = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= kappa * 1e-11


def test_full_gmres_terminates_in_n_steps():
    rng = np.random.default_rng(1)
    n = 25
    A = scipy.sparse.csr_matrix(rng.standard_normal((n, n)) + 6 * np.eye(n))
    b = rng.standard_normal(n)
    x, it, rel, st = krylov.gmres(A, b, np.zeros(n), 1e-12, n, 10 * n)
    assert st == krylov.CONVERGED and it <= n


def test_arnoldi_relation_and_orthogonality():
    A, b = _system(workloads.plain_nonsym(16), 1)
    rec = []
    krylov.gmres(A, b, np.zeros_like(b), 1e-14, 30, 30, record=rec)
    V, Hbar = rec[0]
    k = Hbar.shape[1]
    lhs = A @ V[:, :k]
    rhs = V @ Hbar
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)
    G = V.T @ V
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-13


def test_gmres_residual_estimate_matches_true_residual():
    """After one cycle the Givens estimate |g_k| equals ||b - A x||."""
    A, b = _system(workloads.plain_nonsym(16), 5)
    x1, it, rel, st = krylov.gmres(A, b, np.zeros_like(b), 1e-30, 30, 30)
    true = np.linalg.norm(b - A @ x1)
    # Direct dense minimisation over the same Krylov space gives the same residual.
    K = np.zeros((b.size, 30))
    v = b / np.linalg.norm(b)
    for j in range(30):
        K[:, j] = v
        v = A @ v
        for i in range(j + 1):
            v -= np.dot(K[:, i], v) * K[:, i]
        v -= K[:, :j + 1] @ (K[:, :j + 1].T @ v)
        v /= np.linalg.norm(v)
    AK = A @ K
    z = np.linalg.lstsq(AK, b, rcond=None)[0]
    assert true == pytest.approx(np.linalg.norm(AK @ z - b), rel=1e-6)


def test_mixed_refinement_reaches_fp64_tolerance():
    p = workloads.plain_nonsym(24)
    A, b = _system(p, 3)
    A32 = A.astype(np.float32)
    x, inner, nref, rel, st = krylov.mixed_refine(A, A32, b, np.zeros_like(b), 1e-10,
                                                  "gmres", 30, 20000)
    assert st == krylov.CONVERGED and rel <= 1e-10 and nref >= 2
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)


def test_mixed_refinement_cg_inner():
    p = workloads.plain_spd(24)
    A, b = _system(p, 3)
    x, inner, nref, rel, st = krylov.mixed_refine(A, A.astype(np.float32), b,
                                                  np.zeros_like(b), 1e-10, "cg", 30, 20000)
    assert st == krylov.CONVERGED and rel <= 1e-10


def _two_level_diagonal(k=8):
    """A = diag(1, 3, 1, 3, ...) and b = ones (2k unknowns).  For a right-hand
    side whose entries on the two halves have equal magnitude, the first CG
    step has alpha = (r.r)/(r.Ar) = 1/2 exactly and leaves r1 = r0 (1 - lambda/2):
    the magnitudes halve and the signs on the lambda = 3 half flip, so the
    pattern repeats.  The second CG step solves exactly (two distinct
    eigenvalues).  All values are powers of two, exact in float32."""
    d = np.tile([1.0, 3.0], k)
    A = scipy.sparse.diags(d).tocsr()
    return A, A.astype(np.float32), np.ones(2 * k)


@pytest.mark.parametrize("tol,theta,inner_tol,iters,refs", [
    # inner tolerance max(0.1, 0.5 * 0.6) = 0.3 < 1/2: the inner CG takes both
    # steps, one refinement suffices
    (0.6, 0.5, 0.1, 2, 1),
    # max(0.1, 0.9 * 0.6) = 0.54 >= 1/2: one inner step, residual 1/2 <= 0.6
    (0.6, 0.9, 0.1, 1, 1),
    # the floor 0.55 governs: one step, residual 1/2 <= 0.6
    (0.6, 0.5, 0.55, 1, 1),
    # one step per refinement: residuals 1/2 > 0.3, then 1/4 <= 0.3
    (0.3, 0.5, 0.55, 2, 2),
    # residual 2^-k after k refinements: ten to pass 1.5 * 2^-10
    (1.5 * 2.0 ** -10, 0.5, 0.55, 10, 10),
])
def test_mixed_refinement_inner_tolerance_and_count(tol, theta, inner_tol, iters, refs):
    """The inner relative tolerance is max(inner_tol, theta tol ||b|| / ||r||)
    and every refinement is one inner solve from d = 0; on the two-level
    diagonal system the CG residuals are known in closed form, so the inner
    iterations and refinements of each case follow by hand (comments above)."""
    A64, A32, b = _two_level_diagonal()
    x, inner, nref, rel, st = krylov.mixed_refine(A64, A32, b, np.zeros_like(b), tol, "cg", 30,
                                                  1000, inner_tol=inner_tol, theta=theta)
    assert st == krylov.CONVERGED
    assert (inner, nref) == (iters, refs)
    if iters == refs:       # one halving step per refinement: exact residual 2^-refs
        assert rel == 2.0 ** -refs


@pytest.mark.parametrize("scale", [1e-36, 1e30])
def test_mixed_refinement_is_scale_invariant(scale):
    """b scaled by 1e-36 (its float32 image would be subnormal or zero) or
    1e30: the inner float32 solves see r / ||r||, so refinements, inner
    iterations and the relative residual history do not change, and x scales
    with b."""
    A64, A32, b = _two_level_diagonal()
    ref = krylov.mixed_refine(A64, A32, b, np.zeros_like(b), 1.5 * 2.0 ** -10, "cg", 30, 1000,
                              inner_tol=0.55, max_refinements=50)
    got = krylov.mixed_refine(A64, A32, b * scale, np.zeros_like(b), 1.5 * 2.0 ** -10, "cg", 30,
                              1000, inner_tol=0.55, max_refinements=50)
    assert got[4] == krylov.CONVERGED and ref[4] == krylov.CONVERGED
    assert got[1:3] == ref[1:3] == (10, 10)
    assert got[3] == pytest.approx(ref[3], rel=1e-12)
    assert np.allclose(got[0], ref[0] * scale, rtol=1e-12, atol=0)


def test_mixed_refinement_refinement_cap():
    """max_refinements stops the loop with NOT_CONVERGED and the residual
    reached: 2^-3 after three halving refinements."""
    A64, A32, b = _two_level_diagonal()
    x, inner, nref, rel, st = krylov.mixed_refine(A64, A32, b, np.zeros_like(b), 1e-6, "cg", 30,
                                                  1000, inner_tol=0.55, max_refinements=3)
    assert st == krylov.NOT_CONVERGED and nref == 3 and inner == 3 and rel == 2.0 ** -3
    assert np.array_equal(np.abs(b - A64 @ x), np.full(b.size, 2.0 ** -3))


def test_not_converged_status():
    A, b = _system(workloads.plain_nonsym(20), 1)
    x, it, rel, st = krylov.gmres(A, b, np.zeros_like(b), 1e-12, 30, 7)
    assert st == krylov.NOT_CONVERGED and it == 7 and rel > 1e-12


def test_arnoldi_relation_on_stiff_operator():
    """Eigenvalues spread over 12 decades: CGS2 keeps V orthonormal to rounding
    and A V_k = V_{k+1} Hbar holds to rounding."""
    n = 300
    A = scipy.sparse.diags(np.logspace(0, 12, n)).tocsr()
    b = np.ones(n)
    rec = []
    krylov.gmres(A, b, np.zeros(n), 1e-30, 30, 30, record=rec)
    V, Hbar = rec[0]
    lhs = A @ V[:, :30]
    assert np.linalg.norm(lhs - V @ Hbar) <= 1e-14 * np.linalg.norm(lhs)
    assert np.abs(V.T @ V - np.eye(31)).max() < 1e-13


# ---- right preconditioning by damped Jacobi sweeps --------------------------

def _nonsym(N=12, i=3):
    import workloads
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    return krylov.csr(rowptr, colind, vals, p.n), b


def test_jacobi_sweeps_one_sweep_is_scaled_jacobi():
    A, b = _nonsym()
    minv = krylov.jacobi_sweeps(A, 1, 0.8)
    np.testing.assert_array_equal(minv(b), (0.8 * (1.0 / A.diagonal())) * b)
    assert krylov.jacobi_sweeps(A, 0, 0.8) is None


@pytest.mark.parametrize("d,omega", [(2, 0.8), (5, 0.7), (8, 1.0)])
def test_jacobi_sweeps_equal_the_neumann_polynomial(d, omega):
    """The recurrence equals sum_{k<d} (I - omega D^-1 A)^k omega D^-1."""
    A, b = _nonsym(8)
    Ad = A.toarray()
    n = Ad.shape[0]
    Dinv = np.diag(1.0 / np.diag(Ad))
    T = np.eye(n) - omega * Dinv @ Ad
    P = np.zeros((n, n))
    Tk = np.eye(n)
    for _ in range(d):
        P += Tk @ (omega * Dinv)
        Tk = Tk @ T
    u = np.random.default_rng(d).standard_normal(n)
    got = krylov.jacobi_sweeps(A, d, omega)(u)
    np.testing.assert_allclose(got, P @ u, rtol=1e-12, atol=1e-12 * np.abs(P @ u).max())


def test_jacobi_sweeps_converge_to_the_inverse_on_a_dominant_matrix():
    rng = np.random.default_rng(3)
    n = 40
    M = rng.standard_normal((n, n)) * 0.1
    M += np.diag(np.abs(M).sum(axis=1) + 1.0)          # strictly diagonally dominant
    import scipy.sparse as sp
    A = sp.csr_matrix(M)
    u = rng.standard_normal(n)
    z = krylov.jacobi_sweeps(A, 300, 1.0)(u)
    np.testing.assert_allclose(z, np.linalg.solve(M, u), rtol=1e-12, atol=1e-12)


def test_preconditioned_gmres_exact_inverse_takes_one_iteration():
    A, b = _nonsym(10)
    lu = scipy.sparse.linalg.splu(A.tocsc())
    x, it, rel, st = krylov.gmres(A, b, np.zeros_like(b), 1e-10, 30, 100, minv=lu.solve)
    assert st == krylov.CONVERGED and it == 1 and rel <= 1e-10


def test_preconditioned_gmres_arnoldi_relation_and_gain():
    A, b = _nonsym(24)
    minv = krylov.jacobi_sweeps(A, 4, 0.8)
    rec = []
    x, it, rel, st = krylov.gmres(A, b, np.zeros_like(b), 1e-10, 30, 20000, record=rec, minv=minv)
    assert st == krylov.CONVERGED
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
    V, Hbar = rec[0]
    k = Hbar.shape[1]
    AMV = np.column_stack([A @ minv(V[:, c]) for c in range(k)])
    assert np.linalg.norm(AMV - V @ Hbar) <= 1e-12 * np.linalg.norm(AMV)
    _, it0, _, st0 = krylov.gmres(A, b, np.zeros_like(b), 1e-10, 30, 20000)
    assert st0 == krylov.CONVERGED and it < it0


def test_direct_solve_matches_dense_lu_and_refines():
    """The reference solver equals dense LU on a small nonsymmetric system
    (to kappa times rounding) and its refined residual sits at rounding level."""
    A, b = _system(workloads.plain_nonsym(18), 5)
    x_ref = np.linalg.solve(A.toarray(), b)
    x, rel = krylov.direct_solve(A, b)
    kappa = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - x_ref) <= 1e-15 * kappa * np.linalg.norm(x_ref)
    assert rel <= 1e-14 and rel == pytest.approx(
        np.linalg.norm(b - A @ x) / np.linalg.norm(b), rel=1e-12)
    x0, rel0 = krylov.direct_solve(A, b, refinements=0)
    assert rel <= rel0 + 1e-16


# ---- Chebyshev polynomial preconditioner ----

def _cheb_T(d, x):
    """T_d(x) from its trigonometric / hyperbolic closed form."""
    x = np.asarray(x, dtype=np.float64)
    inside = np.abs(x) <= 1
    out = np.empty_like(x)
    out[inside] = np.cos(d * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** d * np.cosh(d * np.arccosh(np.abs(xo)))
    return out


@pytest.mark.parametrize("degree,lo,hi", [(1, 0.2, 1.8), (2, 0.05, 2.0), (5, 0.1, 1.9), (8, 0.02, 2.0)])
def test_chebyshev_residual_polynomial_closed_form(degree, lo, hi):
    """On a diagonal operator (D^{-1} taken as the identity) the residual
    1 - lam p(lam) left by the recurrence equals T_d((theta - lam) / delta) /
    T_d(theta / delta) at every eigenvalue, inside and outside [lo, hi]."""
    lam = np.concatenate([np.linspace(lo, hi, 41), [0.5 * lo, 1.2 * hi]])
    A = scipy.sparse.diags(lam).tocsr()
    minv = krylov.chebyshev_sweeps(A, degree, lo, hi, dinv=np.ones(lam.size))
    u = np.random.default_rng(degree).standard_normal(lam.size)
    res = (u - A @ minv(u)) / u
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    want = _cheb_T(degree, (theta - lam) / delta) / _cheb_T(degree, np.array(theta / delta))
    assert np.all(np.abs(res - want) <= 1e-13 * np.maximum(1.0, np.abs(want)))


@pytest.mark.parametrize("degree", [2, 4, 8])
def test_chebyshev_is_the_minimax_polynomial_on_the_interval(degree):
    """max over [lo, hi] of |1 - lam p(lam)| equals 1 / T_d(theta / delta), reached
    with alternating signs at the d + 1 points theta - delta cos(j pi / d)
    (equioscillation, hence optimal among degree-d polynomials with p's
    residual equal to 1 at 0), and it beats the residual (1 - omega lam)^d of d
    damped Jacobi sweeps for every omega."""
    lo, hi = 0.05, 2.0
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    grid = np.linspace(lo, hi, 4001)
    A = scipy.sparse.diags(grid).tocsr()
    minv = krylov.chebyshev_sweeps(A, degree, lo, hi, dinv=np.ones(grid.size))
    u = np.ones(grid.size)
    res = u - A @ minv(u)
    bound = 1.0 / _cheb_T(degree, np.array(theta / delta))
    assert np.abs(res).max() == pytest.approx(bound, rel=1e-9)
    ext = theta - delta * np.cos(np.arange(degree + 1) * np.pi / degree)
    Ae = scipy.sparse.diags(ext).tocsr()
    me = krylov.chebyshev_sweeps(Ae, degree, lo, hi, dinv=np.ones(ext.size))
    re = 1.0 - Ae @ me(np.ones(ext.size))
    assert np.allclose(np.abs(re), bound, rtol=1e-9)
    assert np.all(np.sign(re[1:]) == -np.sign(re[:-1]))
    for omega in np.linspace(0.1, 1.9, 37):
        assert np.abs((1 - omega * grid) ** degree).max() > bound


def test_chebyshev_degree_one_is_scaled_jacobi():
    A, b = _system(workloads.plain_nonsym(12), 3)
    minv = krylov.chebyshev_sweeps(A, 1, 0.1, 1.9)
    assert np.allclose(minv(b), b / A.diagonal() / 1.0, rtol=1e-15)


def test_chebyshev_operator_equals_the_matrix_chebyshev_polynomial():
    """On a real system: I - M^{-1} A equals T_d(X) / T_d(sigma) with
    X = (theta I - D^{-1} A) / delta, T_d formed by the matrix recurrence
    T_{k+1} = 2 X T_k - T_{k-1} in dense algebra (not the recurrence the
    operator uses)."""
    A, _ = _system(workloads.plain_nonsym(9), 2)
    n = A.shape[0]
    lo, hi, d = 0.1, 1.9, 6
    minv = krylov.chebyshev_sweeps(A, d, lo, hi)
    MA = np.column_stack([minv(A[:, j].toarray().ravel()) for j in range(n)])
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    B = np.diag(1.0 / A.diagonal()) @ A.toarray()
    X = (theta * np.eye(n) - B) / delta
    T_prev, T_cur = np.eye(n), X.copy()
    for _ in range(d - 1):
        T_prev, T_cur = T_cur, 2 * X @ T_cur - T_prev
    want = T_cur / _cheb_T(d, np.array(theta / delta))
    assert np.abs((np.eye(n) - MA) - want).max() <= 1e-12


def test_gershgorin_bound():
    """The bound is the largest absolute row sum of D^{-1} A (dense algebra)
    and every eigenvalue of D^{-1} A lies within it."""
    A, _ = _system(workloads.plain_nonsym(15), 4)
    B = np.diag(1.0 / A.diagonal()) @ A.toarray()
    g = krylov.gershgorin_bound(A)
    assert g == pytest.approx(np.abs(B).sum(axis=1).max(), rel=1e-14)
    assert np.abs(np.linalg.eigvals(B)).max() <= g * (1 + 1e-12)


def test_mixed_refinement_accepts_a_chebyshev_preconditioner():
    A, b = _system(workloads.plain_nonsym(24), 3)
    A32 = A.astype(np.float32)
    lmax = krylov.gershgorin_bound(A32)
    pc = lambda M: krylov.chebyshev_sweeps(M, 6, lmax / 30, lmax)
    x, inner, nref, rel, st = krylov.mixed_refine(A, A32, b, np.zeros_like(b), 1e-10, "gmres", 30,
                                                  20000, precond=pc)
    assert st == krylov.CONVERGED and rel <= 1e-10
