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
