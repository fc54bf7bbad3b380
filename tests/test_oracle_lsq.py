"""Pins of the oracle's pivoted Householder least squares (CPU only)."""
import numpy as np
import pytest

from oracle import lsq


@pytest.mark.parametrize("s,m,seed", [(40, 10, 0), (80, 20, 1), (48, 12, 2), (21, 20, 3)])
def test_matches_lapack_full_rank(s, m, seed):
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((s, m)) * np.logspace(0, 3, m)     # uneven column scales
    wb = rng.standard_normal(s)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(W1, wb, 1e-12)
    y_ref = np.linalg.lstsq(W1, wb, rcond=None)[0]
    assert rank == m
    np.testing.assert_allclose(y, y_ref, rtol=1e-10, atol=1e-12 * np.abs(y_ref).max())
    assert rho == pytest.approx(np.linalg.norm(W1 @ y_ref - wb), rel=1e-12)


def test_single_column_closed_form():
    rng = np.random.default_rng(4)
    w1 = rng.standard_normal(40)
    wb = rng.standard_normal(40)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(w1[:, None], wb, 1e-12)
    assert rank == 1
    assert y[0] == pytest.approx(np.dot(w1, wb) / np.dot(w1, w1), rel=1e-14)


def test_consistent_rhs_is_exact():
    rng = np.random.default_rng(5)
    W1 = rng.standard_normal((80, 20))
    c = rng.standard_normal(20)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(W1, W1 @ c, 1e-12)
    np.testing.assert_allclose(y, c, rtol=1e-12, atol=1e-13)
    assert rho < 1e-13 * np.linalg.norm(W1 @ c)


def test_normal_equations_hold():
    rng = np.random.default_rng(6)
    W1 = rng.standard_normal((80, 20)) @ np.diag(np.logspace(0, -6, 20))
    wb = rng.standard_normal(80)
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(W1, wb, 1e-12)
    r = W1 @ y - wb
    # W1^T r = 0 up to rounding, measured column by column.
    rel = np.abs(W1.T @ r) / (np.linalg.norm(W1, axis=0) * np.linalg.norm(r))
    assert rel.max() < 1e-10


def test_rank_deficient_duplicate_column():
    rng = np.random.default_rng(7)
    W1 = rng.standard_normal((40, 6))
    W1[:, 4] = W1[:, 1]                              # exact duplicate
    wb = rng.standard_normal(40)
    y, rank, rho, perm, rdiag = lsq.pivoted_qr_lstsq(W1, wb, 1e-12)
    assert rank == 5
    assert y[1] == 0.0 or y[4] == 0.0
    best = np.linalg.norm(W1 @ np.linalg.lstsq(W1, wb, rcond=None)[0] - wb)
    assert rho == pytest.approx(best, rel=1e-12)


def test_zero_column_gets_zero_coefficient():
    rng = np.random.default_rng(8)
    W1 = rng.standard_normal((30, 5))
    W1[:, 2] = 0.0
    wb = rng.standard_normal(30)
    y, rank, rho, perm, _ = lsq.pivoted_qr_lstsq(W1, wb, 1e-12)
    assert rank == 4 and y[2] == 0.0
    keep = [0, 1, 3, 4]
    y_ref = np.linalg.lstsq(W1[:, keep], wb, rcond=None)[0]
    np.testing.assert_allclose(y[keep], y_ref, rtol=1e-11)


def test_pivoting_order_and_truncation():
    """After scaling, |R_kk| is non-increasing; tiny directions are truncated."""
    rng = np.random.default_rng(9)
    U, _ = np.linalg.qr(rng.standard_normal((80, 8)))
    Vt, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    W1 = U @ np.diag([1, 1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-14, 1e-15]) @ Vt
    wb = rng.standard_normal(80)
    y, rank, rho, perm, rdiag = lsq.pivoted_qr_lstsq(W1, wb, 1e-12)
    assert np.all(np.abs(rdiag[1:]) <= np.abs(rdiag[:-1]) * (1 + 1e-12))
    assert rank == 6
    # The residual equals the projection onto the kept 6-dim range, to rounding.
    Q6 = U[:, :6]
    best6 = np.linalg.norm(wb - Q6 @ (Q6.T @ wb))
    assert rho == pytest.approx(best6, rel=1e-6)


def test_empty_problem():
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(np.zeros((10, 0)), np.ones(10), 1e-12)
    assert y.shape == (0,) and rank == 0 and rho == pytest.approx(np.sqrt(10))


def test_reflector_sign_convention_and_near_axis_column():
    """alpha = -sign(x_0) ||x||: R_kk has the sign opposite to the pivot column's
    leading entry, which avoids cancellation for columns close to e_1."""
    W1 = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    _, _, _, _, rdiag = lsq.pivoted_qr_lstsq(W1, np.ones(3), 1e-12)
    assert rdiag[0] == -1.0 and rdiag[1] == -1.0
    W1 = np.array([[-3.0], [0.0]])
    _, _, _, _, rdiag = lsq.pivoted_qr_lstsq(W1, np.ones(2), 1e-12)
    assert rdiag[0] == 1.0
    W1 = np.array([[1.0, 0.3], [1e-9, 1.0], [0.0, 2.0], [3e-10, 0.5]])
    c = np.array([0.7, -1.1])
    y, rank, rho, _, _ = lsq.pivoted_qr_lstsq(W1, W1 @ c, 1e-12)
    np.testing.assert_allclose(y, c, rtol=1e-14)
