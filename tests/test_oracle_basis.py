"""Pins of oracle/basis.py (POD, Algorithm 2; randomised range finder, Algorithm 4)."""
import math

import numpy as np
import pytest
from scipy import stats

import workloads
from oracle import basis, krylov, method, sketch


def test_box_muller_closed_forms():
    u1 = np.array([1.0, math.exp(-0.5), math.exp(-0.5), math.exp(-2.0), math.exp(-4.5)])
    u2 = np.array([0.3, 0.0, 0.5, 0.25, 0.0])
    g = basis.box_muller(u1, u2)
    np.testing.assert_allclose(g, [0.0, 1.0, -1.0, 0.0, 3.0], atol=1e-15)


def test_gaussian_stream_moments_and_counter():
    N = 200_000
    g = basis.gaussians(0xBADC0DE, 0, N)
    assert abs(g.mean()) < 4.0 / math.sqrt(N)
    assert abs(g.var() - 1.0) < 4.0 * math.sqrt(2.0 / N)
    assert abs(stats.kurtosis(g, fisher=False) - 3.0) < 0.1
    assert stats.kstest(g, "norm").pvalue > 1e-3
    # counter-based: any window equals the slice of a longer stream
    assert np.array_equal(basis.gaussians(0xBADC0DE, 1234, 77), g[1234:1311])
    # a different seed gives a different stream
    assert not np.allclose(basis.gaussians(0xBADC0DF, 0, 16), g[:16])


def _columns(n, count, seed):
    """Smooth-in-time columns (a slowly rotating low-rank signal plus noise)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, 6))
    out = []
    for i in range(count):
        t = 0.05 * i
        coef = np.array([math.cos(t), math.sin(t), math.cos(2 * t), t, t * t, 1.0])
        out.append(B @ coef + 1e-3 * rng.standard_normal(n))
    return out


@pytest.mark.parametrize("M,m,refresh", [(8, 5, 1000), (6, 9, 1000), (10, 4, 7)])
def test_progressive_update_equals_from_scratch(M, m, refresh):
    """The progressive updates keep Omega = X Z for the current X and Z (exact in exact
    arithmetic), through the start-up, the full ring and refreshes."""
    cols = _columns(200, 40, 1)
    rrf = basis.RandRangeFinder(m, refresh, seed=11)
    hist = method.History(200, M)
    scratches = 0
    for i, c in enumerate(cols):
        X = hist.matrix()
        if X.shape[1]:
            before = rrf.counter
            om = rrf.basis(X)
            if rrf.updates == 0:
                scratches += 1
                assert rrf.counter == before + X.shape[1] * m
            Z = rrf.Zmat()
            assert Z.shape == (X.shape[1], m)
            assert np.linalg.norm(om - X @ Z) <= 1e-12 * np.linalg.norm(om)
        leaving = hist.cols[0] if len(hist.cols) == M else None
        rrf.on_push(c, leaving)
        hist.push(c)
    expected = 1 + (len(cols) - 2) // refresh if refresh < len(cols) else 1
    assert scratches == expected


def test_refresh_redraws_z():
    cols = _columns(100, 12, 2)
    rrf = basis.RandRangeFinder(3, 2, seed=5)
    hist = method.History(100, 4)
    hist.push(cols[0])
    rrf.basis(hist.matrix())
    Z0 = rrf.Zmat().copy()
    for c in cols[1:3]:
        rrf.on_push(c, hist.cols[0] if len(hist.cols) == 4 else None)
        hist.push(c)
    assert rrf.updates == 2
    om = rrf.basis(hist.matrix())
    assert rrf.updates == 0
    Z = rrf.Zmat()
    assert Z.shape == (3, 3) and not np.allclose(Z[0], Z0[0])
    np.testing.assert_allclose(om, hist.matrix() @ Z, rtol=0, atol=1e-13 * np.abs(om).max())


def _matrix_with_singular_values(n, sig, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, len(sig))))
    V, _ = np.linalg.qr(rng.standard_normal((len(sig), len(sig))))
    return U @ np.diag(sig) @ V.T


def test_randomised_svd_expected_error_bound():
    """E ||(I - Q Q^T) X||_F <= (1 + r/(p-1))^(1/2) (sum_{k>r} sigma_k^2)^(1/2)
    (Section 2.2), and no draw beats the POD error of the same size."""
    sig = 2.0 ** -np.arange(20)
    X = _matrix_with_singular_values(300, sig, 3)
    r, p = 6, 4
    m = r + p
    errs = []
    for seed in range(300):
        rrf = basis.RandRangeFinder(m, 50, seed=seed)
        Q = basis.orthonormal_basis(rrf.basis(X))
        errs.append(np.linalg.norm(X - Q @ (Q.T @ X)))
    bound = math.sqrt(1 + r / (p - 1)) * math.sqrt(np.sum(sig[r:] ** 2))
    assert np.mean(errs) <= bound
    pod = math.sqrt(np.sum(sig[m:] ** 2))
    assert min(errs) >= pod * (1 - 1e-9)


@pytest.mark.parametrize("m", [1, 4, 9])
def test_pod_optimality_identity(m):
    sig = np.array([3.0, 2.0, 1.5, 1.0, 0.5, 0.25, 0.1, 0.05, 0.01, 0.001])
    X = _matrix_with_singular_values(150, sig, 4)
    Q = basis.pod_basis(X, m)
    assert np.allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    err2 = np.linalg.norm(X - Q @ (Q.T @ X)) ** 2
    assert err2 == pytest.approx(np.sum(sig[m:] ** 2), rel=1e-10, abs=1e-24)
    rng = np.random.default_rng(m)
    for _ in range(50):
        R, _ = np.linalg.qr(rng.standard_normal((150, m)))
        assert np.linalg.norm(X - R @ (R.T @ X)) ** 2 >= err2 * (1 - 1e-12)
    # the leading singular vectors: Q spans the same space as U[:, :m]
    U, _, _ = np.linalg.svd(X, full_matrices=False)
    assert np.linalg.norm(Q @ (Q.T @ U[:, :m]) - U[:, :m]) < 1e-10


def _system(N=12, i=3):
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    return krylov.csr(rowptr, colind, vals, p.n), b, p.n


def test_full_span_limit():
    """m >= M_i: span(Omega) = span(X) = span(Q_POD), so both guesses equal the
    guess over the whole history."""
    A, b, n = _system()
    rng = np.random.default_rng(7)
    X = rng.standard_normal((n, 6))
    S = sketch.sparse_sign_matrix(n, 24, 8, 9)
    ref = method.sketched_guess(A, b, X, S)
    g_pod = basis.pod_guess(A, b, X, 6, S)
    rrf = basis.RandRangeFinder(8, 50, seed=1)
    g_rand = basis.rand_guess(A, b, rrf, X, S)
    for g in (g_pod, g_rand):
        assert np.linalg.norm(g.x0 - ref.x0) <= 1e-9 * np.linalg.norm(ref.x0)
        assert g.rho_s == pytest.approx(ref.rho_s, rel=1e-9)


def test_compressed_guess_residuals_are_ordered():
    """The minimiser over a subspace of span(X) is never better than over
    span(X) (sketched residuals), and the POD subspace of size m is a
    subspace of span(X)."""
    A, b, n = _system(16, 5)
    cols = _columns(n, 10, 8)
    X = np.stack(cols, axis=1)
    S = sketch.sparse_sign_matrix(n, 40, 8, 3)
    full = method.sketched_guess(A, b, X, S)
    for m in (2, 4, 8):
        g = basis.pod_guess(A, b, X, m, S)
        assert g.rho_s >= full.rho_s * (1 - 1e-9)
        rrf = basis.RandRangeFinder(m, 50, seed=m)
        g2 = basis.rand_guess(A, b, rrf, X, S)
        assert g2.rho_s >= full.rho_s * (1 - 1e-9)


def test_unsketched_limit_is_the_projection_of_algorithm_1():
    """With S = I the sketched guess over Q is Algorithm 1's exact minimiser."""
    A, b, n = _system(8, 2)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((n, 5))
    Q = basis.pod_basis(X, 3)
    g = method.sketched_guess(A, b, Q, np.eye(n))
    ref = method.projected_guess(A, b, Q)
    assert np.linalg.norm(g.x0 - ref.x0) <= 1e-12 * np.linalg.norm(ref.x0)
