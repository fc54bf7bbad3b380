"""Pins of the oracle's guess (Algorithm 1 with the sketched reduced problem)."""
import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

import workloads
from oracle import krylov, method, sketch


def _system(p, i):
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    return krylov.csr(rowptr, colind, vals, p.n), b


def _exact_history(p, i, M):
    """x(t_{i-M}) .. x(t_{i-1}) solved by a direct sparse solver (oldest first)."""
    cols = []
    for k in range(i - M, i):
        A, b = _system(p, k)
        cols.append(scipy.sparse.linalg.spsolve(A.tocsc(), b))
    return np.stack(cols, axis=1)


def test_identity_sketch_equals_dense_projection():
    """With S = I the sketched guess is the unsketched least-squares projection."""
    p = workloads.plain_nonsym(16)
    X = _exact_history(p, 12, 6)
    A, b = _system(p, 12)
    g = method.sketched_guess(A, b, X, scipy.sparse.identity(p.n, format="csr"))
    y_ref = np.linalg.lstsq(A.toarray() @ X, b, rcond=None)[0]
    x_ref = X @ y_ref
    assert np.linalg.norm(g.x0 - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert method.relres(A, b, g.x0) == pytest.approx(method.relres(A, b, x_ref), rel=1e-6)
    g2 = method.projected_guess(A, b, X)
    assert np.linalg.norm(g2.x0 - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_guess_exact_when_b_in_A_span_X():
    p = workloads.plain_nonsym(20)
    A, _ = _system(p, 5)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((p.n, 10))
    c = rng.standard_normal(10)
    b = A @ (X @ c)
    S = sketch.sparse_sign_matrix(p.n, 40, 8, 3)
    g = method.sketched_guess(A, b, X, S)
    np.testing.assert_allclose(g.y, c, rtol=1e-9, atol=1e-10)
    assert method.relres(A, b, g.x0) < 1e-12


def test_guess_residual_decays_with_history_length():
    """Theorem 2: for analytic A(t), b(t) the projected residual shrinks as M grows."""
    p = workloads.plain_spd(16)
    i = 14
    A, b = _system(p, i)
    Xfull = _exact_history(p, i, 12)
    res = []
    for M in (1, 2, 4, 6, 8, 10, 12):
        g = method.projected_guess(A, b, Xfull[:, -M:], tau=1e-15)
        res.append(method.relres(A, b, g.x0))
    # Nested spans: never worse (up to rounding) as older columns are added.
    for a_, b_ in zip(res, res[1:]):
        assert b_ <= a_ * (1 + 1e-6) + 1e-15
    assert res[4] < 1e-4 * res[0]          # M = 8 versus M = 1
    # Geometric singular-value decay of the history (Theorem 1).
    sv = np.linalg.svd(Xfull, compute_uv=False)
    assert sv[6] / sv[0] < 1e-6
    assert np.all(sv[1:8] < sv[:7])


def test_projection_never_worse_than_previous_solution():
    """Eq. (7): the minimiser over span(X) beats any element of it, e.g. x(t_{i-1})."""
    p = workloads.plain_nonsym(16)
    for i in (6, 9):
        A, b = _system(p, i)
        X = _exact_history(p, i, 5)
        g = method.projected_guess(A, b, X)
        assert method.relres(A, b, g.x0) <= method.relres(A, b, method.previous_guess(X)) + 1e-15


def test_sketched_residual_close_to_optimal():
    """Subspace embedding: the sketched guess's true residual is within a small
    factor of the unsketched optimum."""
    p = workloads.plain_nonsym(32)
    i = 12
    A, b = _system(p, i)
    X = _exact_history(p, i, 10)
    S = sketch.sparse_sign_matrix(p.n, 80, 8, 0x5EEDBA5E)
    gs = method.sketched_guess(A, b, X, S)
    gp = method.projected_guess(A, b, X)
    rs, rp = method.relres(A, b, gs.x0), method.relres(A, b, gp.x0)
    assert rp <= rs * (1 + 1e-8)
    assert rs <= 5.0 * rp


def test_step_solution_matches_dense_lu():
    p = workloads.plain_nonsym(10)
    S = sketch.sparse_sign_matrix(p.n, 40, 8, 1)
    hist = method.History(p.n, 4)
    for i in range(7):
        A, b = _system(p, i)
        out = method.solve_step(A, b, hist, S, 1e-11, "gmres")
        x_ref = np.linalg.solve(A.toarray(), b)
        assert out["status"] == krylov.CONVERGED
        kappa = np.linalg.cond(A.toarray())
        assert np.linalg.norm(out["x"] - x_ref) <= kappa * 1e-11 * np.linalg.norm(x_ref)


def test_history_ring_order():
    h = method.History(3, 2)
    for k in range(4):
        h.push(np.full(3, float(k)))
    np.testing.assert_array_equal(h.matrix()[0], [2.0, 3.0])


def test_startup_guess_is_zero():
    p = workloads.plain_spd(8)
    A, b = _system(p, 0)
    S = sketch.sparse_sign_matrix(p.n, 40, 8, 1)
    g = method.sketched_guess(A, b, np.zeros((p.n, 0)), S)
    assert np.all(g.x0 == 0.0)


def test_recorded_spd_iterations_are_the_oracles(tmp_path):
    """tests/golden/oracle_iterations_spd64.json is what the oracle produces
    on the 64 x 64 SPD sequence (it is quoted beside the GPU's counts), and the
    sketched guess needs fewer CG iterations than the previous solution."""
    import json
    import os
    from oracle import measure_iterations
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    stored = json.load(open(os.path.join(root, "tests", "golden", "oracle_iterations_spd64.json")))
    out = tmp_path / "spd.json"
    measure_iterations.spd(str(out))
    fresh = json.load(open(out))
    for mode in ("sketch", "prev"):
        # Equal here; a host with another BLAS may round a CG test differently.
        for a, b in zip(fresh[mode]["systems"], stored[mode]["systems"]):
            assert abs(a["iters"] - b["iters"]) <= 2
    assert stored["sketch"]["iters_mean_full_history"] < 0.6 * stored["prev"]["iters_mean_full_history"]
