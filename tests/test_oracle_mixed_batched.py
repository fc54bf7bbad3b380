"""Pins of the oracle's mixed-precision guess and step and of its batched step.

The mixed guess is checked against the FP64 guess (itself pinned) within the
float32 rounding-error bound of the two sparse products, and against the
exact-span case; the mixed and batched steps against dense LU solutions,
residuals formed independently with dense matrices, the startup and
exact-span special cases, and independence of the sequences in a batch.
"""
import numpy as np
import pytest

import workloads
from oracle import krylov, method, sketch

U32 = 2.0 ** -24                     # unit roundoff of float32


def _gamma(k):
    return k * U32 / (1.0 - k * U32)


def _system(p, i):
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    return krylov.csr(rowptr, colind, vals, p.n), b


def _max_row_nnz(M):
    M = M.tocsr()
    return int(np.diff(M.indptr).max())


def test_mixed_sketch_block_within_float32_rounding_bound():
    """W = S [A X | b] formed in float32 differs from the same product formed in
    FP64 from the same float32 values by at most gamma_{k1+k2} |S| [|A||X| | |b|]
    entrywise (k1, k2 the longest rows of A and S)."""
    p = workloads.plain_nonsym(24)
    A, b = _system(p, 7)
    A32 = A.astype(np.float32)
    rng = np.random.default_rng(11)
    X32 = rng.standard_normal((p.n, 6)).astype(np.float32)
    S = sketch.sparse_sign_matrix(p.n, 48, 8, 5)
    S32 = S.astype(np.float32)
    g32 = method.sketched_guess_mixed(A32, b, X32, S)
    # The FP64 oracle on the float32-exact operands.
    g64 = method.sketched_guess(A32.astype(np.float64), b.astype(np.float32).astype(np.float64),
                                X32.astype(np.float64), S32.astype(np.float64))
    absS = abs(S32.astype(np.float64))
    absA = abs(A32.astype(np.float64))
    mag = np.column_stack([absS @ (absA @ np.abs(X32.astype(np.float64))),
                           absS @ np.abs(b.astype(np.float32).astype(np.float64))])
    bound = _gamma(_max_row_nnz(A) + _max_row_nnz(S32) + 2) * mag
    err = np.abs(g32.W - g64.W)
    assert np.all(err <= bound)
    # The bound is not vacuous: the float32 block does differ from FP64.
    assert err.max() > 0
    assert err.max() < 1e-5 * np.abs(g64.W).max()


def test_mixed_guess_recovers_exact_span_coefficients():
    """b = A X c exactly (X, A float32-exact): y = c up to kappa(W1) times the
    float32 rounding of W, and x0 = X c to the same order."""
    p = workloads.plain_nonsym(20)
    A, _ = _system(p, 3)
    A32 = A.astype(np.float32)
    rng = np.random.default_rng(4)
    X32 = rng.standard_normal((p.n, 8)).astype(np.float32)
    c = rng.standard_normal(8)
    A64, X64 = A32.astype(np.float64), X32.astype(np.float64)
    b = A64 @ (X64 @ c)
    S = sketch.sparse_sign_matrix(p.n, 40, 8, 9)
    g = method.sketched_guess_mixed(A32, b, X32, S)
    kappa = np.linalg.cond(g.W[:, :8])
    eps = 10.0 * kappa * _gamma(_max_row_nnz(A) + _max_row_nnz(S) + 2)
    assert np.linalg.norm(g.y - c) <= eps * np.linalg.norm(c)
    assert np.linalg.norm(g.x0 - X64 @ c) <= eps * np.linalg.norm(X64 @ c)
    assert g.rank == 8


def test_mixed_guess_startup_is_zero():
    p = workloads.plain_spd(8)
    A, b = _system(p, 0)
    S = sketch.sparse_sign_matrix(p.n, 32, 8, 1)
    g = method.sketched_guess_mixed(A.astype(np.float32), b, np.zeros((p.n, 0), np.float32), S)
    assert np.all(g.x0 == 0.0) and g.rank == 0
    assert g.rho_s == pytest.approx(np.linalg.norm(S @ b), rel=1e-15)


@pytest.mark.parametrize("kind,maker", [("gmres", workloads.plain_nonsym), ("cg", workloads.plain_spd)])
def test_mixed_step_matches_dense_lu(kind, maker):
    """Every step of a short sequence: the FP64 residual (dense) meets the
    tolerance, the solution is within kappa tol of dense LU, and the history
    receives the float32 rounding of the solution."""
    p = maker(10)
    S = sketch.sparse_sign_matrix(p.n, 32, 8, 2)
    hist = method.History(p.n, 4)
    tol = 1e-10
    for i in range(6):
        A, b = _system(p, i)
        Ad = A.toarray()
        out = method.solve_step_mixed(A, A.astype(np.float32), b, hist, S, tol, kind)
        assert out["status"] == krylov.CONVERGED
        x = out["x"]
        rd = np.linalg.norm(b - Ad @ x) / np.linalg.norm(b)
        assert rd <= tol * (1 + 1e-9)
        assert out["relres"] == pytest.approx(rd, rel=1e-6)
        x_ref = np.linalg.solve(Ad, b)
        assert np.linalg.norm(x - x_ref) <= np.linalg.cond(Ad) * tol * np.linalg.norm(x_ref)
        np.testing.assert_array_equal(hist.matrix()[:, -1], x.astype(np.float32).astype(np.float64))
        if i == 0:
            assert out["refinements"] >= 1 and np.all(out["x0"] == 0.0)


def _batch(Ns, i):
    ps = [workloads.plain_spd(N) for N in Ns]
    return ps, [_system(p, i) for p in ps]


def test_batched_step_solutions_match_dense_lu():
    """Uneven sizes, several steps: each sequence's solution is within kappa tol
    of dense LU, its reported residual is the dense one, and its history
    receives that solution."""
    Ns = (8, 11, 6)
    tol = 1e-8
    ps, _ = _batch(Ns, 0)
    hists = [method.History(p.n, 3) for p in ps]
    sks = [sketch.sparse_sign_matrix(p.n, 24, 4, 100 + k) for k, p in enumerate(ps)]
    for i in range(5):
        _, systems = _batch(Ns, i)
        outs = method.batched_step(systems, hists, sks, tol)
        for (A, b), h, o in zip(systems, hists, outs):
            Ad = A.toarray()
            assert o["status"] == krylov.CONVERGED
            rd = np.linalg.norm(b - Ad @ o["x"]) / np.linalg.norm(b)
            assert rd <= tol * (1 + 1e-9)
            assert o["relres"] == pytest.approx(rd, rel=1e-6)
            x_ref = np.linalg.solve(Ad, b)
            assert np.linalg.norm(o["x"] - x_ref) <= np.linalg.cond(Ad) * tol * np.linalg.norm(x_ref)
            np.testing.assert_array_equal(h.matrix()[:, -1], o["x"])
            if i == 0:
                assert np.all(o["x0"] == 0.0) and o["guess_relres"] == 1.0
            else:
                assert o["guess_relres"] < 1.0


def test_batched_step_sequences_are_independent():
    """Reversing the batch reverses the results bit for bit."""
    Ns = (7, 9, 5, 8)
    ps, _ = _batch(Ns, 0)

    def run(order):
        hists = [method.History(ps[k].n, 3) for k in order]
        sks = [sketch.sparse_sign_matrix(ps[k].n, 24, 4, 7 + k) for k in order]
        res = None
        for i in range(4):
            _, systems = _batch(Ns, i)
            res = method.batched_step([systems[k] for k in order], hists, sks, 1e-9)
        return res

    fwd = run([0, 1, 2, 3])
    rev = run([3, 2, 1, 0])
    for a, b_ in zip(fwd, reversed(rev)):
        np.testing.assert_array_equal(a["x"], b_["x"])
        assert a["iters"] == b_["iters"] and a["refinements"] == b_["refinements"]


def test_batched_step_exact_span_needs_no_iteration():
    """b in A span(X): the guess meets the tolerance and the solve does no
    iteration and no refinement (the early exit)."""
    p = workloads.plain_spd(9)
    A, _ = _system(p, 2)
    rng = np.random.default_rng(3)
    h = method.History(p.n, 4)
    X = rng.standard_normal((p.n, 4))
    for k in range(4):
        h.push(X[:, k])
    c = rng.standard_normal(4)
    b = A @ (X @ c)
    S = sketch.sparse_sign_matrix(p.n, 24, 4, 5)
    (o,) = method.batched_step([(A, b)], [h], [S], 1e-8)
    assert o["guess_relres"] < 1e-12
    assert o["iters"] == 0 and o["refinements"] == 0
    assert np.linalg.norm(o["x"] - X @ c) <= 1e-10 * np.linalg.norm(X @ c)
