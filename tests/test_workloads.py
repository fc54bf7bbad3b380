"""Checks of the seeded input generator (CPU only)."""
import math

import numpy as np
import pytest

import workloads
from oracle import krylov


@pytest.mark.parametrize("N", [5, 16, 33])
def test_pattern_counts(N):
    rowptr, colind, _ = workloads.pattern(N)
    n = N * N
    assert rowptr[-1] == 5 * n - 4 * N == workloads.plain_spd(N).nnz
    for i in range(n):
        cols = colind[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_spd_matrix_is_exactly_symmetric():
    p = workloads.plain_spd(17)
    rowptr, colind, vals, _ = workloads.csr_system(p, 3)
    A = krylov.csr(rowptr, colind, vals, p.n)
    assert (A - A.T).count_nonzero() == 0
    assert np.linalg.eigvalsh(A.toarray()).min() > 0


def test_row_sums_on_constant_vector():
    """A 1 = 1 in the interior (diffusion and upwind advection annihilate constants)."""
    for p in (workloads.plain_spd(9), workloads.plain_nonsym(9)):
        rowptr, colind, vals, _ = workloads.csr_system(p, 2)
        A = krylov.csr(rowptr, colind, vals, p.n)
        s = (A @ np.ones(p.n)).reshape(p.N, p.N)
        np.testing.assert_allclose(s[1:-1, 1:-1], 1.0, rtol=0, atol=1e-9 * (p.N + 1) ** 2)


def test_rhs_peak_follows_the_circle():
    p = workloads.plain_spd(101)
    t = 0.7
    b = workloads.rhs(p, t).reshape(p.N, p.N)
    j, i = np.unravel_index(np.argmax(b), b.shape)
    h = 1.0 / (p.N + 1)
    assert abs((i + 1) * h - (0.5 + 0.2 * math.cos(t))) <= h
    assert abs((j + 1) * h - (0.5 + 0.2 * math.sin(t))) <= h


def test_batched_draws_in_range():
    ps = workloads.batched_params(512, 0x5EEDBA5E)
    Ns = [p.N for p in ps]
    assert min(Ns) >= 48 and max(Ns) <= 384
    assert all(0 <= p.phi < 2 * math.pi and 0.1 <= p.rc <= 0.3 for p in ps)
    assert 20e6 < sum(p.n for p in ps) < 40e6


# ---- the paper's test sequence (Section 4), workloads/e1.py ----------------

def _e1_apply(N, t, u_fn):
    from workloads import e1
    p = e1.E1Params(N=N)
    rowptr, colind = e1.pattern(N)
    vals = e1.assemble(p, t, rowptr, colind)
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    X, Y = np.meshgrid(i * h, i * h, indexing="xy")
    u = u_fn(X.ravel(), Y.ravel())
    import scipy.sparse as sp
    Au = sp.csr_matrix((vals, colind, rowptr), shape=(N * N, N * N)) @ u
    return Au, X.ravel(), Y.ravel(), h


def test_e1_pattern_counts():
    from workloads import e1
    for N in (5, 17, 100):
        rowptr, colind = e1.pattern(N)
        assert rowptr[-1] == 9 * N * N - 12 * N
        for r in (0, N + 1, N * N - 1):
            seg = colind[rowptr[r]:rowptr[r + 1]]
            assert np.all(np.diff(seg) > 0)


def test_e1_coefficient_gradient():
    from workloads import e1
    rng = np.random.default_rng(0)
    x, y, t = rng.random(50), rng.random(50), 2.3 + rng.random(50)
    a, ax, ay = e1.coef(x, y, t)
    d = 1e-6
    fx = (e1.coef(x + d, y, t)[0] - e1.coef(x - d, y, t)[0]) / (2 * d)
    fy = (e1.coef(x, y + d, t)[0] - e1.coef(x, y - d, t)[0]) / (2 * d)
    np.testing.assert_allclose(ax, fx, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(ay, fy, rtol=1e-7, atol=1e-9)


def test_e1_operator_is_fourth_order():
    """On a smooth u, A u approaches a (u_xx + u_yy) + a_x u_x + a_y u_y at
    O(h^4) at nodes whose stencil lies inside the grid."""
    from workloads import e1
    t = 2.35
    u = lambda x, y: np.sin(2 * np.pi * x) * np.cos(np.pi * y) + x ** 3 * y
    def exact(x, y):
        a, ax, ay = e1.coef(x, y, t)
        ux = 2 * np.pi * np.cos(2 * np.pi * x) * np.cos(np.pi * y) + 3 * x ** 2 * y
        uy = -np.pi * np.sin(2 * np.pi * x) * np.sin(np.pi * y) + x ** 3
        uxx = -4 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.cos(np.pi * y) + 6 * x * y
        uyy = -np.pi ** 2 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
        return a * (uxx + uyy) + ax * ux + ay * uy
    errs = []
    for N in (39, 79):
        Au, X, Y, h = _e1_apply(N, t, u)
        inner = (X > 2.5 * h) & (X < 1 - 2.5 * h) & (Y > 2.5 * h) & (Y < 1 - 2.5 * h)
        errs.append(np.abs(Au - exact(X, Y))[inner].max())
    ratio = errs[0] / errs[1]
    assert 13.0 < ratio < 18.0, ratio


def test_e1_discrete_solution_is_the_manufactured_f():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    from workloads import e1
    p = e1.E1Params(N=30, dt=1e-3)
    rowptr, colind, vals, b, f = e1.system(p, 7)
    A = sp.csr_matrix((vals, colind, rowptr), shape=(p.n, p.n))
    x = spl.spsolve(A.tocsc(), b)
    assert np.abs(x - f).max() <= 1e-11 * np.abs(f).max()
    assert e1.time(p, 7) == pytest.approx(2.307)
