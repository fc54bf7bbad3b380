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
