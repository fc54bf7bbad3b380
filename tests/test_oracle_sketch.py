"""Pins of the oracle's sparse-sign sketch and sketched block (CPU only)."""
import os

import numpy as np
import pytest
import scipy.sparse

import workloads
from oracle import sketch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_kat.txt")


def _kat():
    seed, vals = None, []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("seed"):
                seed = int(line.split()[1])
            else:
                vals.append(int(line))
    return seed, vals


def test_splitmix64_known_answer_vectorised():
    seed, vals = _kat()
    out = sketch.splitmix64_outputs(seed, np.arange(1, len(vals) + 1, dtype=np.uint64))
    assert [int(v) for v in out] == vals


def test_splitmix64_known_answer_scalar_stream():
    seed, vals = _kat()
    assert workloads.splitmix64_stream(seed, len(vals)) == vals


@pytest.mark.parametrize("n,s,zeta,seed", [(1000, 40, 8, 1), (777, 80, 8, 0x5EEDBA5E),
                                           (300, 48, 8, 7), (50, 8, 8, 3), (64, 9, 3, 11)])
def test_columns_structure(n, s, zeta, seed):
    rows, signs = sketch.sparse_sign_columns(n, s, zeta, seed)
    assert rows.shape == (n, zeta) and signs.shape == (n, zeta)
    assert rows.min() >= 0 and rows.max() < s
    for j in range(n):
        assert len(set(rows[j].tolist())) == zeta
    assert set(np.unique(signs).tolist()) <= {-1, 1}
    S = sketch.sparse_sign_matrix(n, s, zeta, seed)
    assert S.nnz == n * zeta
    colnorm2 = np.asarray(S.multiply(S).sum(axis=0)).ravel()
    np.testing.assert_allclose(colnorm2, 1.0, rtol=4e-16 * zeta, atol=0)


def test_acceptance_rule_against_scalar_stream():
    """Column j uses outputs 256 j + c + 1 of one SplitMix64 stream; duplicates skipped."""
    n, s, zeta, seed = 6, 12, 8, 99
    stream = workloads.splitmix64_stream(seed, 256 * n)
    rows, signs = sketch.sparse_sign_columns(n, s, zeta, seed)
    for j in range(n):
        taken, sg = [], []
        for c in range(256):
            h = stream[256 * j + c]
            q = ((h >> 32) * s) >> 32
            if q not in taken:
                taken.append(q)
                sg.append(1 if (h & 1) == 0 else -1)
            if len(taken) == zeta:
                break
        assert rows[j].tolist() == taken
        assert signs[j].tolist() == sg


def test_rows_and_signs_uniform():
    n, s, zeta = 20000, 80, 8
    rows, signs = sketch.sparse_sign_columns(n, s, zeta, 2024)
    counts = np.bincount(rows.ravel(), minlength=s)
    expected = n * zeta / s
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    assert chi2 < 160.0            # 79 dof: mean 79, sd 12.6; 160 is > 6 sd
    frac = float(np.mean(signs == 1))
    assert abs(frac - 0.5) < 5.0 * 0.5 / np.sqrt(n * zeta)


def test_subspace_embedding():
    """For a random k-dim subspace U, the singular values of S U stay near 1."""
    n, s, zeta, k = 4096, 80, 8, 5
    S = sketch.sparse_sign_matrix(n, s, zeta, 5)
    U, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, k)))
    sv = np.linalg.svd(np.asarray(S @ U), compute_uv=False)
    assert sv.max() < 1.6 and sv.min() > 0.5
    # E[S^T S] = I: averaged over many random vectors ||S u||^2 / ||u||^2 -> 1.
    G = np.random.default_rng(1).standard_normal((n, 400))
    ratio = np.sum(np.asarray(S @ G) ** 2, axis=0) / np.sum(G ** 2, axis=0)
    assert abs(ratio.mean() - 1.0) < 0.05


def test_exhausted_candidates_fill_rule():
    """With s == zeta every column holds every row exactly once."""
    rows, _ = sketch.sparse_sign_columns(40, 8, 8, 123)
    for j in range(40):
        assert sorted(rows[j].tolist()) == list(range(8))


def test_sketch_block_brute_force():
    p = workloads.plain_nonsym(12)
    rowptr, colind, vals, b = workloads.csr_system(p, 3)
    n = p.n
    A = scipy.sparse.csr_matrix((vals, colind, rowptr), shape=(n, n))
    X = np.random.default_rng(3).standard_normal((n, 6))
    s, zeta = 40, 8
    rows, signs = sketch.sparse_sign_columns(n, s, zeta, 17)
    Sd = np.zeros((s, n))
    for j in range(n):
        for q, sg in zip(rows[j], signs[j]):
            Sd[q, j] = sg / np.sqrt(zeta)
    Ad = A.toarray()
    W_ref = Sd @ np.column_stack([Ad @ X, b])
    W = sketch.sketch_block(sketch.sparse_sign_matrix(n, s, zeta, 17), A, X, b)
    np.testing.assert_allclose(W, W_ref, rtol=1e-12, atol=1e-12 * np.abs(W_ref).max())
