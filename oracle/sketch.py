"""Sparse-sign row sketch S in R^{s x n} and the sketched block W = S [A X | b].

The paper compresses the history with a Gaussian *column* sketch (Section 2.2,
Algorithm 4).  The hot path built here instead sketches the *rows* of the
reduced least-squares problem of Algorithm 1: it solves
min_y || S (A X y - b) ||_2 with a sparse-sign S ("sketch-and-solve").  The
paper does not define S, so this module fixes it (a reading, stated once here
and implemented independently on the GPU side):

* column j of S has exactly ``zeta`` nonzeros in distinct rows;
* its candidates are outputs 256*j + c + 1 (c = 0, 1, ..., 255) of the
  SplitMix64 generator seeded with ``seed`` (Steele, Lea and Flood 2014), i.e.
  h = mix64(seed + (256 j + c + 1) * 0x9E3779B97F4A7C15 mod 2^64);
* candidate row  q = ((h >> 32) * s) >> 32   (Lemire's multiply-shift),
  candidate sign = +1 if bit 0 of h is 0, else -1;
* candidates are taken in order of c; a row already taken is skipped;
* if 256 candidates do not give zeta distinct rows, the remaining entries take
  the smallest unused rows, in increasing order, with sign +1;
* each nonzero equals sign / sqrt(zeta).

Parity: pinned (published SplitMix64 known-answer values, structural counts,
sign/row uniformity, unit column norms, dense brute force for W).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
CANDIDATES = 256


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser applied elementwise to uint64 states."""
    with np.errstate(over="ignore"):
        z = z.astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64_outputs(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output number k (k >= 1) of SplitMix64(seed) for every k in `counters`."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + counters.astype(np.uint64) * _GAMMA
    return mix64(state)


def sparse_sign_columns(n: int, s: int, zeta: int, seed: int):
    """Rows (int32, n x zeta) and signs (int8, n x zeta) of every column of S.

    Entries of a column are listed in the order they were accepted.
    """
    if not (1 <= zeta <= s):
        raise ValueError("need 1 <= zeta <= s")
    j = np.arange(n, dtype=np.uint64)
    rows = np.full((n, zeta), -1, dtype=np.int64)
    signs = np.zeros((n, zeta), dtype=np.int8)
    count = np.zeros(n, dtype=np.int64)
    for c in range(CANDIDATES):
        if np.all(count == zeta):
            break
        h = splitmix64_outputs(seed, j * np.uint64(CANDIDATES) + np.uint64(c + 1))
        q = ((h >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)
        q = q.astype(np.int64)
        sg = np.where((h & np.uint64(1)) == 0, 1, -1).astype(np.int8)
        dup = np.any(rows == q[:, None], axis=1)
        take = (count < zeta) & ~dup
        idx = np.nonzero(take)[0]
        rows[idx, count[idx]] = q[idx]
        signs[idx, count[idx]] = sg[idx]
        count[idx] += 1
    for col in np.nonzero(count < zeta)[0]:          # exhausted candidates
        free = [q for q in range(s) if q not in set(rows[col, :count[col]].tolist())]
        while count[col] < zeta:
            rows[col, count[col]] = free.pop(0)
            signs[col, count[col]] = 1
            count[col] += 1
    return rows.astype(np.int32), signs


def sparse_sign_matrix(n: int, s: int, zeta: int, seed: int) -> scipy.sparse.csr_matrix:
    """S as an s x n sparse matrix with entries +-1/sqrt(zeta)."""
    rows, signs = sparse_sign_columns(n, s, zeta, seed)
    cols = np.repeat(np.arange(n), zeta)
    vals = signs.ravel().astype(np.float64) / np.sqrt(float(zeta))
    return scipy.sparse.csr_matrix((vals, (rows.ravel(), cols)), shape=(s, n))


def sketch_block(S: scipy.sparse.spmatrix, A: scipy.sparse.spmatrix,
                 X: np.ndarray, b: np.ndarray) -> np.ndarray:
    """W = S [A X | b]  (s x (m+1)), columns of X first, b last."""
    Y = np.column_stack([A @ X, b]) if X.shape[1] else b[:, None]
    return np.asarray(S @ Y)
