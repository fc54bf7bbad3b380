"""The paper's test sequence (Section 4): div(a(x, t) grad f(x, t)) = g(x, t)
on the unit square, discretised by centred fourth-order finite differences on a
uniform N x N interior grid, one system per time t_k = t0 + k dt.

    a(x, y, t) = exp(-(x - 0.5)^2 - (y - 0.5)^2) cos(t x) + 2.1,
    f(x, y, t) = sin(4 pi y t) sin(15 pi x t)
                 [1 + sin(15 pi x t) cos(3 pi y t) exp((x - 0.5)^2 + (y - 0.5)^2 - 0.25^2)].

Readings (the section names the scheme and the functions only):

* the operator is expanded as a (f_xx + f_yy) + a_x f_x + a_y f_y with a and
  its gradient evaluated exactly at the node, and each derivative taken by
  the centred five-point fourth-order formula:
      f_xx ~ (-f_{i-2} + 16 f_{i-1} - 30 f_i + 16 f_{i+1} - f_{i+2}) / (12 h^2),
      f_x  ~ ( f_{i-2} -  8 f_{i-1}            +  8 f_{i+1} - f_{i+2}) / (12 h);
  so every row has up to 9 entries (the 13-point cross without the diagonal
  corners -- a plus of width 2);
* nodes x_i = i h, i = 1..N, h = 1/(N+1); unknown p = (j-1) N + (i-1);
  stencil points outside the interior are dropped from A (their values are
  known data);
* right-hand side b(t) = A(t) f(t) with f sampled at the interior nodes, so the
  discrete solution is exactly the manufactured f at the nodes (the paper's
  g is the continuous operator applied to f; the two differ by the O(h^4)
  truncation error; the manufactured f is not zero on the sides x = 1 and
  y = 1, so the boundary data would have to come from f in any case).

Sizes of the paper's runs: N = 100 (n = 10,000), t0 = 2.3, 200 steps,
dt = 1e-5 (M = 20, m = 10) or dt = 1e-3 (M = 35, m = 20), GMRES to 1e-7.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_D2 = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0
_D1 = np.array([1.0, -8.0, 0.0, 8.0, -1.0]) / 12.0
_OFF = (-2, -1, 0, 1, 2)


@dataclasses.dataclass(frozen=True)
class E1Params:
    N: int = 100
    t0: float = 2.3
    dt: float = 1e-5

    @property
    def n(self) -> int:
        return self.N * self.N


def coef(x, y, t):
    """a, a_x, a_y at (x, y, t)."""
    e = np.exp(-(x - 0.5) ** 2 - (y - 0.5) ** 2)
    c, s = np.cos(t * x), np.sin(t * x)
    a = e * c + 2.1
    ax = e * (-2.0 * (x - 0.5) * c - t * s)
    ay = e * (-2.0 * (y - 0.5) * c)
    return a, ax, ay


def solution(x, y, t):
    """The manufactured f(x, y, t)."""
    g = np.exp((x - 0.5) ** 2 + (y - 0.5) ** 2 - 0.25 ** 2)
    s15 = np.sin(15 * math.pi * x * t)
    return np.sin(4 * math.pi * y * t) * s15 * (1.0 + s15 * np.cos(3 * math.pi * y * t) * g)


def _nodes(N):
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    X, Y = np.meshgrid(i * h, i * h, indexing="xy")     # row j (y), column i (x)
    return h, X.ravel(), Y.ravel()


def _coo(N, wx_of, wy_of):
    """Entries (rows, cols, values) of the cross stencil; wx_of(k) / wy_of(k)
    give the weight of offset _OFF[k] along x / y for every row."""
    n = N * N
    r = np.arange(n)
    i, j = r % N, r // N
    rows, cols, vals = [], [], []
    for k, d in enumerate(_OFF):
        mx = (i + d >= 0) & (i + d < N)
        rows.append(r[mx]); cols.append(r[mx] + d); vals.append(wx_of(k)[mx])
        my = (j + d >= 0) & (j + d < N)
        rows.append(r[my]); cols.append(r[my] + d * N); vals.append(wy_of(k)[my])
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def _csr(N, rows, cols, vals):
    import scipy.sparse as sp
    A = sp.coo_matrix((vals, (rows, cols)), shape=(N * N, N * N)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def pattern(N: int):
    """CSR rowptr, colind (int32, columns sorted) of the 9-entry cross stencil."""
    ones = np.ones(N * N)
    A = _csr(N, *_coo(N, lambda k: ones, lambda k: ones))
    return A.indptr.astype(np.int32), A.indices.astype(np.int32)


def assemble(p: E1Params, t: float, rowptr=None, colind=None) -> np.ndarray:
    """Values (FP64, in the CSR order of `pattern`) of A(t)."""
    N = p.N
    h, X, Y = _nodes(N)
    a, ax, ay = coef(X, Y, t)
    A = _csr(N, *_coo(N, lambda k: a * _D2[k] / h ** 2 + ax * _D1[k] / h,
                      lambda k: a * _D2[k] / h ** 2 + ay * _D1[k] / h))
    if rowptr is not None:
        assert np.array_equal(A.indptr, rowptr) and np.array_equal(A.indices, colind)
    return A.data.copy()


def time(p: E1Params, k: int) -> float:
    return p.t0 + p.dt * k


def system(p: E1Params, k: int, rowptr=None, colind=None):
    """(rowptr, colind, values, b, f) of system k: A(t_k), b = A f, f exact."""
    if rowptr is None:
        rowptr, colind = pattern(p.N)
    t = time(p, k)
    vals = assemble(p, t, rowptr, colind)
    _, X, Y = _nodes(p.N)
    f = solution(X, Y, t)
    import scipy.sparse as sp
    b = sp.csr_matrix((vals, colind, rowptr), shape=(p.n, p.n)) @ f
    return rowptr, colind, vals, b, f
