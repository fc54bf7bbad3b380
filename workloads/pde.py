"""Time sequences of 5-point finite-difference systems A(t) x = b(t).

The operator on the unit square with zero Dirichlet data is

    A u = -div(k grad u) + v(t) . grad u + u,

    k(x, y, t) = 1 + a sin(2 pi (x + t) + phi) cos(2 pi y),
    v(t)       = v0 (cos t, sin t)            (v0 = 0: symmetric positive definite),

and the right-hand side is a Gaussian source circling the centre,

    b(t)_p = exp(-((x - 0.5 - rc cos t)^2 + (y - 0.5 - rc sin t)^2) / 0.02).

Both depend analytically on t, which is the setting of the paper's
Assumption 3 (Section 3).  Discretisation (a reading; the workload statement
fixes only "5-point FD of -div(k grad u)" and "first-order upwind"):

* interior nodes x_i = i h, y_j = j h, h = 1/(N+1), i, j = 1..N; unknown
  p = (j-1) N + (i-1) (x fastest);
* diffusion with k sampled at face midpoints, ((i +- 1/2) h, j h) and
  (i h, (j +- 1/2) h); the same expression gives the same face value for
  both neighbours, so the v0 = 0 matrix is exactly symmetric;
* advection by first-order upwinding: v_x >= 0 uses (u_p - u_W)/h, otherwise
  (u_E - u_p)/h, and likewise in y;
* neighbours outside the domain are dropped (zero Dirichlet);
* CSR rows hold their entries sorted by column: S, W, P, E, N.

So every matrix has nnz = 5 n - 4 N entries and the same sparsity pattern for
all t; only the values change.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


@dataclasses.dataclass(frozen=True)
class PDEParams:
    """One sequence of systems: grid side N and the analytic coefficients."""
    N: int
    a: float = 0.5          # amplitude of the k oscillation
    phi: float = 0.0        # phase inside the sine of k
    rc: float = 0.2         # radius of the source centre's circle
    v0: float = 0.0         # advection speed (0: SPD diffusion-reaction)
    dt: float = 0.01        # t_i = dt * i

    @property
    def n(self) -> int:
        return self.N * self.N

    @property
    def nnz(self) -> int:
        return 5 * self.N * self.N - 4 * self.N


def time_grid(p: PDEParams, i: int) -> float:
    """t_i = dt * i, counted from i = 0."""
    return p.dt * i


def _k(p: PDEParams, x, y, t):
    return 1.0 + p.a * np.sin(2.0 * math.pi * (x + t) + p.phi) * np.cos(2.0 * math.pi * y)


def pattern(N: int):
    """CSR row pointer and column indices of the 5-point pattern (int32)."""
    n = N * N
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")  # jj row (y), ii col (x)
    has_s = (jj > 0).ravel()
    has_w = (ii > 0).ravel()
    has_e = (ii < N - 1).ravel()
    has_n = (jj < N - 1).ravel()
    counts = 1 + has_s.astype(np.int64) + has_w + has_e + has_n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    p = np.arange(n, dtype=np.int64)
    cols = np.full((n, 5), -1, dtype=np.int64)
    cols[:, 0] = np.where(has_s, p - N, -1)
    cols[:, 1] = np.where(has_w, p - 1, -1)
    cols[:, 2] = p
    cols[:, 3] = np.where(has_e, p + 1, -1)
    cols[:, 4] = np.where(has_n, p + N, -1)
    mask = cols >= 0
    colind = cols[mask]
    return rowptr.astype(np.int32), colind.astype(np.int32), mask


def assemble(p: PDEParams, t: float, mask=None):
    """Values of A(t) in the CSR order of :func:`pattern` (float64, length nnz)."""
    N = p.N
    h = 1.0 / (N + 1)
    jj, ii = np.meshgrid(np.arange(1, N + 1, dtype=np.float64),
                         np.arange(1, N + 1, dtype=np.float64), indexing="ij")
    x = ii * h
    y = jj * h
    ke = _k(p, (ii + 0.5) * h, y, t)
    kw = _k(p, (ii - 0.5) * h, y, t)
    kn = _k(p, x, (jj + 0.5) * h, t)
    ks = _k(p, x, (jj - 0.5) * h, t)
    inv_h2 = 1.0 / (h * h)
    diag = (ke + kw + kn + ks) * inv_h2 + 1.0
    e_val = -ke * inv_h2
    w_val = -kw * inv_h2
    n_val = -kn * inv_h2
    s_val = -ks * inv_h2
    if p.v0 != 0.0:
        vx = p.v0 * math.cos(t)
        vy = p.v0 * math.sin(t)
        if vx >= 0.0:
            diag = diag + vx / h
            w_val = w_val - vx / h
        else:
            diag = diag - vx / h
            e_val = e_val + vx / h
        if vy >= 0.0:
            diag = diag + vy / h
            s_val = s_val - vy / h
        else:
            diag = diag - vy / h
            n_val = n_val + vy / h
    vals = np.stack([s_val.ravel(), w_val.ravel(), diag.ravel(),
                     e_val.ravel(), n_val.ravel()], axis=1)
    if mask is None:
        _, _, mask = pattern(N)
    return np.ascontiguousarray(vals[mask])


def rhs(p: PDEParams, t: float) -> np.ndarray:
    """b(t): Gaussian source of width^2 0.02 centred on a circle of radius rc."""
    N = p.N
    h = 1.0 / (N + 1)
    jj, ii = np.meshgrid(np.arange(1, N + 1, dtype=np.float64),
                         np.arange(1, N + 1, dtype=np.float64), indexing="ij")
    x = ii * h
    y = jj * h
    cx = 0.5 + p.rc * math.cos(t)
    cy = 0.5 + p.rc * math.sin(t)
    return np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / 0.02).ravel()


def csr_system(p: PDEParams, i: int):
    """(rowptr, colind, values, b) of system i of the sequence."""
    t = time_grid(p, i)
    rowptr, colind, mask = pattern(p.N)
    return rowptr, colind, assemble(p, t, mask), rhs(p, t)


def splitmix64_stream(seed: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 seeded with `seed`.

    Published generator of Steele, Lea and Flood (OOPSLA 2014): the state
    advances by the golden-ratio constant and each output is the state passed
    through the variant-13 64-bit finaliser.
    """
    out = []
    x = seed & _MASK
    for _ in range(count):
        x = (x + _GOLDEN) & _MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return out


def _unit(u: int) -> float:
    """Top 53 bits of a 64-bit draw as a double in [0, 1)."""
    return (u >> 11) * (1.0 / (1 << 53))


def batched_params(count: int, seed: int, nmin: int = 48, nmax: int = 384,
                   dt: float = 0.01) -> list[PDEParams]:
    """Independent SPD sequences: N ~ U{nmin..nmax}, phi ~ U[0, 2pi), rc ~ U[0.1, 0.3].

    Three SplitMix64 draws per sequence, in that order.
    """
    draws = splitmix64_stream(seed, 3 * count)
    out = []
    span = nmax - nmin + 1
    for s in range(count):
        uN, uphi, urc = draws[3 * s: 3 * s + 3]
        N = nmin + ((uN >> 32) * span >> 32)
        out.append(PDEParams(N=int(N), a=0.5, phi=2.0 * math.pi * _unit(uphi),
                             rc=0.1 + 0.2 * _unit(urc), v0=0.0, dt=dt))
    return out


def learned_amplitudes(count: int, seed: int, lo: float = 0.2, hi: float = 0.8) -> list[float]:
    """k amplitudes a ~ U[lo, hi] for the sequences of the learned workload."""
    return [lo + (hi - lo) * _unit(u) for u in splitmix64_stream(seed, count)]


# Named workloads.  Sizes and coefficients follow the five sequences the
# method is exercised on; dt is the time step of t_i = dt * i.
def plain_spd(N: int = 64) -> PDEParams:
    """SPD diffusion-reaction sequence (CG workload); N = 64 gives n = 4096."""
    return PDEParams(N=N, a=0.5, phi=0.0, rc=0.2, v0=0.0, dt=0.01)


def plain_nonsym(N: int = 1024) -> PDEParams:
    """Nonsymmetric advection-diffusion sequence, v = 20 (cos t, sin t) (GMRES workload)."""
    return PDEParams(N=N, a=0.5, phi=0.0, rc=0.2, v0=20.0, dt=0.005)
