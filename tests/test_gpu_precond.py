"""Right-preconditioned GMRES (damped Jacobi sweeps) on the GPU against the
oracle's krylov.gmres(minv=krylov.jacobi_sweeps(...)).

Tolerances: as for the unpreconditioned GMRES (both sides run the same
stopping test on the true residual; rounding moves the stopping iteration by a
few steps: iterations within max(2, 3%)); the mixed form within 50% of the
oracle's float32 emulation (the inner float32 solves amplify rounding
differences); every final true residual meets the tolerance, checked with the
oracle's FP64 product.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import krylov, method, sketch

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_02156_gb300 as sa
    sa.load()
    yield


def _sa():
    import paper_2309_02156_gb300 as sa
    return sa


def _t(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def _system(N, i):
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    A = _sa().CSR(_t(rowptr, torch.int32), _t(colind, torch.int32), _t(vals))
    return p, A, _t(b), krylov.csr(rowptr, colind, vals, p.n), b


@pytest.mark.parametrize("N,d,omega", [(32, 1, 0.8), (45, 4, 0.8), (40, 3, 1.0), (24, 8, 0.7)])
def test_preconditioned_gmres_matches_oracle(N, d, omega):
    p, A, bd, A_ref, b = _system(N, 4)
    minv = krylov.jacobi_sweeps(A_ref, d, omega)
    x_ref, it_ref, rel_ref, st_ref = krylov.gmres(A_ref, b, np.zeros(p.n), 1e-9, 30, 50000, minv=minv)
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=30, max_iters=50000,
                         precond_sweeps=d, precond_omega=omega)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, bd, 1e-9, x)
    assert info["status"] == 0 and st_ref == 0
    assert abs(info["iters"] - it_ref) <= max(2, 0.03 * it_ref)
    xh = x.cpu().numpy()
    assert method.relres(A_ref, b, xh) <= 1e-9 * (1 + 1e-9)
    assert info["final_relres"] == pytest.approx(method.relres(A_ref, b, xh), rel=1e-6)
    assert np.linalg.norm(xh - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    seq.close()


def test_preconditioning_cuts_iterations_and_profiles_its_kernels():
    p, A, bd, A_ref, b = _system(64, 2)
    its = {}
    for d in (0, 4):
        seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=30, max_iters=50000,
                             precond_sweeps=d)
        seq.set_profiling(True)
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        info = seq.solve(A, bd, 1e-10, x)
        assert info["status"] == 0
        assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-9)
        st = seq.kernel_stats()
        its[d] = info["iters"]
        assert st["spmv"]["launches"] == info["iters"]
        if d:
            # d - 1 sweep kernels per Arnoldi step (the first forms the scaled
            # start vector itself), plus the same per cycle update
            assert st["precond"]["launches"] >= (d - 1) * info["iters"]
        else:
            assert st["precond"]["launches"] == 0
        seq.close()
    assert its[4] < 0.6 * its[0]


def test_mixed_preconditioned_reaches_tolerance():
    p, A, bd, A_ref, b = _system(48, 3)
    A32 = A_ref.astype(np.float32)
    x_ref, it_ref, nref, rel, st = krylov.mixed_refine(A_ref, A32, b, np.zeros(p.n), 1e-10, "gmres",
                                                      30, 100000, precond=(4, 0.8))
    assert st == 0
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", precision="mixed_krylov", restart=30,
                         max_iters=100000, precond_sweeps=4)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, bd, 1e-10, x)
    assert info["status"] == 0
    assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-9)
    assert abs(info["iters"] - it_ref) <= 0.5 * it_ref + 10
    seq.close()


def test_preconditioned_sequence_with_sketched_guess():
    """20 systems: sketched guess + preconditioned GMRES through the C-ABI;
    every system converges (oracle SpMV check)."""
    p = workloads.plain_nonsym(40)
    seq = _sa().Sequence(p.n, 8, 40, krylov="gmres", precond_sweeps=4, max_iters=50000)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    for i in range(20):
        _, A, bd, A_ref, b = _system(40, i)
        seq.guess(A, bd, x)
        info = seq.solve(A, bd, 1e-9, x)
        assert info["status"] == 0
        assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-9 * (1 + 1e-9)
        seq.push(x)
    seq.close()


def test_preconditioner_config_checks():
    sa = _sa()
    for kw in ({"krylov": "cg", "precond_sweeps": 2}, {"precond_sweeps": 33},
               {"precond_sweeps": 2, "precond_omega": 2.0}, {"precond_sweeps": -1}):
        with pytest.raises(sa.SeqError):
            sa.Sequence(100, 4, 16, **kw)


@pytest.mark.parametrize("restart,d", [(1, 1), (5, 2), (30, 6)])
def test_preconditioned_gmres_on_wide_rows(restart, d):
    """The Section 4 fourth-order operator (rows of up to 9 entries: the SELL
    slices are wider than the unrolled width, so the sweeps take the general
    row loop), short restarts included."""
    from workloads import e1
    p = e1.E1Params(N=20, dt=1e-3)
    rowptr, colind, vals, b, _ = e1.system(p, 3)
    A_ref = krylov.csr(rowptr, colind, vals, p.n)
    minv = krylov.jacobi_sweeps(A_ref, d, 0.8)
    _, it_ref, _, st_ref = krylov.gmres(A_ref, b, np.zeros(p.n), 1e-9, restart, 200000, minv=minv)
    A = _sa().CSR(_t(rowptr, torch.int32), _t(colind, torch.int32), _t(vals))
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=restart, max_iters=200000,
                         precond_sweeps=d)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, _t(b), 1e-9, x)
    assert info["status"] == 0 and st_ref == 0
    assert abs(info["iters"] - it_ref) <= max(2, 0.03 * it_ref)
    assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-9 * (1 + 1e-9)
    seq.close()


def _irregular(N, i, far):
    """The N x N advection-diffusion matrix plus extra entries: every 7th row
    gets one more entry (so SELL slices differ in width) and, with far, a
    column more than 32767 away from its row.  The extra values are 1% of the
    row's diagonal, which keeps the matrix diagonally dominant."""
    import scipy.sparse as sp
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    A = krylov.csr(rowptr, colind, vals, p.n).tolil()
    d = A.diagonal()
    for r in range(0, p.n, 7):
        c = (r * 13 + 5) % p.n
        if far and r < p.n // 4:
            c = p.n - 1 - (r % 17)
        if c != r:
            A[r, c] = A[r, c] + 0.01 * d[r]
    A = sp.csr_matrix(A)
    A.sort_indices()
    return p, A, b


@pytest.mark.parametrize("N,far", [(40, False), (190, True)])
def test_preconditioned_gmres_on_irregular_rows(N, far):
    """Right-preconditioned GMRES on a matrix whose SELL slices have different
    widths (N = 40; with far, N = 190, n = 36,100, also columns more than 32767
    from their row) and rows longer than the unrolled SELL path handles (the
    products then take the plain loop).  Same parity as above."""
    p, A_ref, b = _irregular(N, 2, far)
    assert (np.abs(A_ref.tocoo().col - A_ref.tocoo().row).max() > 32767) == far
    minv = krylov.jacobi_sweeps(A_ref, 4, 0.8)
    x_ref, it_ref, rel_ref, st_ref = krylov.gmres(A_ref, b, np.zeros(p.n), 1e-9, 30, 50000, minv=minv)
    A = _sa().CSR(_t(A_ref.indptr.astype(np.int32), torch.int32),
                  _t(A_ref.indices.astype(np.int32), torch.int32), _t(A_ref.data))
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=30, max_iters=50000,
                         precond_sweeps=4)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, _t(b), 1e-9, x)
    assert info["status"] == 0 and st_ref == 0
    assert abs(info["iters"] - it_ref) <= max(2, 0.03 * it_ref)
    assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-9 * (1 + 1e-9)
    seq.close()


@pytest.mark.parametrize("kind", ["jacobi", "chebyshev"])
def test_preconditioned_gmres_without_a_sell_copy(kind):
    """One row holding 1,000 entries (0.1% of the diagonal each) pads its
    32-row slice so far that the SELL copy is not built: the products, the
    folded first sweep included, run on the CSR arrays.  Same parity as above
    against the oracle's preconditioner."""
    import scipy.sparse as sp
    p = workloads.plain_nonsym(40)
    rowptr, colind, vals, b = workloads.csr_system(p, 3)
    A = krylov.csr(rowptr, colind, vals, p.n).tolil()
    d = A.diagonal()
    r0 = 17
    for c in range(0, p.n, max(1, p.n // 1000))[:1000]:
        if c != r0:
            A[r0, c] = A[r0, c] + 0.01 * d[r0] / 10
    A_ref = sp.csr_matrix(A)
    A_ref.sort_indices()
    ns = (p.n + 31) // 32
    assert 32 * np.diff(A_ref.indptr).max() > 2 * A_ref.nnz + 64 * ns     # no SELL copy
    if kind == "jacobi":
        minv = krylov.jacobi_sweeps(A_ref, 4, 0.8)
    else:
        lmax = krylov.gershgorin_bound(A_ref)
        minv = krylov.chebyshev_sweeps(A_ref, 4, lmax / 30, lmax)
    x_ref, it_ref, rel_ref, st_ref = krylov.gmres(A_ref, b, np.zeros(p.n), 1e-9, 30, 50000, minv=minv)
    A = _sa().CSR(_t(A_ref.indptr.astype(np.int32), torch.int32),
                  _t(A_ref.indices.astype(np.int32), torch.int32), _t(A_ref.data))
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=30, max_iters=50000,
                         precond_sweeps=4, precond_kind=kind)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, _t(b), 1e-9, x)
    assert info["status"] == 0 and st_ref == 0
    assert abs(info["iters"] - it_ref) <= max(2, 0.03 * it_ref)
    assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-9 * (1 + 1e-9)
    seq.close()


@pytest.mark.parametrize("N,d,ratio,lfix", [(32, 2, 0.0, 0.0), (45, 4, 0.0, 0.0), (40, 8, 10.0, 0.0),
                                            (24, 6, 0.0, 1.9)])
def test_chebyshev_preconditioned_gmres_matches_oracle(N, d, ratio, lfix):
    """GMRES right-preconditioned by the Chebyshev polynomial of degree d on
    [lmax / ratio, lmax] of D^{-1} A (lmax: the Gershgorin bound, or fixed),
    against the oracle's chebyshev_sweeps on the same interval."""
    p, A, bd, A_ref, b = _system(N, 4)
    lmax = lfix if lfix > 0 else krylov.gershgorin_bound(A_ref)
    r = ratio if ratio > 0 else 30.0
    minv = krylov.chebyshev_sweeps(A_ref, d, lmax / r, lmax)
    x_ref, it_ref, rel_ref, st_ref = krylov.gmres(A_ref, b, np.zeros(p.n), 1e-9, 30, 50000, minv=minv)
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=30, max_iters=50000,
                         precond_sweeps=d, precond_kind="chebyshev", precond_ratio=ratio,
                         precond_lmax=lfix)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, bd, 1e-9, x)
    assert info["status"] == 0 and st_ref == 0
    assert abs(info["iters"] - it_ref) <= max(2, 0.03 * it_ref), (info["iters"], it_ref)
    assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-9 * (1 + 1e-9)
    seq.close()


def test_chebyshev_beats_jacobi_at_equal_degree():
    """Degree-8 Chebyshev on [lmax / 30, lmax] against 8 damped Jacobi sweeps
    (omega 0.8) on a 96 x 96 system: fewer GMRES iterations, both to 1e-9."""
    p, A, bd, A_ref, b = _system(96, 4)
    its = {}
    for kind in ("jacobi", "chebyshev"):
        seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", restart=30, max_iters=50000,
                             precond_sweeps=8, precond_kind=kind)
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        info = seq.solve(A, bd, 1e-9, x)
        assert info["status"] == 0
        assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-9 * (1 + 1e-9)
        its[kind] = info["iters"]
        seq.close()
    assert its["chebyshev"] < its["jacobi"], its


def test_mixed_chebyshev_reaches_tolerance():
    p, A, bd, A_ref, b = _system(48, 3)
    A32 = A_ref.astype(np.float32)
    lmax = krylov.gershgorin_bound(A32)
    pc = lambda M: krylov.chebyshev_sweeps(M, 6, lmax / 30, lmax)
    x_ref, it_ref, nref, rel, st = krylov.mixed_refine(A_ref, A32, b, np.zeros(p.n), 1e-10, "gmres",
                                                      30, 100000, precond=pc)
    assert st == 0
    seq = _sa().Sequence(p.n, 4, 16, krylov="gmres", precision="mixed_krylov", restart=30,
                         max_iters=100000, precond_sweeps=6, precond_kind="chebyshev")
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    info = seq.solve(A, bd, 1e-10, x)
    assert info["status"] == 0
    assert method.relres(A_ref, b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-9)
    assert info["iters"] <= 1.5 * it_ref + 10 and it_ref <= 1.5 * info["iters"] + 10
    seq.close()
