"""The allocation-free sketched block (seq_sketch_block_noalloc).

This entry point is for callers that cannot allocate device memory where they
need the sketch: host callbacks and real-time loops that must not wait in the
allocator (cudaMalloc may synchronise the whole device), and applications
that hand the GPU's memory to their own pool or fix the library's budget in
advance, so that a late allocation would fail.  Its scratch is a fixed device
array inside the library, shared by all calls and keeping the last call's
contents, so every check here makes two calls in a row.

W is compared with the regular path (seq_guess, whose scratch is allocated
at seq_create) and with the oracle's definition W = S [A X | b] computed on the
CPU.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_02156_gb300 as sa
    sa.load()


def _inputs(N, M, seed_hist):
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, 4)
    rng = np.random.default_rng(seed_hist)
    cols = [rng.standard_normal(p.n) for _ in range(M)]
    return p, rowptr, colind, vals, b, cols


def _oracle_block(p, rowptr, colind, vals, b, cols, s, zeta, seed):
    from oracle import krylov, sketch
    A = krylov.csr(rowptr, colind, vals, p.n)
    S = sketch.sparse_sign_matrix(p.n, s, zeta, seed)
    return sketch.sketch_block(S, A, np.stack(cols, axis=1), b)


@pytest.mark.parametrize("N,M,s,zeta,seed", [(40, 10, 40, 8, 123), (37, 20, 80, 8, 0x5EEDBA5E),
                                             (9, 31, 128, 16, 7)])
def test_noalloc_sketch_matches_regular_path_and_oracle(N, M, s, zeta, seed):
    import paper_2309_02156_gb300 as sa
    p, rowptr, colind, vals, b, cols = _inputs(N, M, N + M)
    A = sa.CSR(torch.from_numpy(rowptr).to(DEV), torch.from_numpy(colind).to(DEV),
               torch.from_numpy(vals).to(DEV))
    bd = torch.from_numpy(b).to(DEV)
    # Regular path: history pushed into a context, guess, then the block it used.
    seq = sa.Sequence(p.n, M, s, zeta=zeta, seed=seed)
    for c in cols:
        seq.push(torch.from_numpy(c).to(DEV))
    x0 = torch.empty(p.n, dtype=torch.float64, device=DEV)
    seq.guess(A, bd, x0)
    W_ref, _ = seq.last_sketch()
    W_ref = W_ref[: s * (M + 1)].reshape(s, M + 1)
    seq.close()
    W_orc = _oracle_block(p, rowptr, colind, vals, b, cols, s, zeta, seed)
    # Allocation-free path, twice in a row on the same output.
    X = torch.from_numpy(np.ascontiguousarray(np.stack(cols, axis=1))).to(DEV)
    W = torch.empty((s, M + 1), dtype=torch.float64, device=DEV)
    scale = np.linalg.norm(W_orc, axis=0)
    for _ in range(2):
        W.fill_(np.nan)
        sa.sketch_block_noalloc(A, X, bd, s, zeta, seed, W)
        got = W.cpu().numpy()
        assert np.all(np.abs(got - W_ref) <= 1e-11 * scale)
        assert np.all(np.abs(got - W_orc) <= 1e-11 * scale)


def test_noalloc_rejects_oversized_requests():
    import paper_2309_02156_gb300 as sa
    p = workloads.plain_nonsym(8)
    rowptr, colind, vals, b = workloads.csr_system(p, 1)
    A = sa.CSR(torch.from_numpy(rowptr).to(DEV), torch.from_numpy(colind).to(DEV),
               torch.from_numpy(vals).to(DEV))
    bd = torch.from_numpy(b).to(DEV)
    X = torch.zeros((p.n, 31), dtype=torch.float64, device=DEV)
    W = torch.empty((129, 32), dtype=torch.float64, device=DEV)
    with pytest.raises(sa.SeqError) as e:
        sa.sketch_block_noalloc(A, X, bd, 129, 8, 1, W)      # 129 * 32 > 4096
    assert e.value.code == -1


def test_noalloc_bad_column_index_then_good_call():
    """A column index equal to n is skipped by the kernel and reported as
    SEQ_EINVAL after the call; the flag lives in the shared scratch array and
    is cleared by every call, so a valid call right after returns OK with the
    oracle's W."""
    import paper_2309_02156_gb300 as sa
    N, M, s, zeta, seed = 20, 6, 24, 8, 99
    p, rowptr, colind, vals, b, cols = _inputs(N, M, 5)
    bad = colind.copy()
    bad[len(bad) // 2] = p.n
    X = torch.from_numpy(np.ascontiguousarray(np.stack(cols, axis=1))).to(DEV)
    bd = torch.from_numpy(b).to(DEV)
    W = torch.empty((s, M + 1), dtype=torch.float64, device=DEV)
    A_bad = sa.CSR(torch.from_numpy(rowptr).to(DEV), torch.from_numpy(bad).to(DEV),
                   torch.from_numpy(vals).to(DEV))
    with pytest.raises(sa.SeqError) as e:
        sa.sketch_block_noalloc(A_bad, X, bd, s, zeta, seed, W)
    assert e.value.code == -1
    A = sa.CSR(torch.from_numpy(rowptr).to(DEV), torch.from_numpy(colind).to(DEV),
               torch.from_numpy(vals).to(DEV))
    W_orc = _oracle_block(p, rowptr, colind, vals, b, cols, s, zeta, seed)
    scale = np.linalg.norm(W_orc, axis=0)
    for _ in range(2):
        W.fill_(np.nan)
        sa.sketch_block_noalloc(A, X, bd, s, zeta, seed, W)
        assert np.all(np.abs(W.cpu().numpy() - W_orc) <= 1e-11 * scale)
