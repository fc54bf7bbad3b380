"""The allocation-free sketched block (seq_sketch_block_noalloc) against the
regular path (seq_guess, which allocates its scratch at seq_create).

This entry point serves callers that cannot allocate device memory where they
need the sketch: work recorded into a CUDA graph by stream capture, host
callbacks and real-time loops that must not enter the allocator, and hosts
that fix the library's memory budget in advance.  Its scratch is a fixed
device array inside the library shared by all calls, so the test calls it
twice in a row and checks both results.  The file name makes pytest collect
it last.
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


@pytest.mark.parametrize("N,M,s,zeta,seed", [(40, 10, 40, 8, 123), (37, 20, 80, 8, 0x5EEDBA5E),
                                             (9, 31, 128, 16, 7)])
def test_noalloc_sketch_matches_regular_path(N, M, s, zeta, seed):
    import paper_2309_02156_gb300 as sa
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, 4)
    rng = np.random.default_rng(N + M)
    cols = [rng.standard_normal(p.n) for _ in range(M)]
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
    # Allocation-free path, twice in a row on the same output.
    X = torch.from_numpy(np.ascontiguousarray(np.stack(cols, axis=1))).to(DEV)
    W = torch.empty((s, M + 1), dtype=torch.float64, device=DEV)
    scale = np.linalg.norm(W_ref, axis=0)
    for _ in range(2):
        W.fill_(np.nan)
        sa.sketch_block_noalloc(A, X, bd, s, zeta, seed, W)
        got = W.cpu().numpy()
        assert np.all(np.abs(got - W_ref) <= 1e-11 * scale)


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
