"""Record exact (direct-solve) solutions of the first systems of a sequence,
as sampled entries, so that the error of an iterative solution against the
exact one can be stated per result.

Test infrastructure: runs entirely in the oracle (krylov.direct_solve: sparse
LU plus FP64 iterative refinement) and writes JSON.  Default workload: the
2048 x 2048 advection-diffusion sequence (n = 4,194,304, v = 20 (cos t, sin t),
dt = 0.005), systems 0..4.  For each system it stores the solution's 2-norm,
its sum, the relative residual of the direct solve, and the solution at
`samples` seeded indices (numpy PCG64, seed 0x5EEDBA5E + i, without
replacement, sorted).  An error estimate from the samples is
    err = sqrt(n / k * sum_idx (x - x_ref)^2) / ||x_ref||.

    python -m oracle.reference_solutions --N 2048 --steps 5 \
        --out tests/golden/reference_solutions_nonsym2048.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import krylov  # noqa: E402

SAMPLE_SEED = 0x5EEDBA5E


def sample_indices(n: int, k: int, i: int) -> np.ndarray:
    """The k sampled unknowns of system i (sorted, distinct)."""
    rng = np.random.default_rng(SAMPLE_SEED + i)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--samples", type=int, default=1024)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    p = workloads.plain_nonsym(a.N)
    doc = {"workload": f"nonsym {a.N}x{a.N} (n={p.n}), v=20(cos t, sin t), dt={p.dt}, "
                       f"systems 0..{a.steps - 1}",
           "solver": "oracle.krylov.direct_solve (SuperLU, COLAMD, 2 FP64 refinements)",
           "sample_seed": SAMPLE_SEED, "host": platform.machine(), "systems": []}
    for i in range(a.steps):
        t0 = time.perf_counter()
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        A = krylov.csr(rowptr, colind, vals, p.n)
        x, rel = krylov.direct_solve(A, b)
        idx = sample_indices(p.n, a.samples, i)
        doc["systems"].append({
            "i": i, "relres": rel, "norm2": math.sqrt(float(np.dot(x, x))),
            "sum": float(np.sum(x)), "idx": idx.tolist(), "x": [float(v) for v in x[idx]],
            "seconds": time.perf_counter() - t0})
        print(json.dumps({"i": i, "relres": rel, "seconds": doc["systems"][-1]["seconds"]}),
              flush=True)
        with open(a.out, "w") as f:
            json.dump(doc, f)


if __name__ == "__main__":
    main()
