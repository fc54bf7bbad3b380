"""Record the oracle's own Krylov iteration counts on a sequence.

Test infrastructure: runs entirely in the oracle and writes JSON.

--workload nonsym (default): Algorithm 1 with the sketched reduced problem
followed by GMRES(30) to a relative residual of 1e-8 on the 1024 x 1024
advection-diffusion sequence (M = 20, s = 80, zeta = 8, seed 0x5EEDBA5E);
per-system iteration counts and timings.  The CPU baseline of the benchmark
uses the mean count of the systems with a full history to turn a timed
sample (one guess plus a bounded number of GMRES iterations) into systems
per second.

--workload spd: the 64 x 64 SPD sequence (n = 4096, M = 10, s = 40, CG to
1e-10, 60 systems), once with the sketched guess and once with the previous
solution (the paper's baseline), each in its own sequence; the benchmark
quotes the means over the systems with a full history beside its own.

--workload spread: GMRES(30) from x0 = 0 on system 0 of the 1024 x 1024
sequence to 1e-8, with b multiplied entrywise by 1 + 1e-15 g (g seeded
standard normal, one seed per trial): how far the iteration count of
restarted GMRES moves under a rounding-level change of its input.

    python -m oracle.measure_iterations --steps 26 --out tests/golden/oracle_iterations_nonsym1024.json
    python -m oracle.measure_iterations --workload spd --out tests/golden/oracle_iterations_spd64.json
    python -m oracle.measure_iterations --workload spread --trial 1 --out spread_1.json  (trials 1..3)
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import krylov, method, sketch  # noqa: E402


def spd(out_path: str, N: int = 64, M: int = 10, s: int = 40, steps: int = 60,
        tol: float = 1e-10) -> None:
    p = workloads.plain_spd(N)
    S = sketch.sparse_sign_matrix(p.n, s, 8, 0x5EEDBA5E)
    doc = {"workload": f"SPD {N}x{N} (n={p.n}), M={M}, s={s}, zeta=8, seed 0x5EEDBA5E, "
                       f"CG to {tol:g}, {steps} systems",
           "host": platform.machine()}
    for mode in ("sketch", "prev"):
        hist = method.History(p.n, M)
        rows = []
        for i in range(steps):
            rowptr, colind, vals, b = workloads.csr_system(p, i)
            A = krylov.csr(rowptr, colind, vals, p.n)
            out = method.solve_step(A, b, hist, S, tol, "cg", guess=mode, max_iters=100000)
            assert out["status"] == krylov.CONVERGED
            rows.append({"i": i, "iters": int(out["iters"]), "guess_relres": out["guess_relres"],
                         "relres": out["relres"]})
        full = [r["iters"] for r in rows if r["i"] >= M]
        doc[mode] = {"systems": rows, "iters_mean_full_history": float(np.mean(full))}
        print(mode, doc[mode]["iters_mean_full_history"], flush=True)
    with open(out_path, "w") as f:
        json.dump(doc, f, indent=1)


def spread(out_path: str, trial: int, N: int = 1024) -> None:
    p = workloads.plain_nonsym(N)
    rowptr, colind, vals, b = workloads.csr_system(p, 0)
    A = krylov.csr(rowptr, colind, vals, p.n)
    g = np.random.default_rng(trial).standard_normal(p.n)
    bb = b * (1 + 1e-15 * g) if trial else b
    t0 = time.perf_counter()
    _, it, rel, st = krylov.gmres(A, bb, np.zeros(p.n), 1e-8, 30, 60000)
    doc = {"workload": f"nonsym {N}x{N} system 0, GMRES(30) from 0 to 1e-8, b (1 + 1e-15 g)",
           "trial": trial, "iters": int(it), "relres": rel, "status": int(st),
           "seconds": time.perf_counter() - t0, "host": platform.machine()}
    print(json.dumps(doc), flush=True)
    with open(out_path, "w") as f:
        json.dump(doc, f, indent=1)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=("nonsym", "spd", "spread"), default="nonsym")
    ap.add_argument("--trial", type=int, default=1)
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--M", type=int, default=20)
    ap.add_argument("--s", type=int, default=80)
    ap.add_argument("--steps", type=int, default=26)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    if a.workload == "spd":
        spd(a.out)
        return
    if a.workload == "spread":
        spread(a.out, a.trial, a.N)
        return
    p = workloads.plain_nonsym(a.N)
    S = sketch.sparse_sign_matrix(p.n, a.s, 8, 0x5EEDBA5E)
    hist = method.History(p.n, a.M)
    rows = []
    for i in range(a.steps):
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        A = krylov.csr(rowptr, colind, vals, p.n)
        t0 = time.perf_counter()
        out = method.solve_step(A, b, hist, S, 1e-8, "gmres", restart=30, max_iters=60000)
        dt = time.perf_counter() - t0
        rows.append({"i": i, "iters": int(out["iters"]), "guess_relres": out["guess_relres"],
                     "relres": out["relres"], "status": int(out["status"]), "seconds": dt})
        print(json.dumps(rows[-1]), flush=True)
        full = [r["iters"] for r in rows if r["i"] >= a.M]
        doc = {"workload": f"nonsym {a.N}x{a.N}, v=20(cos t, sin t), dt=0.005, M={a.M}, "
                           f"s={a.s}, zeta=8, GMRES(30) to 1e-8",
               "host": platform.machine(), "systems": rows,
               "mean_iters_full_history": float(np.mean(full)) if full else None}
        with open(a.out, "w") as f:
            json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
