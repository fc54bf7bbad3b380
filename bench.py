#!/usr/bin/env python3
"""Systems per second to a relative residual of 1e-8 on the 1024 x 1024
advection-diffusion sequence (sketched subspace guess + GMRES(30)).

Workload (one system = one step): A(t_i) u = -div(k grad u) + v(t).grad u + u
on a 1024 x 1024 interior grid (n = 1,048,576, nnz = 5,238,784, first-order
upwind, v = 20 (cos t, sin t)), b(t) a circling Gaussian source, t_i = 0.005 i;
history M = 20, sparse-sign sketch s = 80 rows with 8 nonzeros per column,
GMRES(30) with CGS2 to ||b - A x|| <= 1e-8 ||b||, FP64.  A step is seq_guess +
seq_solve + seq_push_solution on device-resident A(t_i), b(t_i).

The history is primed with the first M systems (untimed), then W warm-up steps
and K timed steps follow.  Each step reads a different A(t_i) and the history
(168 MB) and Krylov basis (260 MB) exceed the 129 MB L2, so no flush is needed.

Prints one JSON line (rank 0).  With torchrun every rank runs an independent
replica of the sequence ("replicas only": a single sequence is not sharded).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID, M_HIST, S_ROWS, ZETA, SEED, TOL, RESTART = 1024, 20, 80, 8, 0x5EEDBA5E, 1e-8, 30
METRIC = "systems/sec to rel-res 1e-8 (guess+Krylov)"
WORKLOAD = ("nonsym advection-diffusion 1024x1024 (n=1048576, nnz=5238784), M=20, s=80 "
            "sparse-sign (zeta=8), GMRES(30)-CGS2 to rel-res 1e-8, FP64")


def _gen(i):
    import workloads
    p = workloads.plain_nonsym(N_GRID)
    t = workloads.time_grid(p, i)
    return i, workloads.assemble(p, t), workloads.rhs(p, t)


def generate(steps, workers=8):
    """values and b of systems `steps` (host numpy), generated in a spawn pool."""
    ctx = mp.get_context("spawn")
    out = {}
    with ctx.Pool(min(workers, len(steps))) as pool:
        for i, v, b in pool.imap_unordered(_gen, steps):
            out[i] = (v, b)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(ms, dist=None, device=None):
    """The slowest rank's time in ms (every rank receives it); the time itself
    with a single process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms, world):
    """Units per second of the whole job: all ranks' units over the slowest
    rank's time (replicas: every rank processes the same number of units)."""
    return world * units_per_rank / (ms / 1e3)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Committed ncu summaries that record DRAM/algorithmic byte ratios, by the
# precision of the Krylov kernels: the summary and the kernel sources (in
# csrc/) its counters were taken on; its source_sha256_16 line is the first 16
# hex digits of the SHA-256 of those sources concatenated in this order.
TRAFFIC_PROFILES = {
    "f64": ("arnoldi_kernels_nonsym1024.txt", ("krylov_kernels.cuh",)),
    "f32": ("arnoldi_fp32_kernels_nonsym1024.txt",
            ("krylov_f32_kernels.cuh", "krylov_kernels.cuh")),
    "f32_precond": ("precond_sweeps_nonsym1024.txt",
                    ("precond_kernels.cuh", "krylov_kernels.cuh")),
}


def sources_digest(sources):
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2309_02156_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(kind, algorithmic_bytes, precision="f64"):
    """Per-launch DRAM traffic of `kind` in the given precision ("f64" or "f32"):
    the DRAM/algorithmic byte ratio that the committed ncu summary measured
    times this launch's algorithmic bytes; null when no summary covers the
    kernel or it was taken on different kernel sources."""
    key = "f32_precond" if (precision == "f32" and kind == "precond") else precision
    if key not in TRAFFIC_PROFILES:
        return None
    name, sources = TRAFFIC_PROFILES[key]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if line.startswith("source_sha256_16:"):
            vals["sha"] = line.split(":", 1)[1].strip()
        if line.startswith(f"traffic_ratio[{kind}]:"):
            vals["ratio"] = float(line.split(":", 1)[1].split()[0])
    if vals.get("sha") != sources_digest(sources) or "ratio" not in vals:
        return None
    return vals["ratio"] * algorithmic_bytes


def config_line(world=1):
    """The `config` object of both arms' lines (same workload, same keys)."""
    return {"workload": WORKLOAD, "form": "plain FP64", "history_primed": M_HIST,
            "l2": "inputs larger than L2 (history 168 MB, basis 260 MB, new A(t_i) per step)",
            "parallelism": "replicas" if world > 1 else "single"}


def _oracle_sample_step(A, b, hist, S, gmres_iters):
    """One bounded oracle step: the sketched guess of Algorithm 1 from the
    history, then `gmres_iters` GMRES(30) iterations from it (the tolerance is
    unreachable, so exactly that many run); the iterate is pushed.  Returns
    (guess seconds, seconds per iteration, iterations)."""
    from oracle import krylov, method
    t0 = time.perf_counter()
    g = method.sketched_guess(A, b, hist.matrix(), S)
    t1 = time.perf_counter()
    xk, it, _, _ = krylov.gmres(A, b, g.x0, 1e-30, RESTART, gmres_iters)
    t2 = time.perf_counter()
    hist.push(xk)
    return t1 - t0, (t2 - t1) / max(it, 1), it


def _oracle_history(p, S, upto, gmres_iters):
    """The oracle's own history for system `upto`: systems 0..upto-1 run through
    _oracle_sample_step (guess + capped GMRES, iterate pushed)."""
    from oracle import krylov, method
    import workloads
    hist = method.History(p.n, M_HIST)
    for i in range(max(0, upto - M_HIST), upto):
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        _oracle_sample_step(krylov.csr(rowptr, colind, vals, p.n), b, hist, S, gmres_iters)
    return hist


def cpu_baseline_worker(iters_per_system: float, gmres_iters: int) -> None:
    """Time the oracle on a bounded sample (with the BLAS threads the caller
    set) and print one JSON line."""
    import workloads
    from oracle import krylov, sketch
    p = workloads.plain_nonsym(N_GRID)
    S = sketch.sparse_sign_matrix(p.n, S_ROWS, ZETA, SEED)
    i = M_HIST + 3
    hist = _oracle_history(p, S, i, 10)
    rowptr, colind, vals, b = workloads.csr_system(p, i)
    A = krylov.csr(rowptr, colind, vals, p.n)
    t0 = time.perf_counter()
    tg, ti, it = _oracle_sample_step(A, b, hist, S, gmres_iters)
    timed = time.perf_counter() - t0
    per_system = tg + iters_per_system * ti
    print(json.dumps({"t_guess": tg, "t_iter": ti, "iters_sampled": it, "timed_s": timed,
                      "per_system_s": per_system, "value": 1.0 / per_system}))


def run_cpu_baseline(iters_per_system: float, gmres_iters: int = 120, threads: int = 1):
    """The oracle on `threads` host threads (the BLAS thread count; the sparse
    products are single-threaded either way), in a child process."""
    t = str(threads)
    env = dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker",
           "--iters-per-system", repr(iters_per_system), "--gmres-iters", str(gmres_iters)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": "systems/s", "cores": threads, "kind": "oracle",
                "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    where = "1 host thread" if threads == 1 else f"{threads} host threads"
    return {"value": d["value"], "unit": "systems/s", "cores": threads, "kind": "oracle",
            "timed_s": d["timed_s"],
            "extrapolated": {"timed_iterations": d["iters_sampled"],
                             "iterations_per_system": iters_per_system,
                             "formula": "1 / (guess seconds + iterations_per_system x seconds "
                                        "per timed iteration)"},
            "sample": (f"one 1024x1024 system (history: the oracle's own iterates of the 20 "
                       f"systems before it): oracle sketched guess ({d['t_guess']:.2f} s) + "
                       f"{d['iters_sampled']} GMRES(30) iterations ({d['t_iter'] * 1e3:.1f} ms each) "
                       f"on {where}, timed {d['timed_s']:.1f} s; per-system time = guess + "
                       f"{iters_per_system:.1f} iterations (mean of the GPU run)")}


def oracle_iterations_per_system():
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations_nonsym1024.json")
    if os.path.exists(path):
        d = json.load(open(path))
        if d.get("mean_iters_full_history"):
            return float(d["mean_iters_full_history"]), "oracle run recorded by oracle/measure_iterations.py"
    return None, "no recorded oracle run"


def reference_arm(args):
    """The oracle timed on the host cores, same metric and workload.  Each step
    is a bounded sample of one system of the sequence: the oracle's sketched
    guess from its own history, then 30 GMRES(30) iterations, the iterate
    pushed into the history.  `steps` and `ms_per_step` describe exactly those
    timed samples; `value` extrapolates them to whole systems with the oracle's
    own recorded iteration count (field `extrapolated`)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ips, src = oracle_iterations_per_system()
    import workloads
    from oracle import krylov, sketch
    p = workloads.plain_nonsym(N_GRID)
    S = sketch.sparse_sign_matrix(p.n, S_ROWS, ZETA, SEED)
    gmres_iters = 30
    hist = _oracle_history(p, S, M_HIST, gmres_iters)
    rows = []
    for step in range(args.warmup + args.steps):
        i = M_HIST + step
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        A = krylov.csr(rowptr, colind, vals, p.n)
        t0 = time.perf_counter()
        tg, ti, it = _oracle_sample_step(A, b, hist, S, gmres_iters)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            rows.append((tg, ti, dt))
    tg = statistics.mean(r[0] for r in rows)
    ti = statistics.mean(r[1] for r in rows)
    ms_step = 1e3 * statistics.mean(r[2] for r in rows)
    iters = ips if ips else 0.0
    per = tg + iters * ti
    value = 1.0 / per
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", "0")) or os.cpu_count()
    sample = (f"per step: one 1024x1024 system, oracle sketched guess from the oracle's own "
              f"history + {gmres_iters} GMRES(30) iterations ({ms_step:.0f} ms); per-system time "
              f"= guess + {iters:.1f} iterations ({src})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "systems/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_line(1),
            "extrapolated": {"timed_iterations_per_step": gmres_iters,
                             "iterations_per_system": iters, "source": src,
                             "guess_s": tg, "iteration_s": ti,
                             "formula": "value = 1 / (guess_s + iterations_per_system x "
                                        "iteration_s); ms_per_step is the timed sample"},
            "cpu_baseline": {"value": value, "unit": "systems/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "systems/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_run(iters: int, precision: str = "f64", guess: str = "sketch", sweeps: int = 0,
                precond: str = "jacobi") -> None:
    """A bounded full-size command for ncu: one guess (`guess` mode; m = 10 for
    POD / RAND) from a synthetic 20-column history and `iters` GMRES(30)
    iterations (`precision`: f64, or mixed_krylov = FP32 inner iterations;
    `sweeps` > 0: right-preconditioned by that many Jacobi sweeps) on system 23
    of the 1024 x 1024 sequence, so that a profiler can capture every launch of
    the run."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    p = workloads.plain_nonsym(N_GRID)
    rowptr, colind, vals, b = workloads.csr_system(p, M_HIST + 3)
    dev = torch.device("cuda", 0)
    A = sa.CSR(torch.from_numpy(rowptr).to(dev), torch.from_numpy(colind).to(dev),
               torch.from_numpy(vals).to(dev))
    bd = torch.from_numpy(b).to(dev)
    kw = {"basis_m": 10} if guess in ("pod", "rand") else {}
    seq = sa.Sequence(p.n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, krylov="gmres",
                      restart=RESTART, max_iters=iters, precision=precision, guess=guess,
                      precond_sweeps=sweeps, precond_kind=precond, **kw)
    rng = np.random.default_rng(1)
    for _ in range(M_HIST):
        seq.push(torch.from_numpy(rng.standard_normal(p.n)).to(dev))
    x = torch.empty(p.n, dtype=torch.float64, device=dev)
    g = seq.guess(A, bd, x)
    info = seq.solve(A, bd, TOL, x, allow=(0, 1))
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": True, "guess_launches": g["launches"],
                      "solve_launches": info["launches"], "iters": info["iters"]}))
    seq.close()


def batched_form(K, W, hbm_peak, count=512, plain_sample=16, one_block_ref=False,
                 schedule="auto"):
    """512 independent SPD sequences (grid side 48..384, M = 12, s = 48), FP32 CG
    inside FP64 refinement to 1e-8, one persistent launch per time step (CUDA
    graph).  Systems are assembled on the device between timed steps."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    from workloads.torch_pde import BatchedSystems
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = workloads.batched_params(count, SEED)
    gen = BatchedSystems(ps, dev)
    pats = [(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)) for rp, ci in gen.patterns]
    M, S = 12, 48
    bt = sa.Batch(pats, M=M, s=S, zeta=ZETA, seed=SEED, max_iters=200000)
    xs = [torch.empty(p.n, dtype=torch.float64, device=dev) for p in ps]
    stream = torch.cuda.current_stream()

    def inputs(i):
        v = gen.values(i)
        b = gen.rhs(i)
        torch.cuda.synchronize()
        return gen.split(v, gen.nnz_off), gen.split(b, gen.n_off), (v, b)

    # The plain FP64 GPU method (single-sequence API: sketched guess, FP64 CG,
    # push) on a sample of the sequences, fed the batch's solutions so that it
    # sees the same histories; timed on the step after the batched timing.
    sample = (list(range(0, count, max(1, count // plain_sample)))[:plain_sample]
              if plain_sample else [])
    plain = {k: sa.Sequence(ps[k].n, M, S, zeta=ZETA, seed=SEED, krylov="cg", max_iters=200000)
             for k in sample} if plain_sample else {}

    def feed():
        for k, ctx in plain.items():
            ctx.push(xs[k])

    for i in range(M):
        vs, bs, keep = inputs(i)
        bt.step(vs, bs, xs, TOL)
        feed()
    vs, bs, keep = inputs(M)
    if schedule == "one_block":                # fixed: 1,024 threads, one block per sequence
        bt.set_schedule(1024, 1, 0)
        chosen = bt.schedule()
    else:
        chosen = bt.autotune(vs, bs, xs, TOL)
    for i in range(M, M + W):
        vs, bs, keep = inputs(i)
        bt.step(vs, bs, xs, TOL)
        feed()
    total_ms, infos_all = 0.0, []
    for i in range(M + W, M + W + K):
        vs, bs, keep = inputs(i)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = bt.step(vs, bs, xs, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        infos_all.append(infos)
        feed()
    one_block = None
    if one_block_ref and chosen["ctas_per_sequence"] > 1:
        # the same step under the one-block schedule, for comparison
        vs, bs, keep = inputs(M + W + K)
        bt.set_schedule(1024, 1, 0)
        bt.step(vs, bs, xs, TOL)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        vs, bs, keep = inputs(M + W + K + 1)
        e0.record(stream)
        bt.step(vs, bs, xs, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        one_block = e0.elapsed_time(e1)
    bt.close()
    plain_out = None
    if plain:
        i = M + W + K
        vs, bs, keep = inputs(i)
        pms, pits, prel = 0.0, [], []
        for k, ctx in plain.items():
            A = sa.CSR(pats[k][0], pats[k][1], vs[k].contiguous())
            bk = bs[k].contiguous()
            x = torch.empty(ps[k].n, dtype=torch.float64, device=dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.guess(A, bk, x)
            info = ctx.solve(A, bk, TOL, x)
            ctx.push(x)
            e1.record(stream)
            torch.cuda.synchronize()
            pms += e0.elapsed_time(e1)
            pits.append(info["iters"])
            prel.append(info["final_relres"])
            ctx.close()
        plain_out = {"method": "plain FP64 GPU method, one sequence at a time (sketched guess, FP64 CG, "
                               "push) on %d of the %d sequences (every %d-th), same histories, "
                               "the step after the timed ones" % (len(plain), count, count // len(plain)),
                     "value": 1e3 * len(plain) / pms, "unit": "systems/s",
                     "iters_mean": float(np.mean(pits)), "final_relres_max": max(prel),
                     "sample_n_mean": float(np.mean([ps[k].n for k in plain])),
                     "all_n_mean": float(np.mean([p.n for p in ps]))}
    n = np.array([p.n for p in ps], dtype=np.float64)
    nnz = np.array([p.nnz for p in ps], dtype=np.float64)
    byts = 0.0
    for infos in infos_all:
        it = np.array([f["iters"] for f in infos], dtype=np.float64)
        ref = np.array([f["refinements"] for f in infos], dtype=np.float64)
        # guess (A, X, b, x0 = X y, push), FP32 copy of A, FP64 residuals, FP32 CG
        byts += float(np.sum(12 * nnz + 8 * n * (M + 3) + 12 * nnz + (ref + 1) * (12 * nnz + 24 * n)
                             + it * (8 * nnz + 28 * n)))
    secs = total_ms / 1e3
    flat = [f for infos in infos_all for f in infos]
    return {
        "form": "batched: %d SPD sequences (N 48..384, sum n = %d), M = 12, s = 48, FP32 CG "
                "inside FP64 refinement to 1e-8, one persistent launch per step" % (count, int(n.sum())),
        "value": count * K / secs, "unit": "systems/s", "ms_per_step": total_ms / K,
        "schedule": chosen, "iters_mean": float(np.mean([f["iters"] for f in flat])),
        "refinements_mean": float(np.mean([f["refinements"] for f in flat])),
        "final_relres_max": max(f["final_relres"] for f in flat),
        "all_converged": all(f["status"] == 0 for f in flat),
        "plain_fp64": plain_out,
        "one_block_ms_per_step": one_block,
        "roofline": {"bound": "hbm",
                     "kernel": ("batched_cluster_kernel" if chosen["ctas_per_sequence"] > 1
                                else "batched_step_kernel"),
                     "achieved": byts / secs / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": byts / secs / 1e9 / hbm_peak},
    }


def _gen_learned(job):
    import workloads
    from workloads.pde import PDEParams
    a, N, i = job
    p = PDEParams(N=N, a=a, phi=0.0, rc=0.2, v0=20.0, dt=0.005)
    t = workloads.time_grid(p, i)
    return workloads.assemble(p, t), workloads.rhs(p, t)


def learned_ablation(args):
    """The learned form's ablation as a separate mode (one JSON line)."""
    print(json.dumps(learned_run(args.learned_train, args.learned_eval, args.learned_grid,
                                 args.learned_seqs, args.learned_epochs)), flush=True)


def learned_bounded(args):
    """A bounded ablation of the learned form for the default line: one 512 x 512
    sequence, training on systems 0..119, evaluation on 120..159."""
    out = learned_run(120, 40, 512, 1, args.learned_epochs)
    out["bound"] = ("the least-squares y minimises the sketched residual, so the network can at "
                    "best equal it on that measure (rho_s(net) >= rho_s(LS)); its guess is used "
                    "when rho_s(net) <= 1.5 rho_s(LS)")
    return out


def learned_run(T, E, N, nseq, epochs):
    """Learned coefficient predictor against sketched least squares.

    Workload: advection-diffusion sequences as in the main line on a 512 x 512
    grid (n = 262,144), one per k amplitude a ~ U[0.2, 0.8] (seeded), M = 20,
    s = 80, GMRES(30) to 1e-8 (FP64).  The predictor (160 -> 256 -> 256 -> 20,
    BF16 weights) is trained on the GPU on the samples of steps 0..T-1 and
    evaluated on steps T..T+E-1.  Two contexts see identical histories (the
    least-squares path's solution is pushed into both); each evaluation system
    is solved from both guesses.  Prints one JSON line."""
    import numpy as np
    amps = __import__("workloads").learned_amplitudes(nseq, SEED)
    pool = mp.get_context("spawn").Pool(8)
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    dev = torch.device("cuda", 0)
    rowptr, colind, _ = workloads.pattern(N)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    n = N * N
    net = sa.MLP(M_HIST, S_ROWS, hidden=256, max_batch=64, seed=SEED)
    stride = net.stride

    def systems(a, lo, hi, chunk=32):
        nxt = pool.map_async(_gen_learned, [(a, N, i) for i in range(lo, min(lo + chunk, hi))])
        for c0 in range(lo, hi, chunk):
            got = nxt.get()
            c1 = c0 + chunk
            if c1 < hi:
                nxt = pool.map_async(_gen_learned, [(a, N, i) for i in range(c1, min(c1 + chunk, hi))])
            for k, (v, b) in enumerate(got):
                yield c0 + k, torch.from_numpy(v).to(dev), torch.from_numpy(b).to(dev)

    mk = lambda: sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, guess="learned",
                             krylov="gmres", restart=RESTART, max_iters=60000)
    ctxs, samples, train_iters = [], [], []
    t0 = time.time()
    for a in amps:
        c_ls, c_net = mk(), mk()
        x = torch.empty(n, dtype=torch.float64, device=dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        for i, v, b in systems(a, 0, T):
            A = sa.CSR(rp, ci, v)
            c_ls.guess(A, b, x)
            c_net.guess(A, b, y)
            buf = torch.empty(stride, dtype=torch.float32, device=dev)
            try:
                c_ls.last_sample(buf)
                samples.append(buf)
            except sa.SeqError:
                pass
            info = c_ls.solve(A, b, TOL, x)
            train_iters.append(info["iters"])
            c_ls.push(x)
            c_net.push(x)
        ctxs.append((a, c_ls, c_net))
    gen_s = time.time() - t0
    St = torch.stack(samples)
    net.fit_normalization(St)
    torch.cuda.synchronize()
    t1 = time.time()
    losses = net.train(St, epochs=epochs, batch=32, lr=1e-3, seed=SEED)
    torch.cuda.synchronize()
    train_s = time.time() - t1
    rec = {"ls_guess": [], "net_guess": [], "ls_iters": [], "net_iters": [], "fallback": [],
           "ls_rho": [], "net_rho": [], "ratio": [], "fp32_floor": [], "ymax": []}
    for a, c_ls, c_net in ctxs:
        c_net.set_learned(net)
        x = torch.empty(n, dtype=torch.float64, device=dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        for i, v, b in systems(a, T, T + E):
            A = sa.CSR(rp, ci, v)
            g1 = c_ls.guess(A, b, x)
            g2 = c_net.guess(A, b, y)
            i1 = c_ls.solve(A, b, TOL, x)
            i2 = c_net.solve(A, b, TOL, y)
            rec["ls_guess"].append(g1["guess_relres"])
            rec["net_guess"].append(g2["guess_relres"])
            rec["ls_rho"].append(g1["sketch_resid"])
            rec["net_rho"].append(g2["sketch_resid"])
            rec["ls_iters"].append(i1["iters"])
            rec["net_iters"].append(i2["iters"])
            rec["fallback"].append(bool(g2["fallback"]))
            if g2["net_resid"] > 0 and g1["sketch_resid"] > 0:
                rec["ratio"].append(g2["net_resid"] / g1["sketch_resid"])
            # Floor of any FP32-output predictor: the least-squares y itself
            # rounded to FP32, tested in FP64 on the same sketched block.
            Wf, yf = c_ls.last_sketch()
            Wf = Wf.reshape(S_ROWS, M_HIST + 1)
            r64 = np.linalg.norm(Wf[:, :M_HIST] @ yf - Wf[:, M_HIST])
            r32 = np.linalg.norm(Wf[:, :M_HIST] @ yf.astype(np.float32).astype(np.float64)
                                 - Wf[:, M_HIST])
            if r64 > 0:
                rec["fp32_floor"].append(r32 / r64)
                rec["ymax"].append(float(np.abs(yf).max()))
            c_ls.push(x)
            c_net.push(x)
        c_ls.close()
        c_net.close()
    pool.close()
    gm = lambda v: float(np.exp(np.mean(np.log(np.asarray(v, dtype=np.float64)))))
    used = [not f for f in rec["fallback"]]
    out = {
        "learned_ablation": True,
        "workload": "advection-diffusion %dx%d (n=%d), a ~ U[0.2,0.8] x %d sequences, M=20, s=80, "
                    "GMRES(30) to 1e-8; train steps 0..%d, evaluate %d..%d"
                    % (N, N, n, nseq, T - 1, T, T + E - 1),
        "amplitudes": amps, "samples": int(St.shape[0]), "epochs": epochs,
        "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]),
        "train_seconds": train_s, "data_seconds": gen_s,
        "train_iters_mean": float(np.mean(train_iters)),
        "eval_systems": len(rec["ls_iters"]),
        "ls": {"guess_relres_geomean": gm(rec["ls_guess"]), "iters_mean": float(np.mean(rec["ls_iters"])),
               "sketch_resid_geomean": gm(rec["ls_rho"])},
        "net": {"guess_relres_geomean": gm(rec["net_guess"]),
                "iters_mean": float(np.mean(rec["net_iters"])),
                "sketch_resid_geomean": gm(rec["net_rho"]),
                "used_fraction": float(np.mean(used)),
                "net_over_ls_sketch_resid_geomean": gm(rec["ratio"]) if rec["ratio"] else None,
                "net_over_ls_sketch_resid_min": float(min(rec["ratio"])) if rec["ratio"] else None},
        "fp32_rounded_ls_y_over_ls_sketch_resid_geomean": gm(rec["fp32_floor"]),
        "fp32_rounded_ls_y_rejected_fraction": float(np.mean(np.asarray(rec["fp32_floor"]) > 1.5)),
        "ls_y_absmax_geomean": gm(rec["ymax"]),
        "net_over_ls_guess_relres_geomean": gm(np.asarray(rec["net_guess"]) / np.asarray(rec["ls_guess"])),
    }
    net.close()
    return out


def spd_small(steps=60):
    """The 64 x 64 SPD sequence (n = 4096, M = 10, s = 40, CG to 1e-10, 60
    systems): the sketched guess against the previous-solution guess (the
    paper's baseline), each in its own sequence; CG iterations and device time
    per system over systems M..59 (this size is L2- and latency-bound, so the
    time per system, not an HBM fraction, is the figure)."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    dev = torch.device("cuda", torch.cuda.current_device())
    p = workloads.plain_spd(64)
    M, S = 10, 40
    systems = []
    for i in range(steps):
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        systems.append((torch.from_numpy(rowptr).to(dev), torch.from_numpy(colind).to(dev),
                        torch.from_numpy(vals).to(dev), torch.from_numpy(b).to(dev)))
    stream = torch.cuda.current_stream()
    out = {"workload": "SPD 64x64 (n=4096), M=10, s=40, CG to rel-res 1e-10, %d systems" % steps}
    for mode in ("sketch", "prev"):
        seq = sa.Sequence(p.n, M, S, zeta=ZETA, seed=SEED, krylov="cg", guess=mode, max_iters=100000)
        x = torch.zeros(p.n, dtype=torch.float64, device=dev)
        its, ms = [], 0.0
        for i, (rp, ci, v, b) in enumerate(systems):
            A = sa.CSR(rp, ci, v)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            seq.guess(A, b, x)
            info = seq.solve(A, b, 1e-10, x)
            seq.push(x)
            e1.record(stream)
            torch.cuda.synchronize()
            assert info["status"] == 0
            if i >= M:
                its.append(info["iters"])
                ms += e0.elapsed_time(e1)
        seq.close()
        out[mode] = {"iters_mean": float(np.mean(its)), "us_per_system": 1e3 * ms / len(its),
                     "systems_per_s": 1e3 * len(its) / ms}
    out["iteration_ratio_prev_over_sketch"] = out["prev"]["iters_mean"] / max(out["sketch"]["iters_mean"], 1e-9)
    rec = os.path.join(ROOT, "tests", "golden", "oracle_iterations_spd64.json")
    if os.path.exists(rec):
        d = json.load(open(rec))
        out["oracle"] = {"sketch_iters_mean": d["sketch"]["iters_mean_full_history"],
                         "prev_iters_mean": d["prev"]["iters_mean_full_history"],
                         "source": "recorded by oracle/measure_iterations.py --workload spd "
                                   "(same sequence, systems M..59)"}
    return out


def guess_modes(args):
    """Guess modes compared on identical histories (the comparison of the
    paper's Section 4 experiment on the 1024 x 1024 sequence): the previous
    solution (the paper's baseline), Algorithm 1 over the whole span (sketched),
    POD (Algorithm 2) and the randomised range finder (Algorithm 4, refresh 50),
    m = args.basis_m.  A driver context (whole span) primes and advances the
    history; at each timed step every mode guesses from the same history and
    solves from its own guess (GMRES(30) to 1e-8, FP64); the driver's solution
    is pushed into all contexts.  Prints one JSON line."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    K = args.modes_steps
    dev = torch.device("cuda", 0)
    total = M_HIST + K
    host = generate(list(range(total)))
    rowptr, colind, _ = workloads.pattern(N_GRID)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    n = N_GRID * N_GRID
    mk = lambda g, **kw: sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, guess=g, krylov="gmres",
                                     restart=RESTART, max_iters=200000, **kw)
    modes = {"prev": mk("prev"), "sketch": mk("sketch"),
             "pod": mk("pod", basis_m=args.basis_m), "rand": mk("rand", basis_m=args.basis_m, refresh=50)}
    x = torch.empty(n, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rec = {k: {"iters": [], "guess": [], "guess_ms": [], "solve_ms": []} for k in modes}
    for i in range(total):
        v = torch.from_numpy(host[i][0]).to(dev)
        b = torch.from_numpy(host[i][1]).to(dev)
        A = sa.CSR(rp, ci, v)
        timed = i >= M_HIST
        if timed:
            for k, ctx in modes.items():
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                torch.cuda.synchronize()
                ev[0].record(stream)
                g = ctx.guess(A, b, y)
                ev[1].record(stream)
                info = ctx.solve(A, b, TOL, y)
                ev[2].record(stream)
                torch.cuda.synchronize()
                r = rec[k]
                r["iters"].append(info["iters"])
                r["guess"].append(g["guess_relres"])
                r["guess_ms"].append(ev[0].elapsed_time(ev[1]))
                r["solve_ms"].append(ev[1].elapsed_time(ev[2]))
                if k == "sketch":
                    x.copy_(y)              # the whole-span solution advances every history
        else:
            for k, ctx in modes.items():
                if k == "sketch":
                    ctx.guess(A, b, x)
                    ctx.solve(A, b, TOL, x)
            for k, ctx in modes.items():
                if k != "sketch":
                    ctx.guess(A, b, y)      # keeps each mode's state in step (RAND: Omega)
        for ctx in modes.values():
            ctx.push(x)
    for ctx in modes.values():
        ctx.close()
    gm = lambda v: float(np.exp(np.mean(np.log(np.maximum(np.asarray(v, dtype=np.float64), 1e-300)))))
    out = {"guess_modes": True, "workload": WORKLOAD, "basis_m": args.basis_m, "steps": K,
           "modes": {k: {"iters_mean": float(np.mean(r["iters"])),
                         "guess_relres_geomean": gm(r["guess"]),
                         "guess_ms_mean": float(np.mean(r["guess_ms"])),
                         "solve_ms_mean": float(np.mean(r["solve_ms"])),
                         "systems_per_s": 1e3 * K / (sum(r["guess_ms"]) + sum(r["solve_ms"]))}
                     for k, r in rec.items()}}
    print(json.dumps(out), flush=True)


def e1_sequence(args):
    """The paper's Section 4 test sequence (workloads/e1.py): N x N fourth-order
    discretisation of div(a grad f) = g, t0 = 2.3, `steps` systems, GMRES(30)
    to 1e-7, unpreconditioned (the paper uses ILU, so the iteration counts are
    not those of its Figure 1).  For each of dt = 1e-5 (M = 20, m = 10) and
    dt = 1e-3 (M = 31, m = 20: the paper's M = 35 exceeds this library's
    M <= 31), every guess mode runs its own sequence.  Prints one JSON line."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    from workloads import e1
    dev = torch.device("cuda", 0)
    N, steps, tol = args.e1_grid, args.e1_steps, 1e-7
    rowptr, colind = e1.pattern(N)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    n = N * N
    out = {"e1": True, "grid": N, "steps": steps, "tol": tol, "precond_sweeps": args.e1_sweeps,
           "runs": []}
    for dt, M, m in ((1e-5, 20, 10), (1e-3, 31, 20)):
        p = e1.E1Params(N=N, dt=dt)
        sysv = [e1.system(p, k, rowptr, colind) for k in range(steps)]
        vals = [torch.from_numpy(v[2]).to(dev) for v in sysv]
        bs = [torch.from_numpy(v[3]).to(dev) for v in sysv]
        fx = [v[4] for v in sysv]
        run = {"dt": dt, "M": M, "m": m, "modes": {}}
        for mode in ("prev", "sketch", "pod", "rand"):
            kw = {"basis_m": m, "refresh": 50} if mode in ("pod", "rand") else {}
            seq = sa.Sequence(n, M, 80, zeta=ZETA, seed=SEED, guess=mode, krylov="gmres",
                              restart=RESTART, max_iters=500000, precond_sweeps=args.e1_sweeps, **kw)
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            its, zero, errs = [], 0, []
            torch.cuda.synchronize()
            t0 = time.time()
            for k in range(steps):
                A = sa.CSR(rp, ci, vals[k])
                seq.guess(A, bs[k], x)
                info = seq.solve(A, bs[k], tol, x)
                its.append(info["iters"])
                zero += info["iters"] == 0
                seq.push(x)
                if k % 50 == 0:
                    errs.append(float(np.abs(x.cpu().numpy() - fx[k]).max() / np.abs(fx[k]).max()))
            torch.cuda.synchronize()
            wall = time.time() - t0
            seq.close()
            run["modes"][mode] = {"iters_mean": float(np.mean(its)), "iters_total": int(np.sum(its)),
                                  "zero_iteration_steps": int(zero), "seconds": wall,
                                  "iters_first10": its[:10], "iters_last10": its[-10:],
                                  "max_rel_error_vs_f_sampled": max(errs)}
        out["runs"].append(run)
    print(json.dumps(out), flush=True)


def precond_form(args):
    """The 1024 x 1024 sequence with right-preconditioned GMRES(30) (M^{-1} =
    `sweeps` damped Jacobi sweeps, omega 0.8), in FP64 and in the mixed form
    (FP32 inner solves in FP64 refinement), to rel-res 1e-8; sketched guess
    M = 20, s = 80.  M + W priming systems, then K timed steps (guess + solve +
    push, CUDA events).  Prints one JSON line."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    K, W, d = args.steps, args.warmup, args.precond_sweeps
    total = M_HIST + W + K
    host = generate(list(range(total)))
    dev = torch.device("cuda", 0)
    rowptr, colind, _ = workloads.pattern(N_GRID)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    n = N_GRID * N_GRID
    vals = {i: torch.from_numpy(host[i][0]).to(dev) for i in range(total)}
    bs = {i: torch.from_numpy(host[i][1]).to(dev) for i in range(total)}
    stream = torch.cuda.current_stream()
    out = {"precond_form": True, "workload": WORKLOAD.replace("GMRES(30)", "right-preconditioned GMRES(30)"),
           "sweeps": d, "omega": 0.8, "steps": K, "forms": {}}
    for prec in ("f64", "mixed_krylov"):
        seq = sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, krylov="gmres", restart=RESTART,
                          max_iters=200000, precision=prec, precond_sweeps=d)
        x = torch.empty(n, dtype=torch.float64, device=dev)
        rec = []

        def step(i):
            A = sa.CSR(rp, ci, vals[i])
            seq.guess(A, bs[i], x)
            info = seq.solve(A, bs[i], TOL, x)
            seq.push(x)
            return info
        for i in range(M_HIST + W):
            step(i)
        seq.set_profiling(True)
        seq.kernel_stats(reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(M_HIST + W, total):
            rec.append(step(i))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stats = seq.kernel_stats(reset=True)
        seq.close()
        tot_ms = sum(v["ms"] for v in stats.values()) or 1.0
        out["forms"][prec] = {
            "value": 1e3 * K / ms, "unit": "systems/s", "ms_per_step": ms / K,
            "iters_per_system": float(np.mean([r["iters"] for r in rec])),
            "refinements_per_system": float(np.mean([r["refinements"] for r in rec])),
            "final_relres_max": max(r["final_relres"] for r in rec),
            "all_converged": all(r["status"] == 0 for r in rec),
            "kernels": {k: {"launches": v["launches"], "share": v["ms"] / tot_ms,
                            "GB/s": v["bytes"] / (v["ms"] * 1e6) if v["ms"] else 0.0}
                        for k, v in stats.items() if v["launches"]}}
    print(json.dumps(out), flush=True)


def _gen_nonsym(job):
    import workloads
    N, i = job
    p = workloads.plain_nonsym(N)
    t = workloads.time_grid(p, i)
    return workloads.assemble(p, t), workloads.rhs(p, t)


def precision_form(args):
    """Precision form on the 2048 x 2048 advection-diffusion sequence
    (n = 4,194,304, nnz = 20,963,328): FP32 CSR values, FP32 history and sketch
    of A X, FP32 GMRES(30) inner solves inside FP64 residual refinement to
    ||b - A x|| <= 1e-10 ||b||, FP64 least squares (M = 20, s = 80).  The first
    `prime` systems fill the history (untimed, same method), then W warm-up and
    K timed steps (seq_guess + seq_solve + seq_push_solution).  Prints one JSON
    line; the per-step FP64 residuals are computed on the device by the library."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    N, tol = args.precision_grid, 1e-10
    P, W, K = args.precision_prime, args.precision_warmup, args.precision_steps
    pool = mp.get_context("spawn").Pool(8)
    dev = torch.device("cuda", 0)
    rowptr, colind, _ = workloads.pattern(N)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    n = N * N
    seq = sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, precision=args.precision_kind,
                      krylov="gmres", restart=RESTART, max_iters=400000,
                      precond_sweeps=args.precision_sweeps, precond_kind=args.precision_precond)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    total = P + W + K
    nxt = pool.map_async(_gen_nonsym, [(N, i) for i in range(0, min(4, total))])
    rows, timed_ms = [], []
    stream = torch.cuda.current_stream()
    for c0 in range(0, total, 4):
        got = nxt.get()
        if c0 + 4 < total:
            nxt = pool.map_async(_gen_nonsym, [(N, i) for i in range(c0 + 4, min(c0 + 8, total))])
        for k, (v, b) in enumerate(got):
            i = c0 + k
            vd = torch.from_numpy(v).to(dev)
            bd = torch.from_numpy(b).to(dev)
            A = sa.CSR(rp, ci, vd)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            w0 = time.time()
            e0.record(stream)
            g = seq.guess(A, bd, x)
            info = seq.solve(A, bd, tol, x)
            seq.push(x)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rows.append({"i": i, "guess_relres": g["guess_relres"], "iters": info["iters"],
                         "refinements": info["refinements"], "final_relres": info["final_relres"],
                         "status": info["status"], "ms": ms, "wall_s": time.time() - w0})
            if i >= P + W:
                timed_ms.append(ms)
            print(json.dumps({"precision_step": rows[-1]}), file=sys.stderr, flush=True)
    pool.close()
    seq.close()
    timed = rows[P + W:]
    out = {
        "precision_form": True,
        "workload": "nonsym advection-diffusion %dx%d (n=%d), M=20, s=80, %s: FP32 values/history/"
                    "inner GMRES(30)%s, FP64 refinement to rel-res 1e-10"
                    % (N, N, n, args.precision_kind,
                       " right-preconditioned by %s of degree %d" % (args.precision_precond,
                                                                       args.precision_sweeps)
                       if args.precision_sweeps else ""),
        "value": 1e3 * K / sum(timed_ms), "unit": "systems/s", "ms_per_step": sum(timed_ms) / K,
        "steps": K, "warmup": W, "prime": P,
        "iters_mean": float(np.mean([r["iters"] for r in timed])),
        "refinements_mean": float(np.mean([r["refinements"] for r in timed])),
        "guess_relres_geomean": float(np.exp(np.mean(np.log([r["guess_relres"] for r in timed])))),
        "final_relres_max": max(r["final_relres"] for r in timed),
        "all_converged": all(r["status"] == 0 for r in rows),
        "per_step": rows,
    }
    print(json.dumps(out), flush=True)


def precision_startup(hbm_peak):
    """The precision form on the first five systems of the 2048 x 2048 sequence
    (SEQ_MIXED: FP32 values, history, sketch and inner GMRES(30) right-
    preconditioned by the degree-8 Chebyshev polynomial of D^-1 A, FP64
    refinement to 1e-10), with
    the error of every solution against the oracle's direct solve recorded by
    oracle/reference_solutions.py (sampled entries; see the error estimate
    there).  Systems 0..4 have histories of 0..4 columns."""
    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    path = os.path.join(ROOT, "tests", "golden", "reference_solutions_nonsym2048.json")
    ref = json.load(open(path)) if os.path.exists(path) else None
    N, tol, steps = 2048, 1e-10, 5
    with mp.get_context("spawn").Pool(5) as pool:
        systems = pool.map(_gen_nonsym, [(N, i) for i in range(steps)])
    dev = torch.device("cuda", torch.cuda.current_device())
    rowptr, colind, _ = workloads.pattern(N)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    n = N * N
    seq = sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, precision="mixed", krylov="gmres",
                      restart=RESTART, max_iters=400000, precond_sweeps=8,
                      precond_kind="chebyshev")
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rows = []
    for i, (v, b) in enumerate(systems):
        vd = torch.from_numpy(v).to(dev)
        bd = torch.from_numpy(b).to(dev)
        A = sa.CSR(rp, ci, vd)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = seq.guess(A, bd, x)
        info = seq.solve(A, bd, tol, x)
        seq.push(x)
        e1.record(stream)
        torch.cuda.synchronize()
        row = {"i": i, "history_cols": g["history_cols"], "guess_relres": g["guess_relres"],
               "inner_iters": info["iters"], "refinements": info["refinements"],
               "final_relres": info["final_relres"], "status": info["status"],
               "ms": e0.elapsed_time(e1)}
        if ref and i < len(ref["systems"]):
            r = ref["systems"][i]
            idx = torch.tensor(r["idx"], dtype=torch.int64, device=dev)
            xs = x[idx].cpu().numpy()
            xo = np.asarray(r["x"])
            row["err_vs_oracle"] = float(math.sqrt(n / len(idx) * float(np.sum((xs - xo) ** 2)))
                                         / r["norm2"])
            row["err_max_sampled"] = float(np.max(np.abs(xs - xo)) / np.max(np.abs(xo)))
            row["norm_rel_diff"] = abs(float(torch.linalg.vector_norm(x)) - r["norm2"]) / r["norm2"]
        rows.append(row)
    seq.close()
    total = sum(r["ms"] for r in rows)
    return {
        "form": "precision: nonsym 2048x2048 (n=4194304), FP32 values/history/sketch/inner "
                "GMRES(30) with the degree-8 Chebyshev preconditioner, FP64 QR, refinement "
                "residual and test to 1e-10",
        "systems": "0..4 (start of the sequence: histories of 0..4 columns)",
        "value": 1e3 * steps / total, "unit": "systems/s", "ms_per_step": total / steps,
        "all_converged": all(r["status"] == 0 for r in rows),
        "error_reference": ("oracle.krylov.direct_solve (sparse LU + FP64 refinement), "
                            "recorded by oracle/reference_solutions.py: err = sqrt(n/k sum "
                            "(x - x_oracle)^2 over k = 1024 sampled entries) / ||x_oracle||")
        if ref else "no recorded reference solutions",
        "per_step": rows,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-chosen", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--cpu-baseline-worker", action="store_true")
    ap.add_argument("--iters-per-system", type=float, default=0.0)
    ap.add_argument("--gmres-iters", type=int, default=120)
    ap.add_argument("--profile-run", type=int, default=0, metavar="ITERS")
    ap.add_argument("--profile-precision", default="f64", choices=["f64", "mixed_krylov"])
    ap.add_argument("--profile-guess", default="sketch", choices=["sketch", "pod", "rand"])
    ap.add_argument("--profile-sweeps", type=int, default=0)
    ap.add_argument("--profile-precond", default="jacobi", choices=["jacobi", "chebyshev"])
    ap.add_argument("--batched-only", action="store_true")
    ap.add_argument("--batched-schedule", default="auto", choices=["auto", "one_block"])
    ap.add_argument("--batched-count", type=int, default=512)
    ap.add_argument("--precond-form", action="store_true")
    ap.add_argument("--precond-sweeps", type=int, default=4)
    ap.add_argument("--precond-ratio", type=float, default=0.0,
                    help="Chebyshev interval ratio lmax/lmin (0: the library default)")
    ap.add_argument("--e1", action="store_true")
    ap.add_argument("--e1-grid", type=int, default=100)
    ap.add_argument("--e1-steps", type=int, default=200)
    ap.add_argument("--e1-sweeps", type=int, default=0)
    ap.add_argument("--guess-modes", action="store_true")
    ap.add_argument("--modes-steps", type=int, default=8)
    ap.add_argument("--basis-m", type=int, default=10)
    ap.add_argument("--precision-form", action="store_true")
    ap.add_argument("--precision-kind", default="mixed", choices=["mixed", "mixed_krylov", "f64"])
    ap.add_argument("--precision-grid", type=int, default=2048)
    ap.add_argument("--precision-prime", type=int, default=20)
    ap.add_argument("--precision-warmup", type=int, default=1)
    ap.add_argument("--precision-steps", type=int, default=5)
    ap.add_argument("--precision-sweeps", type=int, default=0)
    ap.add_argument("--precision-precond", default="jacobi", choices=["jacobi", "chebyshev"])
    ap.add_argument("--learned-ablation", action="store_true")
    ap.add_argument("--learned-train", type=int, default=400)
    ap.add_argument("--learned-eval", type=int, default=400)
    ap.add_argument("--learned-grid", type=int, default=512)
    ap.add_argument("--learned-seqs", type=int, default=1)
    ap.add_argument("--learned-epochs", type=int, default=300)
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    args = ap.parse_args()
    if args.learned_ablation:
        learned_ablation(args)
        return
    if args.precision_form:
        precision_form(args)
        return
    if args.guess_modes:
        guess_modes(args)
        return
    if args.e1:
        e1_sequence(args)
        return
    if args.precond_form:
        precond_form(args)
        return
    if args.profile_run:
        profile_run(args.profile_run, args.profile_precision, args.profile_guess,
                    args.profile_sweeps, args.profile_precond)
        return
    if args.batched_only:
        import torch
        hbm_peak, _ = peaks()
        torch.cuda.set_device(0)
        print(json.dumps(batched_form(args.batched_steps, args.warmup, hbm_peak, args.batched_count,
                                      schedule=args.batched_schedule)))
        return
    if args.cpu_baseline_worker:
        cpu_baseline_worker(args.iters_per_system, args.gmres_iters)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    K, W = args.steps, args.warmup
    KP = max(1, min(K, 3))          # steps of the separate per-kernel profiled pass
    steps_dev = list(range(M_HIST + W + K + KP))
    steps_e2e = list(range(M_HIST + W, M_HIST + W + K))    # the timed systems again
    host = generate(steps_dev)     # before any CUDA call (spawn pool)

    import numpy as np
    import torch
    import paper_2309_02156_gb300 as sa
    import workloads
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    p = workloads.plain_nonsym(N_GRID)
    n = p.n
    rowptr, colind, _ = workloads.pattern(N_GRID)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colind).to(dev)
    vals = {i: torch.from_numpy(host[i][0]).to(dev) for i in steps_dev}
    bs = {i: torch.from_numpy(host[i][1]).to(dev) for i in steps_dev}
    seq = sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, krylov="gmres", restart=RESTART,
                      max_iters=60000)
    x = torch.empty(n, dtype=torch.float64, device=dev)

    def step(i):
        A = sa.CSR(rp, ci, vals[i])
        g = seq.guess(A, bs[i], x)
        info = seq.solve(A, bs[i], TOL, x)
        seq.push(x)
        return g, info

    fp64_peak = sa.probe_fp64_peak()
    hbm_peak, hbm_src = peaks()
    stream = torch.cuda.current_stream()
    t_first = M_HIST + W
    timed_steps = range(t_first, t_first + K)
    prof_steps = range(t_first + K, t_first + K + KP)

    def timed(steps):
        """Device time (max over ranks) of seq steps, un-instrumented."""
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = [step(i) for i in steps]
        b.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return max_over_ranks(a.elapsed_time(b), dist, dev), out

    def profiled(steps):
        """Per-kernel statistics (CUDA events between the kernels of the
        restart-cycle graph) over a separate pass of seq steps."""
        seq.set_profiling(True)
        seq.kernel_stats(reset=True)
        out = [step(i) for i in steps]
        torch.cuda.synchronize()
        st = seq.kernel_stats(reset=True)
        seq.set_profiling(False)
        return st, out

    def roofline(stats, label_steps, fp64=True):
        """Roof of the dominant kernel: FP64 FMA throughput when its FP64
        arithmetic takes longer than its bytes at the HBM peak; otherwise (and
        always for FP32 kernels, whose FP32 rate is ~70x the FP64 one) HBM."""
        dom = max(stats, key=lambda k: stats[k]["ms"])
        st = stats[dom]
        t_launch = st["ms"] / 1e3 / max(st["launches"], 1)
        bytes_l = st["bytes"] / max(st["launches"], 1)
        flops_l = st["flops"] / max(st["launches"], 1)
        t_hbm = bytes_l / (hbm_peak * 1e9)
        t_alu = flops_l / (fp64_peak * 1e12) if fp64 else 0.0
        if t_alu > t_hbm:
            roof = {"bound": "alu", "achieved": flops_l / t_launch / 1e12, "peak": fp64_peak,
                    "unit": "TFLOP/s", "peak_source": "FP64 FMA probe measured in this run"}
        else:
            roof = {"bound": "hbm", "achieved": bytes_l / t_launch / 1e9, "peak": hbm_peak,
                    "unit": "GB/s", "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({hbm_src})"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["traffic"] = profile_traffic(dom, bytes_l, "f64" if fp64 else "f32")
        roof["kernel"] = dom
        if dom == "precond":
            roof["note"] = ("the sweeps of one preconditioner application re-read the same matrix, "
                            "which stays in L2 between them; the algorithmic bytes count it at "
                            "every sweep, so the fraction of the HBM copy rate can exceed 1 "
                            "(profiles/precond_sweeps_nonsym1024.txt: DRAM reads per sweep with "
                            "a cold and a warm L2)")
        roof["algorithmic_bytes_per_launch"] = bytes_l
        roof["algorithmic_flops_per_launch"] = flops_l
        roof["launch_us"] = t_launch * 1e6
        roof["timing"] = ("CUDA events on the context's stream between the kernels of the "
                          "restart-cycle graph (the sweeps of one preconditioner application "
                          "between one pair), averaged over every launch of a separate "
                          "profiled pass (systems %d..%d)" % (label_steps[0], label_steps[-1]))
        total_ms = sum(v["ms"] for v in stats.values())
        kernels = {k: {"launches": v["launches"],
                       "share": v["ms"] / total_ms if total_ms else None,
                       "GB/s": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] else None,
                       "TFLOP/s": v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] else None}
                   for k, v in stats.items() if v["launches"]}
        return roof, kernels

    # The last M solutions before the timed region are kept so that the end-to-
    # end pass can replay the timed systems from the same history (the library
    # is deterministic: same inputs, same iterations).
    hist_keep = []
    prime = []
    for i in range(t_first):
        out = step(i)
        if i < M_HIST:
            prime.append(out)
        if i >= t_first - M_HIST:
            hist_keep.append(x.clone())
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[local].strip().isdigit():
        gpu_index = int(vis.split(",")[local])
    sampler = ClockSampler(gpu_index)
    sampler.start()
    ms, infos = timed(timed_steps)
    clocks = sampler.stop()
    stats, _ = profiled(prof_steps)
    value = whole_job_rate(K, ms, world)
    iters = [inf["iters"] for _, inf in infos]
    launches = sum(g["launches"] + inf["launches"] + 1 for g, inf in infos)
    worst = max(inf["final_relres"] for _, inf in infos)
    assert all(inf["status"] == 0 for _, inf in infos), "a timed solve did not converge"
    roof, kernels = roofline(stats, list(prof_steps))

    # End to end through the public API: the timed systems again, from the same
    # history, in a fresh context; every step copies its inputs from pinned
    # host memory and the solution back.
    seq.close()
    seq = sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, krylov="gmres", restart=RESTART,
                      max_iters=60000)
    zero = torch.zeros(n, dtype=torch.float64, device=dev)
    for _ in range(t_first - M_HIST):      # same ring slots as the timed context
        seq.push(zero)
    for xk in hist_keep:
        seq.push(xk)
    del hist_keep, zero
    pin = {i: (torch.from_numpy(host[i][0]).pin_memory(), torch.from_numpy(host[i][1]).pin_memory())
           for i in steps_e2e}
    rp_h = torch.from_numpy(rowptr).pin_memory()
    ci_h = torch.from_numpy(colind).pin_memory()
    v_d = torch.empty_like(vals[steps_dev[0]])
    b_d = torch.empty_like(bs[steps_dev[0]])
    rp_d = torch.empty_like(rp)
    ci_d = torch.empty_like(ci)
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    h2d = rp_h.numel() * 4 + ci_h.numel() * 4 + v_d.numel() * 8 + b_d.numel() * 8
    d2h = n * 8
    # One untimed guess and solve of the first system without a push: the
    # fresh context builds its restart-cycle graph and SELL buffers here, as
    # the timed context did in its warm-up steps; the history is unchanged.
    i0 = steps_e2e[0]
    rp_d.copy_(rp_h, non_blocking=True)
    ci_d.copy_(ci_h, non_blocking=True)
    v_d.copy_(pin[i0][0], non_blocking=True)
    b_d.copy_(pin[i0][1], non_blocking=True)
    A = sa.CSR(rp_d, ci_d, v_d)
    seq.guess(A, b_d, x)
    seq.solve(A, b_d, TOL, x)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    e2e_iters = []
    for i in steps_e2e:
        rp_d.copy_(rp_h, non_blocking=True)
        ci_d.copy_(ci_h, non_blocking=True)
        v_d.copy_(pin[i][0], non_blocking=True)
        b_d.copy_(pin[i][1], non_blocking=True)
        A = sa.CSR(rp_d, ci_d, v_d)
        seq.guess(A, b_d, x)
        e2e_iters.append(seq.solve(A, b_d, TOL, x)["iters"])
        seq.push(x)
        x_h.copy_(x, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), dist, dev)
    e2e_value = whole_job_rate(K, ms_e2e, world)

    # Other forms on the same systems, each with its own priming: the mixed
    # form (FP64 history, sketch and guess, FP32 GMRES(30) inner solves inside
    # FP64 refinement) and right-preconditioned GMRES (damped Jacobi sweeps),
    # all to the same 1e-8 on the FP64 true residual.
    def run_form(label, precision, sweeps, kind="jacobi"):
        nonlocal seq
        seq.close()
        seq = sa.Sequence(n, M_HIST, S_ROWS, zeta=ZETA, seed=SEED, krylov="gmres",
                          restart=RESTART, max_iters=60000, precision=precision,
                          precond_sweeps=sweeps, precond_kind=kind,
                          precond_ratio=args.precond_ratio)
        for i in range(t_first):
            step(i)
        cms, cinfos = timed(timed_steps)
        cst, _ = profiled(prof_steps)
        assert all(inf["status"] == 0 for _, inf in cinfos), "a %s solve did not converge" % label
        croof, ckern = roofline(cst, list(prof_steps), fp64=precision == "f64")
        return {
            "form": label, "value": whole_job_rate(K, cms, world), "unit": "systems/s",
            "ms_per_step": cms / K,
            "dtype": "f32 inner + f64 refinement" if precision != "f64" else "f64",
            "iters_per_system": float(np.mean([inf["iters"] for _, inf in cinfos])),
            "ms_per_krylov_iteration": cms / K / float(np.mean([inf["iters"] for _, inf in cinfos])),
            "refinements_per_system": float(np.mean([inf["refinements"] for _, inf in cinfos])),
            "final_relres_max": max(inf["final_relres"] for _, inf in cinfos),
            "roofline": croof, "kernels": ckern,
            "gpu_launches": sum(g["launches"] + inf["launches"] + 1 for g, inf in cinfos),
        }

    chosen = None
    preconditioned = None
    if not args.no_chosen:
        chosen = run_form("FP64 history/sketch/QR/guess, FP32 GMRES(30)-CGS2 inner solves, FP64 "
                          "iterative refinement of the true residual to rel-res 1e-8",
                          "mixed_krylov", 0)
        chosen["vs_plain_f64"] = chosen["value"] / value
        preconditioned = {
            "f64_jacobi4": run_form("FP64 GMRES(30) right-preconditioned by 4 damped Jacobi "
                                    "sweeps (omega 0.8), rel-res 1e-8", "f64", 4),
            "mixed_jacobi8": run_form("FP32 GMRES(30) inner solves right-preconditioned by 8 "
                                      "damped Jacobi sweeps, FP64 refinement to rel-res 1e-8",
                                      "mixed_krylov", 8),
        }
        preconditioned["f64_cheb4"] = run_form(
            "FP64 GMRES(30) right-preconditioned by the degree-4 Chebyshev polynomial on "
            "[lmax/%g, lmax] of D^-1 A (lmax: Gershgorin), rel-res 1e-8" % args.precond_ratio,
            "f64", 4, "chebyshev")
        preconditioned["mixed_cheb8"] = run_form(
            "FP32 GMRES(30) inner solves right-preconditioned by the degree-8 Chebyshev "
            "polynomial on [lmax/%g, lmax] of D^-1 A, FP64 refinement to rel-res 1e-8"
            % args.precond_ratio, "mixed_krylov", 8, "chebyshev")
        for k, f in preconditioned.items():
            f["vs_plain_f64"] = f["value"] / value
        preconditioned["mixed_jacobi8"]["vs_f64_jacobi4"] = (
            preconditioned["mixed_jacobi8"]["value"] / preconditioned["f64_jacobi4"]["value"])
        preconditioned["mixed_cheb8"]["vs_f64_cheb4"] = (
            preconditioned["mixed_cheb8"]["value"] / preconditioned["f64_cheb4"]["value"])
        preconditioned["note"] = ("precision gain like for like: chosen.vs_plain_f64 (both "
                                  "unpreconditioned), mixed_jacobi8.vs_f64_jacobi4 and "
                                  "mixed_cheb8.vs_f64_cheb4 (both preconditioned, each with its "
                                  "best degree)")
    seq.close()

    batched = None
    if not args.no_batched:
        batched = batched_form(args.batched_steps, 2, hbm_peak)
        # fewer sequences than SMs: the autotuner's cluster schedules spread
        # each sequence over several SMs
        sb = batched_form(args.batched_steps, 2, hbm_peak, count=64, plain_sample=0,
                          one_block_ref=True)
        batched["batch_of_64"] = {k: sb[k] for k in ("form", "value", "unit", "ms_per_step",
                                                      "schedule", "one_block_ms_per_step",
                                                      "iters_mean", "all_converged")}
        batched["batch_of_64"]["frac"] = sb["roofline"]["frac"]

    small = None
    if not args.no_chosen:
        small = spd_small()

    precision = None
    if not args.no_precision:
        precision = precision_startup(hbm_peak)

    learned = None
    if not args.no_learned:
        learned = learned_bounded(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(float(np.mean(iters)))
        ncores = os.cpu_count() or 1
        if cpu.get("value") is not None and ncores > 1:
            allc = run_cpu_baseline(float(np.mean(iters)), threads=ncores)
            cpu["all_cores"] = {k: allc.get(k) for k in ("value", "cores", "sample", "timed_s",
                                                         "extrapolated", "error") if k in allc}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_line(world),
            "timing": ("value: CUDA events around K un-instrumented steps (guess + solve + push); "
                       "roofline and kernel shares: a separate profiled pass of %d further "
                       "steps" % KP),
            "iters_per_system": float(np.mean(iters)),
            # ms_per_step / iters_per_system: restarted GMRES(30) counts move at the
            # rounding level with the order of FP64 sums, the time per iteration does not
            "ms_per_krylov_iteration": ms / K / float(np.mean(iters)),
            "iters_per_system_prev_steps": [inf["iters"] for _, inf in prime[-3:]],
            "guess_relres_mean": float(np.mean([g["guess_relres"] for g, _ in infos])),
            "final_relres_max": worst,
            "roofline": roof, "kernels": kernels, "clocks": clocks,
            "chosen": chosen,
            "preconditioned": preconditioned,
            "spd_4096": small,
            "batched": batched,
            "precision_2048": precision,
            "learned": learned,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "systems/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "systems": "the timed systems replayed from the same history in a fresh "
                               "context (iterations identical: %s)" % (e2e_iters == iters)},
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
