"""Host logic of bench.py that needs no GPU: the DRAM-traffic lookup that
scales the committed ncu ratio, and reports nothing once the kernel source
differs from the one the counters were taken on."""
import hashlib
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PROFILE = os.path.join("profiles", "arnoldi_kernels_nonsym1024.txt")
SOURCE = os.path.join("paper_2309_02156_gb300", "csrc", "krylov_kernels.cuh")


def _ratios(path):
    out = {}
    for line in open(path):
        if line.startswith("traffic_ratio["):
            kind = line[len("traffic_ratio["):line.index("]")]
            out[kind] = float(line.split(":", 1)[1].split()[0])
    return out


def _copy_tree(tmp_path, monkeypatch):
    """The committed summary and kernel source in a scratch root, the summary's
    hash line set to the scratch source's hash."""
    for rel in (PROFILE, SOURCE):
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), tmp_path / rel)
    digest = hashlib.sha256(open(tmp_path / SOURCE, "rb").read()).hexdigest()[:16]
    lines = open(tmp_path / PROFILE).read().splitlines(keepends=True)
    with open(tmp_path / PROFILE, "w") as f:
        for line in lines:
            f.write(f"source_sha256_16: {digest}\n" if line.startswith("source_sha256_16:") else line)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))


def test_traffic_scales_the_recorded_ratio(tmp_path, monkeypatch):
    """Every kernel kind the summary lists resolves to its ratio x the launch's
    algorithmic bytes; an unlisted kind resolves to nothing."""
    _copy_tree(tmp_path, monkeypatch)
    ratios = _ratios(tmp_path / PROFILE)
    assert set(ratios) >= {"spmv", "cgs_dot", "cgs_pass2", "cgs_pass3"}
    for kind, r in ratios.items():
        assert 0.5 < r < 1.5
        assert bench.profile_traffic(kind, 2.0e6) == pytest.approx(r * 2.0e6)
    assert bench.profile_traffic("no_such_kernel", 2.0e6) is None


def test_traffic_is_null_once_the_source_changes(tmp_path, monkeypatch):
    _copy_tree(tmp_path, monkeypatch)
    assert bench.profile_traffic("cgs_pass2", 1.0e6) is not None
    with open(tmp_path / SOURCE, "a") as f:
        f.write("\n// edited\n")
    assert bench.profile_traffic("cgs_pass2", 1.0e6) is None
    os.remove(tmp_path / PROFILE)
    assert bench.profile_traffic("cgs_pass2", 1.0e6) is None


def test_each_precision_reads_its_own_summary(tmp_path, monkeypatch):
    """FP64 kernels, FP32 Arnoldi kernels and FP32 preconditioner sweeps each
    take their ratio from their own summary, keyed to the hash of the sources
    that summary names; a change in any one of those sources voids it."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2309_02156_gb300" / "csrc"
    os.makedirs(csrc)
    os.makedirs(tmp_path / "profiles")
    names = {n for _, srcs in bench.TRAFFIC_PROFILES.values() for n in srcs}
    for n in names:
        (csrc / n).write_text(f"// {n}\n")
    ratio = {"f64": 0.91, "f32": 1.07, "f32_precond": 0.83}
    for key, (name, srcs) in bench.TRAFFIC_PROFILES.items():
        kind = "precond" if key == "f32_precond" else "spmv"
        (tmp_path / "profiles" / name).write_text(
            f"source_sha256_16: {bench.sources_digest(srcs)}\n"
            f"traffic_ratio[{kind}]: {ratio[key]} (test)\n")
    assert bench.profile_traffic("spmv", 1e6, "f64") == pytest.approx(0.91e6)
    assert bench.profile_traffic("spmv", 1e6, "f32") == pytest.approx(1.07e6)
    assert bench.profile_traffic("precond", 1e6, "f32") == pytest.approx(0.83e6)
    assert bench.profile_traffic("precond", 1e6, "f64") is None
    srcs = bench.TRAFFIC_PROFILES["f32_precond"][1]
    with open(csrc / srcs[-1], "a") as f:
        f.write("// edited\n")
    assert bench.profile_traffic("precond", 1e6, "f32") is None


def _run_reference(env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_line_with_the_contract_keys():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the main line's metric and unit, its own cpu_baseline and
    an e2e object without host-device traffic."""
    (line,) = _run_reference({"RANK": "0"})
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "systems/s"
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "systems/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # Same workload description as the GPU arm; the timed sample is what
    # steps and ms_per_step describe, the extrapolation is a field of its own.
    assert line["config"] == bench.config_line(1)
    ex = line["extrapolated"]
    assert ex["timed_iterations_per_step"] == 30 and ex["iterations_per_system"] > 30
    per = ex["guess_s"] + ex["iterations_per_system"] * ex["iteration_s"]
    assert line["value"] == pytest.approx(1.0 / per, rel=1e-9)
    assert 1e3 * (ex["guess_s"] + 30 * ex["iteration_s"]) <= 1.5 * line["ms_per_step"]


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_reference({"RANK": "1"}) == []
