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
