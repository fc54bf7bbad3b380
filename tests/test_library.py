"""The C-ABI library builds, loads and exports every declared entry point (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(seq_\w+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = set(_declared())
    for required in ("seq_create", "seq_destroy", "seq_push_solution", "seq_guess", "seq_solve"):
        assert required in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_02156_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def _cc(compiler):
    import shutil
    path = shutil.which(compiler)
    if not path:
        pytest.skip(f"{compiler} not available")
    return path


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_is_plain_c_and_cpp(compiler, std, tmp_path):
    """include/seqaccel.h compiles warning-free as C99 and as C++17 (so the
    boundary is usable without the Python binding)."""
    import subprocess
    src = tmp_path / ("use.c" if compiler == "gcc" else "use.cpp")
    src.write_text('#include "seqaccel.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([_cc(compiler), std, "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_every_entry_point(tmp_path):
    """A C program that takes the address of every declared entry point links
    against the library (unmangled C symbols)."""
    import subprocess
    if not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_02156_gb300 import build
    lib = build.build()
    names = sorted(set(_declared()))
    body = "\n".join(f"    (void)(uintptr_t)&{n};" for n in names)
    src = tmp_path / "link.c"
    src.write_text('#include <stdint.h>\n#include "seqaccel.h"\nint main(void) {\n'
                   + body + "\n    return 0;\n}\n")
    out = tmp_path / "link"
    r = subprocess.run([_cc("gcc"), "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(out), lib, "-Wl,--unresolved-symbols=ignore-in-shared-libs"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_create_rejects_bad_config_without_gpu_work():
    """Argument validation happens on the host before any device call."""
    if not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2309_02156_gb300._binding as b
    lib = b.load()
    h = ctypes.c_void_p()
    bad = [b._Config(0, 10, 40, 8, 1, 0, 2, 1, 30, 100, 0, 0),     # n = 0
           b._Config(100, 10, 10, 8, 1, 0, 2, 1, 30, 100, 0, 0),   # s < M + 1
           b._Config(100, 40, 80, 8, 1, 0, 2, 1, 30, 100, 0, 0),   # M > 31
           b._Config(100, 10, 40, 8, 1, 0, 2, 1, 99, 100, 0, 0),   # restart > 64
           b._Config(100, 10, 40, 41, 1, 0, 2, 1, 30, 100, 0, 0)]  # zeta > s
    for cfg in bad:
        assert lib.seq_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
        assert not h.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library the package raises."""
    import paper_2309_02156_gb300._binding as b
    monkeypatch.setattr(b, "_LIB", None)
    monkeypatch.setattr(b._build, "LIB", str(tmp_path / "missing" / "libseqaccel.so"))
    with pytest.raises(RuntimeError, match="not built"):
        b.load(build_if_needed=False)


def test_device_pointers_are_required():
    """The binding passes device pointers only: a host tensor is rejected
    before any call crosses the boundary."""
    import torch
    import paper_2309_02156_gb300._binding as b
    with pytest.raises((ValueError, TypeError, RuntimeError)):
        b._ptr(torch.zeros(4, dtype=torch.float64), torch.float64, 4)
