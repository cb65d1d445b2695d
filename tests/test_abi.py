"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/gdml.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_symbols():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gdml_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2212_12737_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_paper_entry_points():
    syms = declared_symbols()
    for name in ("gdml_kernel_setup", "gdml_matvec", "gdml_precond_build", "gdml_precond_apply", "gdml_pcg_solve"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(gdml_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_and_binding_knows_every_symbol(lib_path):
    try:
        lib = ctypes.CDLL(lib_path)
    except OSError as e:  # no CUDA runtime on this machine
        pytest.skip(f"cannot dlopen: {e}")
    for s in declared_symbols():
        assert hasattr(lib, s)
    from paper_2212_12737_gb300 import gdml
    assert sorted(gdml.EXPORTS) == declared_symbols()


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the shared library absent, the first call raises."""
    from paper_2212_12737_gb300 import gdml
    monkeypatch.setattr(gdml, "_lib", None)
    monkeypatch.setattr(gdml, "_LIB_PATH", str(tmp_path / "libgdml.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gdml.load()
    with pytest.raises(RuntimeError, match="not built"):
        gdml.rule_of_thumb_k(1000)


def test_plain_c_program_uses_the_abi(lib_path, tmp_path):
    """The headers compile as C99 and a C program links against the library and calls a
    host-only entry point (the rule of thumb: 5833 columns for n = 63000, m = 1, k_min = 100)."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <stdio.h>\n#include "gdml.h"\n#include "gdml_testing.h"\n'
        "int main(void) {\n"
        "  int64_t k = 0;\n"
        "  if (gdml_rule_of_thumb_k(63000, 1.0, 100.0, &k) != GDML_OK) return 1;\n"
        "  if (gdml_rule_of_thumb_k(0, 1.0, 100.0, &k) != GDML_ERR_ARG) return 2;\n"
        '  printf("%lld %s\\n", (long long)k, gdml_last_error(NULL));\n'
        "  return 0;\n}\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib_path)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lgdml",
                    f"-Wl,-rpath,{libdir}"], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    if out.returncode != 0 and "error while loading shared libraries" in out.stderr:
        pytest.skip(f"cannot load the CUDA runtime: {out.stderr.strip()}")
    assert out.returncode == 0, out.stderr
    k, msg = out.stdout.split(" ", 1)
    assert int(k) == 5833 and "rule_of_thumb_k" in msg


def test_binding_rejects_vectors_the_library_would_overrun():
    """The library reads / writes exactly n doubles at each vector's address, so the binding
    refuses anything that is not a contiguous float64 vector of n elements on the right device."""
    import torch
    from paper_2212_12737_gb300 import gdml
    cpu = torch.device("cpu")
    ok = torch.zeros(6, dtype=torch.float64)
    assert gdml._vec_arg(ok, 6, cpu, "v") is ok
    with pytest.raises(ValueError, match="float64"):
        gdml._vec_arg(torch.zeros(6, dtype=torch.float32), 6, cpu, "v")
    with pytest.raises(ValueError, match="6 elements"):
        gdml._vec_arg(torch.zeros(5, dtype=torch.float64), 6, cpu, "v")
    with pytest.raises(ValueError, match="must be on"):
        gdml._vec_arg(torch.zeros(6, dtype=torch.float64, device="meta"), 6, cpu, "v")
    with pytest.raises(ValueError, match="contiguous"):
        gdml._vec_arg(torch.zeros(12, dtype=torch.float64)[::2], 6, cpu, "v")
    with pytest.raises(TypeError):
        gdml._vec_arg([0.0] * 6, 6, cpu, "v")
