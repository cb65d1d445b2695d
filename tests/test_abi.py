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


def test_symmetry_groups_are_checked_on_the_host(lib_path):
    """gdml_kernel_setup_sym rejects permutation sets that are not a group before any device work
    (no GPU needed): not a permutation, identity missing, not closed, repeated rows, S out of range."""
    try:
        lib = ctypes.CDLL(lib_path)
    except OSError as e:
        pytest.skip(f"cannot dlopen: {e}")
    import numpy as np
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    fn = lib.gdml_kernel_setup_sym
    fn.argtypes = [ctypes.POINTER(P), P, I64, I32, P, I32, D, D, I32, P]
    fn.restype = ctypes.c_int
    lib.gdml_last_error.restype = ctypes.c_char_p
    lib.gdml_last_error.argtypes = [P]
    fake_R = ctypes.c_void_p(0x1000)  # never dereferenced: the group is checked first
    idn = list(range(5))
    cases = {
        "not a permutation": [idn, [0, 0, 2, 3, 4]],
        "identity": [[1, 0, 2, 3, 4]],
        "closed under composition": [idn, [1, 2, 0, 3, 4]],
        "twice": [idn, idn],
    }
    for word, perms in cases.items():
        arr = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
        h = ctypes.c_void_p()
        st = fn(ctypes.byref(h), fake_R, 3, 5, arr.ctypes.data_as(ctypes.c_void_p), arr.shape[0], 1.0, 1e-6, 0, None)
        assert st == 1 and not h.value, word
        assert word in lib.gdml_last_error(None).decode(), (word, lib.gdml_last_error(None))
    arr = np.ascontiguousarray(np.asarray([idn, [1, 0, 2, 3, 4]], dtype=np.int32))
    h = ctypes.c_void_p()
    for prec in (1, 2, 3):  # TF32, BF16, DF64 do not take symmetries
        assert fn(ctypes.byref(h), fake_R, 3, 5, arr.ctypes.data_as(ctypes.c_void_p), 2, 1.0, 1e-6, prec, None) == 1
    assert fn(ctypes.byref(h), fake_R, 3, 5, None, 2, 1.0, 1e-6, 0, None) == 1
