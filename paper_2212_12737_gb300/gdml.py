"""Python binding of libgdml (C ABI in include/gdml.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch only provides device
memory (tensors) and the CUDA stream.  Importing this module does not load
the library; the first call does, and raises if it was not built or no CUDA
device is present -- there is no CPU fallback.

Function names follow the C ABI: kernel_setup, matvec, precond_build,
precond_apply, pcg_solve (plus matvec_fp64, precond_info, destroy).
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libgdml.so")
_lib = None

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_SPD", 5: "ERR_BREAKDOWN",
          6: "ERR_NOT_CONVERGED", 7: "ERR_TIMEOUT", 8: "ERR_STATE"}
PRECISION = {"fp64": 0, "tf32": 1, "bf16": 2}
SELECT = {"uniform": 0, "rls": 1, "pivchol": 2}

EXPORTS = ["gdml_kernel_setup", "gdml_matvec", "gdml_matvec_fp64", "gdml_precond_build", "gdml_precond_info",
           "gdml_precond_apply", "gdml_pcg_solve", "gdml_set_inner_rtol", "gdml_last_outer_steps",
           "gdml_last_error", "gdml_destroy", "gdml_test_tc_gemm", "gdml_tc_check",
           "gdml_launch_count", "gdml_matvec_noalloc"]


class GdmlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


def library_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load libgdml.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libgdml.so not built ({_LIB_PATH}); run paper_2212_12737_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I64, I32, D, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
    sig = {
        "gdml_kernel_setup": [ctypes.POINTER(P), P, I64, I32, D, D, I32, P],
        "gdml_matvec": [P, P, P, I32],
        "gdml_matvec_fp64": [P, P, P, I32],
        "gdml_precond_build": [P, I32, I64, U64, P, P],
        "gdml_precond_info": [P, ctypes.POINTER(I64), ctypes.POINTER(D)],
        "gdml_precond_apply": [P, P, P],
        "gdml_pcg_solve": [P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D)],
        "gdml_set_inner_rtol": [P, D],
        "gdml_last_outer_steps": [P, ctypes.POINTER(I32)],
        "gdml_last_error": [P],
        "gdml_destroy": [P],
        "gdml_test_tc_gemm": [I32, P, P, I32, I32, I32, P, P],
        "gdml_tc_check": [P],
        "gdml_launch_count": [],
        "gdml_matvec_noalloc": [P, I64, I32, D, D, P, P, I32, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.gdml_last_error.restype = ctypes.c_char_p
    lib.gdml_destroy.restype = None
    lib.gdml_launch_count.restype = ctypes.c_int64
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One kernel system (Sec. 2.1, Eq. 1) living on the current CUDA device."""

    def __init__(self, R: torch.Tensor, sigma: float, lam: float, precision: str = "fp64", stream=None):
        lib = load()
        if R.dtype != torch.float64 or R.dim() != 3 or R.shape[2] != 3:
            raise ValueError("R must be a float64 CUDA tensor of shape (M, N, 3)")
        R = R.contiguous()
        self.M, self.N = int(R.shape[0]), int(R.shape[1])
        self.n = 3 * self.M * self.N
        self.device = R.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(R.device)
        h = ctypes.c_void_p()
        st = lib.gdml_kernel_setup(ctypes.byref(h), _ptr(R), self.M, self.N, float(sigma), float(lam),
                                   PRECISION[precision], ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise GdmlError(st, lib.gdml_last_error(None).decode())
        self._h = h
        self.precision = precision

    def _check(self, st: int):
        if st != 0:
            raise GdmlError(st, load().gdml_last_error(self._h).decode())

    def _vec(self, out):
        return torch.empty(self.n, dtype=torch.float64, device=self.device) if out is None else out

    def matvec(self, v: torch.Tensor, out: torch.Tensor | None = None, add_lambda: bool = True) -> torch.Tensor:
        out = self._vec(out)
        self._check(load().gdml_matvec(self._h, _ptr(v), _ptr(out), int(add_lambda)))
        return out

    def matvec_fp64(self, v: torch.Tensor, out: torch.Tensor | None = None, add_lambda: bool = True) -> torch.Tensor:
        out = self._vec(out)
        self._check(load().gdml_matvec_fp64(self._h, _ptr(v), _ptr(out), int(add_lambda)))
        return out

    def precond_build(self, method: str, k: int, seed: int = 2, pivots: bool = False, trace: bool = False):
        piv = torch.empty(k, dtype=torch.int64, device=self.device) if pivots else None
        tr = torch.empty(k, dtype=torch.float64, device=self.device) if trace else None
        self._check(load().gdml_precond_build(self._h, SELECT[method], int(k), int(seed), _ptr(piv), _ptr(tr)))
        return piv, tr

    def precond_info(self):
        r = ctypes.c_int64()
        j = ctypes.c_double()
        self._check(load().gdml_precond_info(self._h, ctypes.byref(r), ctypes.byref(j)))
        return int(r.value), float(j.value)

    def precond_apply(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._vec(out)
        self._check(load().gdml_precond_apply(self._h, _ptr(r), _ptr(out)))
        return out

    def set_inner_rtol(self, v: float):
        self._check(load().gdml_set_inner_rtol(self._h, float(v)))

    def pcg_solve(self, y: torch.Tensor, alpha: torch.Tensor | None = None, rtol: float = 1e-8,
                  max_iter: int = 20000, raise_on_nonconvergence: bool = True):
        """Returns (alpha, iterations, true relative residual, outer refinement steps)."""
        if alpha is None:
            alpha = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        it = ctypes.c_int32()
        rel = ctypes.c_double()
        st = load().gdml_pcg_solve(self._h, _ptr(y), _ptr(alpha), float(rtol), int(max_iter), ctypes.byref(it),
                                   ctypes.byref(rel))
        outer = ctypes.c_int32()
        load().gdml_last_outer_steps(self._h, ctypes.byref(outer))
        if st != 0 and (raise_on_nonconvergence or st != 6):
            self._check(st)
        return alpha, int(it.value), float(rel.value), int(outer.value)

    def tc_check(self):
        """Raise if a tensor-core pipeline wait timed out since the last check."""
        self._check(load().gdml_tc_check(self._h))

    def destroy(self):
        if getattr(self, "_h", None):
            load().gdml_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def kernel_setup(R, sigma, lam, precision="fp64", stream=None) -> Context:
    return Context(R, sigma, lam, precision, stream)


def matvec(ctx: Context, v, out=None, add_lambda=True):
    return ctx.matvec(v, out, add_lambda)


def precond_build(ctx: Context, method, k, seed=2, pivots=False, trace=False):
    return ctx.precond_build(method, k, seed, pivots, trace)


def precond_apply(ctx: Context, r, out=None):
    return ctx.precond_apply(r, out)


def pcg_solve(ctx: Context, y, alpha=None, rtol=1e-8, max_iter=20000):
    return ctx.pcg_solve(y, alpha, rtol, max_iter)


def test_tc_gemm(A: torch.Tensor, B: torch.Tensor, bf16: bool = False) -> torch.Tensor:
    """C = A B^T on the tcgen05 tensor cores (operands rounded to TF32 or BF16, FP32 accumulation)."""
    lib = load()
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty(M, N, dtype=torch.float64, device=A.device)
    st = lib.gdml_test_tc_gemm(int(bf16), _ptr(A), _ptr(B), M, N, K, _ptr(C),
                               ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return C


def launch_count() -> int:
    """Kernel launches executed by the library so far (graph replays included)."""
    return int(load().gdml_launch_count())


def matvec_noalloc(R: torch.Tensor, sigma: float, lam: float, v: torch.Tensor, out: torch.Tensor | None = None,
                   add_lambda: bool = True) -> torch.Tensor:
    """K v (+ lam v) with no context and no device allocation inside the library
    (M <= 128 geometries, N <= 24 atoms; scratch is a static device array)."""
    lib = load()
    if R.dtype != torch.float64 or R.dim() != 3 or R.shape[2] != 3:
        raise ValueError("R must be a float64 CUDA tensor of shape (M, N, 3)")
    if out is None:
        out = torch.empty_like(v)
    st = lib.gdml_matvec_noalloc(_ptr(R.contiguous()), int(R.shape[0]), int(R.shape[1]), float(sigma), float(lam),
                                 _ptr(v), _ptr(out), int(add_lambda),
                                 ctypes.c_void_p(torch.cuda.current_stream(R.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return out
