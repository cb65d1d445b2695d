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
PRECISION = {"fp64": 0, "tf32": 1, "bf16": 2, "df64": 3, "ozaki": 4}
SELECT = {"uniform": 0, "rls": 1, "pivchol": 2, "weighted": 3, "svd": 4}

EXPORTS = ["gdml_kernel_setup", "gdml_kernel_setup_sym", "gdml_matvec", "gdml_matvec_fp64", "gdml_precond_build", "gdml_precond_info",
           "gdml_precond_apply", "gdml_pcg_solve", "gdml_set_inner_rtol", "gdml_last_outer_steps",
           "gdml_last_error", "gdml_destroy", "gdml_test_tc_gemm", "gdml_test_oz_gemm", "gdml_test_df_passes", "gdml_test_oz_gemm_tall", "gdml_test_precond_factor", "gdml_test_set_wait_limit",
           "gdml_test_cholesky_jitter", "gdml_test_set_lambda", "gdml_tc_check",
           "gdml_launch_count", "gdml_matvec_noalloc", "gdml_pcg_solve_batched", "gdml_autotune",
           "gdml_set_tuning", "gdml_precond_build_scored", "gdml_rls_scores", "gdml_descriptors",
           "gdml_scorer_create", "gdml_scorer_fit_scaling", "gdml_scorer_train", "gdml_scorer_predict",
           "gdml_scorer_params", "gdml_scorer_grad", "gdml_scorer_destroy", "gdml_rule_of_thumb_k",
           "gdml_predict_forces", "gdml_pcg_spectrum", "gdml_set_inner_levels", "gdml_rls_labels"]

# Table 1 (Sec. 4.3): molecule -> (m, k_min) of the rule of thumb, fitted at n = 31k;
# "default" is the row for molecules without fitted parameters.
ROT_PARAMS = {"default": (1.0, 100.0), "ethanol": (0.87, 10.0), "uracil": (1.07, 32.0), "toluene": (1.01, 44.0),
              "aspirin": (1.14, 236.0), "azobenzene": (1.02, 62.0), "catcher": (1.02, 316.0),
              "nanotube": (0.73, 89.0)}


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
        "gdml_kernel_setup_sym": [ctypes.POINTER(P), P, I64, I32, P, I32, D, D, I32, P],
        "gdml_matvec": [P, P, P, I32],
        "gdml_matvec_fp64": [P, P, P, I32],
        "gdml_precond_build": [P, I32, I64, U64, P, P],
        "gdml_precond_info": [P, ctypes.POINTER(I64), ctypes.POINTER(D)],
        "gdml_precond_apply": [P, P, P],
        "gdml_pcg_solve": [P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D)],
        "gdml_set_inner_rtol": [P, D],
        "gdml_set_inner_levels": [P, I32],
        "gdml_rls_labels": [P, I32, I64, U64, P],
        "gdml_last_outer_steps": [P, ctypes.POINTER(I32)],
        "gdml_last_error": [P],
        "gdml_destroy": [P],
        "gdml_test_tc_gemm": [I32, P, P, I32, I32, I32, P, P],
        "gdml_test_oz_gemm": [P, P, I64, I64, I64, I32, I32, P, P],
        "gdml_test_df_passes": [P, I64, I64, P, P, D, I32, P, P, P],
        "gdml_test_oz_gemm_tall": [P, I64, I64, P, I64, I64, I32, I32, P, P, P],
        "gdml_test_precond_factor": [P, P],
        "gdml_test_set_wait_limit": [ctypes.c_uint32],
        "gdml_test_cholesky_jitter": [P, I64, P, ctypes.POINTER(D), P],
        "gdml_test_set_lambda": [P, D],
        "gdml_tc_check": [P],
        "gdml_launch_count": [],
        "gdml_matvec_noalloc": [P, I64, I32, D, D, P, P, I32, P],
        "gdml_pcg_solve_batched": [P, I32, P, P, D, I32, P, P],
        "gdml_autotune": [P, ctypes.POINTER(I32)],
        "gdml_set_tuning": [P, I32],
        "gdml_precond_build_scored": [P, P, I64, U64, P],
        "gdml_rls_scores": [P, I64, U64, P],
        "gdml_descriptors": [P, P],
        "gdml_scorer_create": [ctypes.POINTER(P), I32, I32, U64, P],
        "gdml_scorer_fit_scaling": [P, P, P, I64],
        "gdml_scorer_train": [P, P, P, I64, I32, I32, D, ctypes.POINTER(D)],
        "gdml_scorer_predict": [P, P, I64, P],
        "gdml_scorer_params": [P, P, I32, ctypes.POINTER(I64)],
        "gdml_scorer_grad": [P, P, P, I64, ctypes.POINTER(D), P],
        "gdml_scorer_destroy": [P],
        "gdml_rule_of_thumb_k": [I64, D, D, ctypes.POINTER(I64)],
        "gdml_predict_forces": [P, P, I64, P, P],
        "gdml_pcg_spectrum": [P, I32, P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.gdml_last_error.restype = ctypes.c_char_p
    lib.gdml_destroy.restype = None
    lib.gdml_scorer_destroy.restype = None
    lib.gdml_launch_count.restype = ctypes.c_int64
    _lib = lib
    return lib


def rule_of_thumb_k(n: int, molecule: str = "default", m: float | None = None, k_min: float | None = None) -> int:
    """Inducing-column count for precond_build by the rule of thumb (Sec. 4.3, Eqs. 7-8):
    Table 1's (m, k_min) for ``molecule``, either overridden by ``m`` / ``k_min``."""
    lib = load()
    m0, k0 = ROT_PARAMS[molecule]
    out = ctypes.c_int64()
    st = lib.gdml_rule_of_thumb_k(int(n), float(m0 if m is None else m), float(k0 if k_min is None else k_min),
                                  ctypes.byref(out))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return out.value


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _vec_arg(t: torch.Tensor, n: int, device: torch.device, name: str) -> torch.Tensor:
    """A float64 vector of n elements on `device`, contiguous: the library reads or writes
    exactly n doubles at its address, so anything else is rejected here."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{name} must hold {n} elements, got {t.numel()}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Context:
    """One kernel system (Sec. 2.1, Eq. 1) living on the current CUDA device."""

    def __init__(self, R: torch.Tensor, sigma: float, lam: float, precision: str = "fp64", stream=None,
                 perms=None):
        lib = load()
        if R.dtype != torch.float64 or R.dim() != 3 or R.shape[2] != 3:
            raise ValueError("R must be a float64 CUDA tensor of shape (M, N, 3)")
        R = R.contiguous()
        self.M, self.N = int(R.shape[0]), int(R.shape[1])
        self.n = 3 * self.M * self.N
        self.device = R.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(R.device)
        h = ctypes.c_void_p()
        if perms is None:
            st = lib.gdml_kernel_setup(ctypes.byref(h), _ptr(R), self.M, self.N, float(sigma), float(lam),
                                       PRECISION[precision], ctypes.c_void_p(self.stream.cuda_stream))
        else:  # permutational symmetries: S x N atom permutations forming a group
            import numpy as np
            P = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
            if P.ndim != 2 or P.shape[1] != self.N:
                raise ValueError(f"perms must have shape (S, {self.N})")
            st = lib.gdml_kernel_setup_sym(ctypes.byref(h), _ptr(R), self.M, self.N,
                                           P.ctypes.data_as(ctypes.c_void_p), int(P.shape[0]), float(sigma),
                                           float(lam), PRECISION[precision],
                                           ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise GdmlError(st, lib.gdml_last_error(None).decode())
        self._h = h
        self.precision = precision

    def _check(self, st: int):
        if st != 0:
            raise GdmlError(st, load().gdml_last_error(self._h).decode())

    def _vec(self, out):
        if out is None:
            return torch.empty(self.n, dtype=torch.float64, device=self.device)
        return _vec_arg(out, self.n, self.device, "out")

    def matvec(self, v: torch.Tensor, out: torch.Tensor | None = None, add_lambda: bool = True) -> torch.Tensor:
        _vec_arg(v, self.n, self.device, "v")
        out = self._vec(out)
        self._check(load().gdml_matvec(self._h, _ptr(v), _ptr(out), int(add_lambda)))
        return out

    def matvec_fp64(self, v: torch.Tensor, out: torch.Tensor | None = None, add_lambda: bool = True) -> torch.Tensor:
        _vec_arg(v, self.n, self.device, "v")
        out = self._vec(out)
        self._check(load().gdml_matvec_fp64(self._h, _ptr(v), _ptr(out), int(add_lambda)))
        return out

    def predict_forces(self, R_query: torch.Tensor, alpha: torch.Tensor,
                       out: torch.Tensor | None = None) -> torch.Tensor:
        """Forces (Q, N, 3) the model with coefficients alpha predicts for query geometries (Q, N, 3)."""
        if R_query.dtype != torch.float64 or R_query.dim() != 3 or tuple(R_query.shape[1:]) != (self.N, 3):
            raise ValueError(f"R_query must be a float64 CUDA tensor of shape (Q, {self.N}, 3)")
        if alpha.dtype != torch.float64 or alpha.numel() != self.n:
            raise ValueError(f"alpha must be {self.n} float64 values")
        R_query = R_query.contiguous()
        Q = int(R_query.shape[0])
        out = torch.empty((Q, self.N, 3), dtype=torch.float64, device=self.device) if out is None else out
        self._check(load().gdml_predict_forces(self._h, _ptr(R_query), Q, _ptr(alpha), _ptr(out)))
        return out

    def precond_build(self, method: str, k: int, seed: int = 2, pivots: bool = False, trace: bool = False):
        piv = torch.empty(k, dtype=torch.int64, device=self.device) if pivots else None
        tr = torch.empty(k, dtype=torch.float64, device=self.device) if trace else None
        self._check(load().gdml_precond_build(self._h, SELECT[method], int(k), int(seed), _ptr(piv), _ptr(tr)))
        return piv, tr

    def precond_build_scored(self, geometry_scores: torch.Tensor, k: int, seed: int = 2, pivots: bool = False):
        piv = torch.empty(k, dtype=torch.int64, device=self.device) if pivots else None
        self._check(load().gdml_precond_build_scored(self._h, _ptr(geometry_scores.contiguous()), int(k), int(seed),
                                                     _ptr(piv)))
        return piv

    def rls_scores(self, k: int, seed: int = 2) -> torch.Tensor:
        tau = torch.empty(self.n, dtype=torch.float64, device=self.device)
        self._check(load().gdml_rls_scores(self._h, int(k), int(seed), _ptr(tau)))
        return tau

    def descriptors(self) -> torch.Tensor:
        X = torch.empty(self.M, self.N * (self.N - 1) // 2, dtype=torch.float64, device=self.device)
        self._check(load().gdml_descriptors(self._h, _ptr(X)))
        return X

    def precond_info(self):
        r = ctypes.c_int64()
        j = ctypes.c_double()
        self._check(load().gdml_precond_info(self._h, ctypes.byref(r), ctypes.byref(j)))
        return int(r.value), float(j.value)

    def precond_apply(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        _vec_arg(r, self.n, self.device, "r")
        out = self._vec(out)
        self._check(load().gdml_precond_apply(self._h, _ptr(r), _ptr(out)))
        return out

    def precond_factor(self) -> torch.Tensor:
        """The built preconditioner's factor L_k (n x rank) as FP64 (test hook)."""
        rank, _ = self.precond_info()
        out = torch.empty(rank, self.n, dtype=torch.float64, device=self.device)
        self._check(load().gdml_test_precond_factor(self._h, _ptr(out)))
        return out.t()

    def test_set_lambda(self, lam: float):
        """Replace lambda (test hook; lam <= 0 makes K + lam I indefinite); drops the preconditioner."""
        self._check(load().gdml_test_set_lambda(self._h, float(lam)))

    def set_inner_levels(self, levels: int):
        """OZAKI contexts: slice levels (1..7) of the matvec inside the PCG loop."""
        self._check(load().gdml_set_inner_levels(self._h, int(levels)))

    def set_inner_rtol(self, v: float):
        self._check(load().gdml_set_inner_rtol(self._h, float(v)))

    def pcg_solve(self, y: torch.Tensor, alpha: torch.Tensor | None = None, rtol: float = 1e-8,
                  max_iter: int = 20000, raise_on_nonconvergence: bool = True):
        """Returns (alpha, iterations, true relative residual, outer refinement steps)."""
        _vec_arg(y, self.n, self.device, "y")
        if alpha is None:
            alpha = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        _vec_arg(alpha, self.n, self.device, "alpha")
        it = ctypes.c_int32()
        rel = ctypes.c_double()
        st = load().gdml_pcg_solve(self._h, _ptr(y), _ptr(alpha), float(rtol), int(max_iter), ctypes.byref(it),
                                   ctypes.byref(rel))
        outer = ctypes.c_int32()
        load().gdml_last_outer_steps(self._h, ctypes.byref(outer))
        if st != 0 and (raise_on_nonconvergence or st != 6):
            self._check(st)
        return alpha, int(it.value), float(rel.value), int(outer.value)

    def pcg_spectrum(self, count: int = 0):
        """Ritz values of the last solve's first CG run (the Lanczos matrix of P^-1 K_lambda):
        (theta_min, theta_max, steps, the `count` largest in descending order as a NumPy array)."""
        import numpy as np
        top = np.full(max(int(count), 0), np.nan)
        tmin, tmax, steps = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        ptr = top.ctypes.data_as(ctypes.c_void_p) if count > 0 else None
        self._check(load().gdml_pcg_spectrum(self._h, int(count), ptr, ctypes.byref(tmin), ctypes.byref(tmax),
                                             ctypes.byref(steps)))
        return float(tmin.value), float(tmax.value), int(steps.value), top

    def autotune(self, cache: str | None = None) -> int:
        """Time the matvec's tunable tile parameters for this context's shapes and keep the
        fastest (FP64 / TF32 / BF16: the K-split of the second contraction; OZAKI: the K chunks
        each CTA of the sliced GEMMs accumulates); with a cache file, reuse / record the choice."""
        import json
        key = f"M{self.M}_N{self.N}_{self.precision}"
        table = {}
        if cache and os.path.exists(cache):
            try:
                table = json.load(open(cache))
            except ValueError:
                table = {}
        if key in table:
            self._check(load().gdml_set_tuning(self._h, int(table[key])))
            return int(table[key])
        ch = ctypes.c_int32()
        self._check(load().gdml_autotune(self._h, ctypes.byref(ch)))
        if cache:
            table[key] = int(ch.value)
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return int(ch.value)

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


def kernel_setup(R, sigma, lam, precision="fp64", stream=None, perms=None) -> Context:
    """A context for one kernel system; perms (S x N atom permutations forming a group) selects
    the symmetric (sGDML) kernel."""
    return Context(R, sigma, lam, precision, stream, perms)


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


def test_oz_gemm(A: torch.Tensor, B: torch.Tensor, chunks_per_cta: int = 0, levels: int = 7) -> torch.Tensor:
    """C = A B^T through the sliced-BF16 tensor-core GEMM (FP64-class accuracy); chunks_per_cta
    256-entry K chunks accumulated per CTA (0: automatic); levels < 7 keeps the slice pairs
    i + j < levels only."""
    lib = load()
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty(M, N, dtype=torch.float64, device=A.device)
    st = lib.gdml_test_oz_gemm(_ptr(A), _ptr(B), M, N, K, int(chunks_per_cta), int(levels), _ptr(C),
                               ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return C


def test_oz_gemm_tall(A: torch.Tensor, B: torch.Tensor, tri_b: bool = False, rowsq: bool = False):
    """The OZAKI build's tall sliced GEMM: C = A B^T with A (n x K) and B (NB x K) FP64 (B lower
    triangular when tri_b).  Returns C (n x NB) and its FP32 copy, or the row square sums of C
    (n,) when rowsq."""
    lib = load()
    n, K = A.shape
    NB = B.shape[0]
    Ac = A.t().contiguous()  # column j at offset j n
    B = B.contiguous()
    if rowsq:
        out = torch.empty(n, dtype=torch.float64, device=A.device)
        out32 = None
    else:
        out = torch.empty(NB, n, dtype=torch.float64, device=A.device)
        out32 = torch.empty(NB, n, dtype=torch.float32, device=A.device)
    st = lib.gdml_test_oz_gemm_tall(_ptr(Ac), n, K, _ptr(B), NB, K, int(tri_b), int(rowsq), _ptr(out), _ptr(out32),
                                    ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return out if rowsq else (out.t(), out32.t())


def test_df_passes(L: torch.Tensor, r: torch.Tensor, u: torch.Tensor, lam: float, staged=True):
    """The two passes over the FP32 factor of the DF64/OZAKI Woodbury apply:
    returns (t, z) with t = L^T r and z = (r - L u) / lam.  L: n x k FP32 (its columns
    are stored contiguously, i.e. L.t().contiguous() is passed), r: n, u: k FP64.
    staged: True (TMA-staged, automatic chunk size), 128 or 256 (that chunk size),
    False (register-streamed)."""
    lib = load()
    n, k = L.shape
    Lc = L.t().contiguous()  # column j at offset j n
    r = r.contiguous()
    u = u.contiguous()
    t = torch.empty(k, dtype=torch.float64, device=L.device)
    z = torch.empty(n, dtype=torch.float64, device=L.device)
    mode = int(staged) if not isinstance(staged, bool) else int(staged)
    st = lib.gdml_test_df_passes(_ptr(Lc), n, k, _ptr(r), _ptr(u), float(lam), mode, _ptr(t), _ptr(z),
                                 ctypes.c_void_p(torch.cuda.current_stream(L.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return t, z


def test_set_wait_limit(polls: int | None):
    """Every bounded device wait gives up after `polls` polls (0: at once); None restores the default."""
    lib = load()
    st = lib.gdml_test_set_wait_limit(0xFFFFFFFF if polls is None else int(polls))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())


def test_cholesky_jitter(A: torch.Tensor):
    """The library's FP64 Cholesky with the jitter retries of the preconditioner build on A (k x k):
    returns (lower factor, jitter)."""
    lib = load()
    A = A.contiguous()
    k = A.shape[0]
    L = torch.zeros_like(A)
    eps = ctypes.c_double()
    st = lib.gdml_test_cholesky_jitter(_ptr(A), k, _ptr(L), ctypes.byref(eps),
                                       ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return torch.tril(L), float(eps.value)


def launch_count() -> int:
    """Kernel launches executed by the library so far (graph replays included)."""
    return int(load().gdml_launch_count())


def matvec_noalloc(R: torch.Tensor, sigma: float, lam: float, v: torch.Tensor, out: torch.Tensor | None = None,
                   add_lambda: bool = True) -> torch.Tensor:
    """K v (+ lam v) with no context and no device allocation inside the library
    (M <= 128 geometries, N <= 24 atoms; scratch is a static device array)."""
    lib = load()
    if R.dtype != torch.float64 or R.dim() != 3 or R.shape[2] != 3 or not R.is_cuda:
        raise ValueError("R must be a float64 CUDA tensor of shape (M, N, 3)")
    n = 3 * int(R.shape[0]) * int(R.shape[1])
    _vec_arg(v, n, R.device, "v")
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=R.device)
    _vec_arg(out, n, R.device, "out")
    R = R.contiguous()
    # the library looks up its static scratch array on the CURRENT device: make it R's
    with torch.cuda.device(R.device):
        st = lib.gdml_matvec_noalloc(_ptr(R), int(R.shape[0]), int(R.shape[1]), float(sigma), float(lam),
                                     _ptr(v), _ptr(out), int(add_lambda),
                                     ctypes.c_void_p(torch.cuda.current_stream(R.device).cuda_stream))
    if st != 0:
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return out


def pcg_solve_batched(ctxs, ys, alphas=None, rtol: float = 1e-8, max_iter: int = 20000,
                      raise_on_nonconvergence: bool = True):
    """Solve many FP64 systems with one CUDA graph launch per round.
    Returns (alphas, iterations list, relative residual list)."""
    lib = load()
    n = len(ctxs)
    if alphas is None:
        alphas = [torch.zeros(c.n, dtype=torch.float64, device=c.device) for c in ctxs]
    H = (ctypes.c_void_p * n)(*[c._h for c in ctxs])
    Y = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    A = (ctypes.c_void_p * n)(*[a.data_ptr() for a in alphas])
    it = (ctypes.c_int32 * n)()
    rel = (ctypes.c_double * n)()
    st = lib.gdml_pcg_solve_batched(H, n, Y, A, float(rtol), int(max_iter), it, rel)
    if st != 0 and (raise_on_nonconvergence or st != 6):
        raise GdmlError(st, lib.gdml_last_error(None).decode())
    return alphas, list(it), list(rel)


class Scorer:
    """Learned inducing-column scorer (BF16 MLP D -> hidden -> hidden -> 1, GELU)."""

    def __init__(self, D: int, hidden: int = 256, seed: int = 0, device=None):
        lib = load()
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        st = lib.gdml_scorer_create(ctypes.byref(h), int(D), int(hidden), int(seed),
                                    ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))
        if st != 0:
            raise GdmlError(st, lib.gdml_last_error(None).decode())
        self._h = h
        self.D, self.hidden = D, hidden

    def _check(self, st):
        if st != 0:
            raise GdmlError(st, load().gdml_last_error(None).decode())

    def fit_scaling(self, X, y):
        self._check(load().gdml_scorer_fit_scaling(self._h, _ptr(X.contiguous()), _ptr(y.contiguous()), X.shape[0]))

    def train(self, X, y, epochs=200, batch=256, lr=1e-3) -> float:
        loss = ctypes.c_double()
        self._check(load().gdml_scorer_train(self._h, _ptr(X.contiguous()), _ptr(y.contiguous()), X.shape[0],
                                             int(epochs), int(batch), float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def predict(self, X) -> torch.Tensor:
        out = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        self._check(load().gdml_scorer_predict(self._h, _ptr(X.contiguous()), X.shape[0], _ptr(out)))
        return out

    def nparam(self) -> int:
        n = ctypes.c_int64()
        self._check(load().gdml_scorer_params(self._h, None, 0, ctypes.byref(n)))
        return int(n.value)

    def params(self) -> torch.Tensor:
        p = torch.empty(self.nparam(), dtype=torch.float32, device=self.device)
        self._check(load().gdml_scorer_params(self._h, _ptr(p), 0, None))
        return p

    def set_params(self, p: torch.Tensor):
        self._check(load().gdml_scorer_params(self._h, _ptr(p.contiguous()), 1, None))

    def grad(self, X, y):
        g = torch.empty(self.nparam(), dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        self._check(load().gdml_scorer_grad(self._h, _ptr(X.contiguous()), _ptr(y.contiguous()), X.shape[0],
                                            ctypes.byref(loss), _ptr(g)))
        return float(loss.value), g

    def destroy(self):
        if getattr(self, "_h", None):
            load().gdml_scorer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def geometry_labels(ctx: Context, k: int = 0, seed: int = 2, exact: bool = False) -> torch.Tensor:
    """Per-geometry ridge-leverage mass (the training label of the learned scorer): the sum of
    the scores of the geometry's 3N columns, exact (dense eigendecomposition, small n) or the
    Nystrom estimate with pilot k, computed and summed in the library."""
    out = torch.empty(ctx.M, dtype=torch.float64, device=ctx.device)
    ctx._check(load().gdml_rls_labels(ctx._h, 1 if exact else 0, int(k), int(seed), _ptr(out)))
    return out


def solve_learned(ctx: Context, scorer: Scorer, y, k: int, seed: int = 2, rtol: float = 1e-8,
                  max_iter: int = 20000, referee_iters: int | None = None):
    """Learned selection with pivoted Cholesky (Alg. 1) as fallback and referee:
    build from the scorer's per-geometry scores; fall back to Alg. 1 if the
    inducing block is not SPD, or if PCG needs more than 1.5x the iterations of
    the Alg. 1 preconditioner (referee_iters; measured here when not given).
    Returns (alpha, iterations, relres, used) with used in {"learned", "pivchol"}."""
    scores = scorer.predict(ctx.descriptors())
    try:
        ctx.precond_build_scored(scores, k, seed)
    except GdmlError as e:
        if e.name != "ERR_NOT_SPD":
            raise
        ctx.precond_build("pivchol", k)
        a, it, rel, _ = ctx.pcg_solve(y, rtol=rtol, max_iter=max_iter)
        return a, it, rel, "pivchol"
    cap = max_iter if referee_iters is None else min(max_iter, int(1.5 * referee_iters) + 1)
    a, it, rel, _ = ctx.pcg_solve(y, rtol=rtol, max_iter=cap, raise_on_nonconvergence=False)
    if rel <= rtol and (referee_iters is None or it <= 1.5 * referee_iters):
        return a, it, rel, "learned"
    ctx.precond_build("pivchol", k)
    a, it2, rel2, _ = ctx.pcg_solve(y, rtol=rtol, max_iter=max_iter)
    return a, it + it2, rel2, "pivchol"
