"""Reduced slice levels in the OZAKI matvec (gdml_set_inner_levels): the sliced GEMM keeps only
the slice pairs i + j < L, and PCG runs on that cheaper operator with FP64 true-residual
restarts (a mixed-precision scheme whose outer residual is FP64).

* GEMM: the error of the L-level product is bounded by the dropped pairs, computed from the
  slicing's definition (x = 2^(e-7) (sum_i s_i 2^-7i + rho), |s_0| <= 128, |s_i| <= 64,
  |rho| <= 2^-43, e the chunk exponent with |x| < 2^e) -- and it is larger than the 7-level
  error, so the pairs really are dropped; with operands that fit in slice 0 one level is exact;
* solves at the configs' lambda = 1e-10, the oracle's FP64 matvec recomputing the true
  residual of the GPU's alpha.
"""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps
KC = 256  # entries per chunk of the slicing


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2212_12737_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    gdml.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gemm(A, B, levels):
    return gdml.test_oz_gemm(dev(A), dev(B), 0, levels).cpu().numpy()


def chunk_exponents(X):
    """e[r, q]: the smallest e with |x| < 2^e over row r's chunk q (0 for an all-zero chunk)."""
    nq = -(-X.shape[1] // KC)
    e = np.zeros((X.shape[0], nq), dtype=np.int64)
    for q in range(nq):
        m = np.abs(X[:, q * KC:(q + 1) * KC]).max(axis=1)
        e[:, q] = np.where(m > 0, np.frexp(m)[1], 0)
    return e


def truncation_bound(A, B, levels):
    """Largest error of the L-level product: per chunk, 2^(eA + eB - 14) times the chunk length
    times (the dropped pairs' largest terms + the slicing remainders' terms)."""
    smax = np.array([128.0] + [64.0] * 6)
    per = 0.0
    for i in range(7):
        for j in range(7):
            if i + j >= levels:
                per += smax[i] * smax[j] * 2.0 ** (-7 * (i + j))
    rho = 2.0 ** -43
    per += 2 * rho * smax.dot(2.0 ** (-7 * np.arange(7))) + rho * rho
    eA, eB = chunk_exponents(A), chunk_exponents(B)
    K = A.shape[1]
    bound = np.zeros((A.shape[0], B.shape[0]))
    for q in range(eA.shape[1]):
        ln = min(KC, K - q * KC)
        bound += np.ldexp(1.0, eA[:, q][:, None] + eB[:, q][None, :] - 14) * ln * per
    return bound


def test_reduced_level_gemm_within_its_truncation_bound():
    rng = np.random.default_rng(11)
    M, N, K = 200, 90, 700  # two tiles of rows, two of columns, 3 chunks (the last ragged)
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, 1))
    B = rng.standard_normal((N, K))
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    errs = {}
    for L in (1, 2, 3, 4, 5, 6, 7):
        C = _gemm(A, B, L)
        d = np.abs(C - ref)
        bound = truncation_bound(A, B, L) + 16 * EPS * scale
        errs[L] = (d / scale).max()
        print(f"levels {L}: max error / |A||B|^T = {errs[L]:.2e}, max error / bound = {(d / bound).max():.3f}")
        assert np.all(d <= bound)
    for L in range(1, 7):  # each dropped level is visible
        assert errs[L] > 10 * errs[L + 1]


def test_one_level_is_exact_when_the_operands_fit_one_slice():
    """|x| <= 64 integers: after the chunk scaling every entry is its own first slice, so the
    pair (0, 0) alone is the exact product (sums stay below 2^24 per chunk)."""
    rng = np.random.default_rng(12)
    A = rng.integers(-64, 65, size=(150, 900)).astype(np.float64)
    B = rng.integers(-64, 65, size=(70, 900)).astype(np.float64)
    for L in (1, 4):
        assert np.array_equal(_gemm(A, B, L), A @ B.T)


def test_inner_levels_arguments():
    R = synth.geometries(synth.template(5, 1), 4, 0.1, 2)
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision="fp64")
    with pytest.raises(gdml.GdmlError) as e:
        ctx.set_inner_levels(6)
    assert e.value.name == "ERR_ARG"
    ctx.destroy()
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision="ozaki")
    for bad in (0, 8):
        with pytest.raises(gdml.GdmlError) as e:
            ctx.set_inner_levels(bad)
        assert e.value.name == "ERR_ARG"
    ctx.set_inner_levels(7)
    ctx.destroy()


@pytest.mark.parametrize("name", ["ethanol9_m200", "aspirin21_m1000"])
@pytest.mark.parametrize("levels", [6, 5])
def test_inner_level_solve_reaches_the_fp64_target(name, levels):
    """lambda = 1e-10 (the configs' value): PCG on the L-level operator, restarted from the FP64
    true residual, reaches 1e-8, and the oracle's own matvec confirms the residual of alpha."""
    w = synth.workload(name)
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam, precision="ozaki")
    ctx.precond_build(w.select, w.k, seed=2)
    ctx.set_inner_levels(levels)
    alpha, iters, rel, runs = ctx.pcg_solve(dev(w.y), rtol=1e-8)
    ctx.tc_check()
    v = dev(np.random.default_rng(3).standard_normal(w.n))
    for _ in range(30):
        v = ctx.matvec(v, add_lambda=False)
        knorm = float(torch.linalg.norm(v))
        v = v / knorm
    ctx.destroy()
    a = alpha.cpu().numpy()
    res = np.linalg.norm(w.y - ok.matvec(w.R, w.sigma, a, w.lam)) / np.linalg.norm(w.y)
    bound = 8 * EPS * knorm * np.linalg.norm(a) / np.linalg.norm(w.y)
    print(f"{name} levels {levels}: {iters} iterations in {runs} runs, GPU relres {rel:.2e}, oracle {res:.2e}")
    assert runs >= 1 and rel <= 1e-8 and res <= 1e-8 + bound
