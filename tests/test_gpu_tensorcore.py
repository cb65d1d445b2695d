"""tcgen05 tensor-core path: the GEMM building block, the TF32/BF16 matvec and the
FP64 iterative refinement around it, against FP64 references.

Error bars (stated per result, not parity claims): operands are rounded to
TF32 (unit roundoff 2^-11) or BF16 (2^-8) and products accumulate in FP32, so
|C - A B^T| <= (2 u + K 2^-23) (|A| |B|^T) elementwise.  The matvec's error is
reported against the FP64 oracle; the refined solve must reach the FP64 true
relative residual 1e-8 like the FP64 form.
"""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 40, 36), (300, 260, 224), (1000, 1000, 210), (77, 513, 861)])
def test_tc_gemm_matches_fp64(bf16, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = gdml.test_tc_gemm(dev(A), dev(B), bf16).cpu().numpy()
    ref = A @ B.T
    u = 2.0 ** -8 if bf16 else 2.0 ** -11
    bound = (2 * u + K * 2.0 ** -23) * (np.abs(A) @ np.abs(B).T)
    assert np.all(np.abs(C - ref) <= bound + 1e-30)
    # and the errors are rounding-sized, not structural
    assert np.linalg.norm(C - ref) <= 4 * u * np.linalg.norm(ref) + 1e-12


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("bf16", 5e-2)])
@pytest.mark.parametrize("name,N,M,sigma", [("ragged_N7_M150", 7, 150, 3.0), ("ethanol9_m200", 9, 200, 10.0)])
def test_tc_matvec_error_vs_fp64_oracle(prec, tol, name, N, M, sigma):
    tmpl = synth.template(N, 5)
    R = synth.geometries(tmpl, M, 0.1, 6)
    lam = 1e-6
    ctx = gdml.kernel_setup(dev(R), sigma, lam, precision=prec)
    v = np.random.default_rng(0).standard_normal(3 * N * M)
    got = ctx.matvec(dev(v)).cpu().numpy()
    ctx.tc_check()
    ref = ok.matvec(R, sigma, v, lam)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"{prec} matvec relative error vs FP64 oracle ({name}): {err:.3e}")
    assert err <= tol
    # the FP64 entry point of the same context is exact to FP64 rounding
    got64 = ctx.matvec_fp64(dev(v)).cpu().numpy()
    assert np.linalg.norm(got64 - ref) <= 1e-12 * np.linalg.norm(ref)
    ctx.destroy()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_precision_refinement_reaches_fp64_residual_when_lambda_dominates(prec):
    """FP64 refinement around the tensor-core PCG converges to the FP64 residual
    target when the ridge lambda is large against the matvec's rounding error."""
    w = synth.workload("ethanol9_m200")
    lam = 1e-2
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, lam, precision=prec)
    ctx.precond_build("uniform", 100, seed=2)
    alpha, iters, rel, outer = ctx.pcg_solve(dev(w.y), rtol=1e-8, max_iter=40000)
    ctx.tc_check()
    a = alpha.cpu().numpy()
    res = np.linalg.norm(w.y - ok.matvec(w.R, w.sigma, a, lam)) / np.linalg.norm(w.y)
    print(f"{prec} lambda={lam}: {iters} inner iterations, {outer} refinements, FP64 residual {res:.2e}")
    assert rel <= 1e-8 and outer >= 2 and res <= 2e-8
    ctx.destroy()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_precision_stagnation_is_reported_at_tiny_lambda(prec):
    """At lambda = 1e-10 the tensor-core rounding error (~1e-4 |K|) swamps the
    small eigen-directions that carry most of y: refinement must stop, keep its
    best iterate and report the true FP64 residual it reached."""
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam, precision=prec)
    ctx.precond_build("uniform", 400, seed=2)
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_solve(dev(w.y), rtol=1e-8, max_iter=40000)
    assert e.value.name == "ERR_NOT_CONVERGED"
    alpha, iters, rel, outer = ctx.pcg_solve(dev(w.y), rtol=1e-8, max_iter=40000, raise_on_nonconvergence=False)
    ctx.tc_check()
    a = alpha.cpu().numpy()
    res = np.linalg.norm(w.y - ok.matvec(w.R, w.sigma, a, w.lam)) / np.linalg.norm(w.y)
    print(f"{prec} lambda=1e-10: {iters} inner iterations, {outer} refinements, FP64 residual {res:.2e}")
    assert rel > 1e-8 and res <= 1.0 + 1e-12  # never worse than the start
    assert abs(res - rel) <= 1e-6 * res + 1e-12  # the reported residual is the true FP64 one
    ctx.destroy()
