"""DF64 form: the matvec's descriptor contractions in double-float arithmetic on
the FP32 lanes (FP64-class accuracy at the FP32 rate), PCG refined by FP64
true-residual restarts.  Unlike TF32/BF16 it must reach the FP64 target at the
paper's lambda = 1e-10."""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2212_12737_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    gdml.load()


@pytest.mark.parametrize("name,N,M,sigma", [("tiny_N5_M3", 5, 3, 1.0), ("single_geometry_N6_M1", 6, 1, 2.0),
                                            ("two_atoms_N2_M7", 2, 7, 1.5), ("ragged_N7_M150", 7, 150, 3.0), ("ethanol9_m200", 9, 200, 10.0),
                                            ("aspirin21_m1000", 21, 1000, 20.0)])
def test_df64_matvec_is_fp64_class(name, N, M, sigma):
    if name.startswith("aspirin"):
        w = synth.workload("aspirin21_m1000")
        R = w.R
    else:
        R = synth.geometries(synth.template(N, 5), M, 0.1, 6)
    ctx = gdml.kernel_setup(torch.from_numpy(R).cuda(), sigma, 1e-6, precision="df64")
    v = np.random.default_rng(0).standard_normal(R.size)
    got = ctx.matvec(torch.from_numpy(v).cuda()).cpu().numpy()
    ref = ok.matvec(R, sigma, v, 1e-6)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    emax = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"df64 matvec relative error vs FP64 oracle ({name}): {err:.2e} (elementwise {emax:.2e})")
    assert err <= 1e-12
    assert emax <= 1e-10
    ctx.destroy()


def test_df64_pcg_reaches_fp64_target_at_tiny_lambda():
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision="df64")
    ctx.precond_build("uniform", 400, seed=2)
    alpha, iters, rel, _ = ctx.pcg_solve(torch.from_numpy(w.y).cuda(), rtol=1e-8)
    a = alpha.cpu().numpy()
    K = ok.force_kernel_dense(w.R, w.sigma)
    res = np.linalg.norm(w.y - K @ a - w.lam * a) / np.linalg.norm(w.y)
    bound = 8 * EPS * np.linalg.norm(K, 2) * np.linalg.norm(a) / np.linalg.norm(w.y)
    ref = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam)
    ref.precond_build("uniform", 400, seed=2)
    _, it64, _, _ = ref.pcg_solve(torch.from_numpy(w.y).cuda(), rtol=1e-8)
    print(f"df64: {iters} iterations (fp64: {it64}), FP64 residual {res:.2e}")
    assert rel <= 1e-8 and res <= 1e-8 + bound
    assert iters <= 2 * it64
    ctx.destroy()
    ref.destroy()


def test_df64_pivchol_preconditioner_solves_like_fp64():
    """FP32-stored Alg. 1 factor with double-float Schur sums: same leading
    pivots as the FP64 build, and a PCG solve to the FP64 target."""
    w = synth.workload("ethanol9_m200")
    y = torch.from_numpy(w.y).cuda()
    out = {}
    for prec in ("fp64", "df64"):
        ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision=prec)
        piv, tr = ctx.precond_build("pivchol", 300, pivots=True, trace=True)
        alpha, iters, rel, _ = ctx.pcg_solve(y, rtol=1e-8)
        out[prec] = (piv.cpu().numpy(), iters, rel, alpha.cpu().numpy())
        ctx.destroy()
    p64, it64, _, _ = out["fp64"]
    pdf, itdf, reldf, a = out["df64"]
    assert np.array_equal(p64[:50], pdf[:50])  # FP32 rounding of L only perturbs late pivots
    K = ok.force_kernel_dense(w.R, w.sigma)
    res = np.linalg.norm(w.y - K @ a - w.lam * a) / np.linalg.norm(w.y)
    bound = 8 * EPS * np.linalg.norm(K, 2) * np.linalg.norm(a) / np.linalg.norm(w.y)
    print(f"pivchol k=300: fp64 {it64} iterations, df64 {itdf} iterations, FP64 residual {res:.2e}")
    assert reldf <= 1e-8 and res <= 1e-8 + bound and itdf <= 1.5 * it64
