"""OZAKI form: the matvec's descriptor contractions on the BF16 tensor cores with
FP64-class accuracy (operands split into exact 7-bit BF16 slices per 256-entry
chunk, exact FP32 accumulation per slice level, double-float combination).
Like DF64 it must reach the FP64 target at the paper's lambda = 1e-10."""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from oracle import precond as op
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


def _gemm(A, B, G=0):
    return gdml.test_oz_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), G).cpu().numpy()


@pytest.mark.parametrize("M,N,K,G", [(1, 1, 1, 0), (128, 64, 256, 0), (130, 70, 300, 0), (257, 65, 1000, 1),
                                     (257, 65, 1000, 2), (257, 65, 1000, 3), (257, 65, 1000, 4), (200, 200, 64, 0),
                                     (300, 90, 5000, 0), (300, 90, 5000, 7)])
def test_sliced_gemm_matches_fp64(M, N, K, G):
    """Several tiles, ragged edges in every dimension, 1-20 K-chunks, and G of them accumulated
    per CTA in double-float before one partial per group is stored (0: the automatic G)."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = _gemm(A, B, G)
    ref = A @ B.T
    scale = (np.abs(A) @ np.abs(B).T).max()
    err = np.abs(C - ref).max() / scale
    print(f"sliced gemm {M}x{N}x{K} G={G}: max error / max(|A||B|^T) = {err:.2e}")
    assert err <= 1e-14


def test_sliced_gemm_is_exact_on_small_integers():
    """Integer operands |a| <= 100 are exact in the slices and every partial sum is
    an integer below 2^48, so the result must equal the exact product bit for bit."""
    rng = np.random.default_rng(7)
    A = rng.integers(-100, 101, size=(190, 1500)).astype(np.float64)
    B = rng.integers(-100, 101, size=(75, 1500)).astype(np.float64)
    C = _gemm(A, B)
    assert np.array_equal(C, A @ B.T)


def test_sliced_gemm_row_scales_and_zero_rows():
    """Per-row/column power-of-two scaling: rows spanning 1e-25..1e25 keep their
    own relative accuracy; an all-zero row and column give exact zeros."""
    rng = np.random.default_rng(8)
    M, N, K = 140, 66, 520
    ra = 10.0 ** rng.uniform(-25, 25, size=M)
    cb = 10.0 ** rng.uniform(-5, 5, size=N)
    A = rng.standard_normal((M, K)) * ra[:, None]
    B = rng.standard_normal((N, K)) * cb[:, None]
    A[3] = 0.0
    B[5] = 0.0
    C = _gemm(A, B)
    ref = A @ B.T
    assert np.all(C[3] == 0.0) and np.all(C[:, 5] == 0.0)
    scale = np.abs(A) @ np.abs(B).T
    rel = np.abs(C - ref) / np.maximum(scale.max(axis=1, keepdims=True), 1e-300)
    assert rel.max() <= 1e-14


@pytest.mark.parametrize("name,N,M,sigma", [("tiny_N5_M3", 5, 3, 1.0), ("single_geometry_N6_M1", 6, 1, 2.0),
                                            ("two_atoms_N2_M7", 2, 7, 1.5), ("ragged_N7_M150", 7, 150, 3.0), ("ethanol9_m200", 9, 200, 10.0),
                                            ("wide_N30_M64", 30, 64, 15.0), ("wider_N48_M40", 48, 40, 25.0),
                                            ("aspirin21_m1000", 21, 1000, 20.0)])
def test_ozaki_matvec_is_fp64_class(name, N, M, sigma):
    """D = N(N - 1)/2 up to 1128: one and several 256-entry chunks per descriptor row (the
    projection fused with the slicing of W up to 4 chunks, the unfused FP64 projection
    beyond), one to five descriptors per thread in the back-projection (the fifth through
    its loop).  M <= 64 pads U's K to 128 entries, not to a whole 256-entry chunk, so U's two
    products run as two launches; larger M runs them as one product over the concatenated
    K."""
    if name.startswith("aspirin"):
        R = synth.workload("aspirin21_m1000").R
    else:
        R = synth.geometries(synth.template(N, 5), M, 0.1, 6)
    ctx = gdml.kernel_setup(torch.from_numpy(R).cuda(), sigma, 1e-6, precision="ozaki")
    v = np.random.default_rng(0).standard_normal(R.size)
    got = ctx.matvec(torch.from_numpy(v).cuda()).cpu().numpy()
    ctx.tc_check()
    ref = ok.matvec(R, sigma, v, 1e-6)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    emax = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"ozaki matvec relative error vs FP64 oracle ({name}): {err:.2e} (elementwise {emax:.2e})")
    assert err <= 1e-12
    assert emax <= 1e-10
    ctx.destroy()


def test_ozaki_pcg_reaches_fp64_target_at_tiny_lambda():
    w = synth.workload("ethanol9_m200")
    y = torch.from_numpy(w.y).cuda()
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision="ozaki")
    ctx.precond_build("uniform", 400, seed=2)
    alpha, iters, rel, _ = ctx.pcg_solve(y, rtol=1e-8)
    a = alpha.cpu().numpy()
    K = ok.force_kernel_dense(w.R, w.sigma)
    res = np.linalg.norm(w.y - K @ a - w.lam * a) / np.linalg.norm(w.y)
    bound = 8 * EPS * np.linalg.norm(K, 2) * np.linalg.norm(a) / np.linalg.norm(w.y)
    ref = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision="df64")
    ref.precond_build("uniform", 400, seed=2)
    _, itdf, _, _ = ref.pcg_solve(y, rtol=1e-8)
    print(f"ozaki: {iters} iterations (df64: {itdf}), FP64 residual {res:.2e}")
    assert rel <= 1e-8 and res <= 1e-8 + bound
    assert iters <= 1.5 * itdf
    ctx.destroy()
    ref.destroy()


def test_ozaki_preconditioner_matches_df64():
    """The OZAKI build forms C = lambda I + L^T L on the sliced tensor cores, the DF64
    build in double-float on the FP32 lanes: same pivots, same factor, and applies that
    agree far below the PCG tolerance."""
    w = synth.workload("ethanol9_m200")
    R = torch.from_numpy(w.R).cuda()
    r = torch.from_numpy(np.random.default_rng(5).standard_normal(w.n)).cuda()
    out = {}
    for prec in ("df64", "ozaki"):
        ctx = gdml.kernel_setup(R, w.sigma, w.lam, precision=prec)
        piv, _ = ctx.precond_build("pivchol", 300, pivots=True, trace=True)
        out[prec] = (piv.cpu().numpy(), ctx.precond_apply(r).cpu().numpy())
        ctx.destroy()
    assert np.array_equal(out["df64"][0], out["ozaki"][0])
    za, zb = out["df64"][1], out["ozaki"][1]
    rel = np.linalg.norm(za - zb) / np.linalg.norm(za)
    print(f"preconditioner apply, ozaki vs df64 build: {rel:.2e}")
    assert rel <= 1e-6


@pytest.mark.parametrize("n,K,NB,tri", [(1, 1, 1, True), (300, 130, 70, False), (1000, 300, 257, True),
                                        (70000, 520, 130, True)])
def test_sliced_tall_gemm_matches_fp64(n, K, NB, tri):
    """The OZAKI build's accumulating GEMM with a column-major tall A: ragged n, K and NB,
    one and several 256-entry K chunks, two row panels (n > 65,536), the triangular K skip,
    the column-major FP64 / FP32 store and the row square sums."""
    rng = np.random.default_rng(n + K + NB)
    A = rng.standard_normal((n, K)) * 10.0 ** rng.uniform(-3, 3, size=(n, 1))
    B = rng.standard_normal((NB, K))
    if tri:
        B = np.tril(B)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C, C32 = gdml.test_oz_gemm_tall(Ad, Bd, tri_b=tri)
    C = C.cpu().numpy()
    ref = A @ B.T
    # the slices keep 49 bits of each entry below its 256-entry chunk's largest magnitude, so a
    # chunk's products err by at most ~2^-48 KC max|a| max|b| (dropped slice pairs far below);
    # the FP64 reference adds its own rounding, 8 eps sum |a||b|
    bound = 8 * EPS * (np.abs(A) @ np.abs(B).T)
    for q0 in range(0, K, 256):
        ma = np.abs(A[:, q0:q0 + 256]).max(axis=1)
        mb = np.abs(B[:, q0:q0 + 256]).max(axis=1)
        bound += 2.0 ** -47 * min(256, K - q0) * np.outer(ma, mb)
    err = (np.abs(C - ref) / np.maximum(bound, 1e-300)).max()
    print(f"tall sliced gemm {n}x{NB}x{K} tri={tri}: max error / bound = {err:.3f}")
    assert err <= 1.0
    assert np.array_equal(C32.cpu().numpy(), C.astype(np.float32))
    sq = gdml.test_oz_gemm_tall(Ad, Bd, tri_b=tri, rowsq=True).cpu().numpy()
    own = np.sum(C * C, axis=1)
    assert np.all(np.abs(sq - own) <= 1e-13 * own)


@pytest.mark.parametrize("prec", ["df64", "ozaki"])
@pytest.mark.parametrize("method,k", [("uniform", 400), ("rls", 150)])
def test_nystrom_factor_matches_oracle(prec, method, k):
    """L_k = K_nk L_kk^-T (Eq. 5) element by element against the oracle's factor for the same
    inducing columns.  DF64 forms it by FP64 substitution, OZAKI as K_nk times the explicit
    triangular inverse on the sliced tensor cores; both store it in FP32.  Bound per entry:
    the FP32 rounding 2^-24 |L| plus 64 eps of the products' magnitude |K_nk| |L_kk^-1|^T."""
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision=prec)
    piv, _ = ctx.precond_build(method, k, seed=2, pivots=True)
    rank, jit = ctx.precond_info()
    Lg = ctx.precond_factor().cpu().numpy()
    ctx.destroy()
    S = piv.cpu().numpy()
    K = ok.force_kernel_dense(w.R, w.sigma)
    Lr, eps = op.nystrom_factor(K[:, S], S)
    assert rank == k and jit == eps
    L_kk, _ = op.cholesky_jitter(K[np.ix_(S, S)])
    Linv = np.linalg.inv(L_kk)
    # magnitudes of the product K_nk L_kk^-T and of the substitution's error terms
    mag = np.abs(K[:, S]) @ np.abs(Linv).T + (np.abs(Lr) @ np.abs(L_kk).T) @ np.abs(Linv).T
    bound = 2.0 ** -24 * np.abs(Lr) + 4 * k * EPS * mag
    worst = (np.abs(Lg - Lr) / bound).max()
    print(f"{prec} {method} k={k} (jitter {jit:.1e}): max |L_gpu - L_oracle| / bound = {worst:.3f}")
    assert worst <= 1.0
    if jit == 0.0:  # Eq. 5: the rows of L_k at the inducing columns are L_kk (lower triangular)
        assert np.abs(np.triu(Lg[S], 1)).max() <= 1e-6 * np.abs(Lr).max()
