"""GPU path vs the FP64 CPU oracle, through the C ABI (FP64 contexts).

Tolerances (FP64 arithmetic on both sides, different summation orders):
* matvec: |dK v|_2 <= 1e-12 |K v|_2 and max |dK v| <= 1e-10 max |K v| (bar: 1e-10 relative);
* selection: bit-exact indices; pivoted-Cholesky pivots bit-exact unless the
  two candidates' residual diagonals tie within 1e-12 of the largest diagonal;
* Woodbury apply: elementwise within 64 eps |C|/lambda of max |z| (Eq. 4 cancels);
* PCG: the oracle's own FP64 relative residual of the GPU's alpha <= rtol plus
  the evaluation error bound 8 eps |K| |alpha| / |y|.
"""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from oracle import precond as op
from oracle import solver as osv
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12737_gb300 import build
    import os
    if not os.path.exists(build.LIB):
        build.build()
    gdml.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def case(N, M, noise, seed):
    tmpl = synth.template(N, seed)
    R = synth.geometries(tmpl, M, noise, seed + 1)
    y = synth.morse_forces(R, tmpl).reshape(-1)
    return R, y


MATVEC_CASES = [
    ("tiny_N5_M3", 5, 3, 0.3, 1.0),
    ("single_geometry_N6_M1", 6, 1, 0.1, 2.0),
    ("two_atoms_N2_M7", 2, 7, 0.1, 1.5),
    ("ragged_N7_M150", 7, 150, 0.1, 3.0),
    ("ethanol9_m200", 9, 200, 0.05, 10.0),
]


@pytest.mark.parametrize("name,N,M,noise,sigma", MATVEC_CASES)
def test_matvec_fp64_matches_oracle(name, N, M, noise, sigma):
    R, _ = case(N, M, noise, 5)
    lam = 1e-6
    ctx = gdml.kernel_setup(dev(R), sigma, lam)
    rng = np.random.default_rng(1)
    for _ in range(2):
        v = rng.standard_normal(3 * N * M)
        got = ctx.matvec(dev(v)).cpu().numpy()
        ref = ok.matvec(R, sigma, v, lam)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    ctx.destroy()


def test_matvec_fp64_full_size_aspirin21_m1000():
    w = synth.workload("aspirin21_m1000")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam)
    v = np.random.default_rng(2).standard_normal(w.n)
    got = ctx.matvec(dev(v)).cpu().numpy()
    ref = ok.matvec(w.R, w.sigma, v, w.lam)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    ctx.destroy()


def test_uniform_selection_is_bit_exact():
    for name in ("ethanol9_m200", "aspirin21_m1000"):
        w = synth.workload(name)
        ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam)
        piv, _ = ctx.precond_build("uniform", min(w.k, 500), seed=2, pivots=True)
        assert np.array_equal(piv.cpu().numpy(), op.select_uniform(w.n, min(w.k, 500), 2))
        ctx.destroy()


def compare_pivots(gpu, ref, dref):
    """Equal pivot sequences, or a first divergence at a certified near-tie."""
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    if np.array_equal(gpu, ref):
        return len(ref)
    m = int(np.argmax(gpu != ref))
    assert abs(dref[m][gpu[m]] - dref[m][ref[m]]) <= 1e-12 * dref[0].max(), f"pivot {m} differs"
    return m


def oracle_pivchol_with_diags(get_col, d, k):
    """Algorithm 1 via the oracle, also returning the residual diagonal before each step."""
    diags = []
    dcur = np.array(d, copy=True)

    def spy(i):
        return get_col(i)

    L, piv, tr = op.pivoted_cholesky(spy, d, k)
    # replay the residual diagonals from the factor (d_m = diag - sum_{j<m} l_j^2)
    acc = np.array(d, copy=True)
    for m in range(L.shape[1]):
        diags.append(acc.copy())
        acc = acc - L[:, m] ** 2
    return L, piv, tr, diags


@pytest.mark.parametrize("name,k", [("ethanol9_m200", 100), ("ethanol9_m200", 400), ("aspirin21_m1000", 48)])
def test_pivoted_cholesky_pivots_and_trace_match_oracle(name, k):
    w = synth.workload(name)
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam)
    piv, tr = ctx.precond_build("pivchol", k, pivots=True, trace=True)
    get_col = ok.column_getter(w.R, w.sigma)
    L, rpiv, rtr, diags = oracle_pivchol_with_diags(get_col, ok.force_kernel_diag(w.R, w.sigma), k)
    m = compare_pivots(piv.cpu().numpy(), rpiv, diags)
    np.testing.assert_allclose(tr.cpu().numpy()[:m], rtr[:m], rtol=1e-8, atol=1e-12 * rtr[0])
    assert np.all(np.diff(tr.cpu().numpy()) <= 1e-12 * rtr[0])
    ctx.destroy()


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_rls_selection_matches_oracle(prec):
    """The scores come from the FP64 Nystrom factor of the pilot set in every form."""
    w = synth.workload("ethanol9_m200")
    k = 100
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam, precision=prec)
    piv, _ = ctx.precond_build("rls", k, seed=3, pivots=True)
    K = ok.force_kernel_dense(w.R, w.sigma)
    S, tau = op.select_rls(lambda idx: K[:, idx], w.n, k, w.lam, 3)
    got = set(piv.cpu().numpy().tolist())
    ref = set(S.tolist())
    # keys -ln(u)/tau: any disagreement must be a near-tie at the k-th key
    from oracle import philox
    u = philox.uniforms(w.n, 3, philox.STREAM_RLS_SAMPLE)
    key = -np.log(u) / tau
    kth = np.sort(key)[k - 1]
    for i in got ^ ref:
        assert abs(key[i] - kth) <= 1e-6 * kth
    assert len(got ^ ref) <= 4
    ctx.destroy()


@pytest.mark.parametrize("lam", [1e-4, 1e-10])
def test_woodbury_apply_matches_oracle(lam):
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, lam)
    piv, _ = ctx.precond_build("uniform", w.k, seed=2, pivots=True)
    S = piv.cpu().numpy()
    K = ok.force_kernel_dense(w.R, w.sigma)
    L, eps = op.nystrom_factor(K[:, S], S)
    rank, jit = ctx.precond_info()
    assert rank == w.k and jit == eps
    LC = op.woodbury_core(L, lam)
    r = np.random.default_rng(3).standard_normal(w.n)
    z = ctx.precond_apply(dev(r)).cpu().numpy()
    amp = max(1.0, np.linalg.norm(L, 2) ** 2 / lam)
    if lam >= 1e-4:
        ref = op.woodbury_apply(L, LC, lam, r)
        np.testing.assert_allclose(z, ref, rtol=0, atol=64 * EPS * amp * np.abs(ref).max())
    # backward check against the dense P of Eq. 3
    Pz = L @ (L.T @ z) + lam * z
    assert np.linalg.norm(Pz - r) <= 64 * EPS * amp * np.linalg.norm(r)
    ctx.destroy()


def test_pcg_fp64_ethanol_uniform_reaches_rtol():
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam)
    ctx.precond_build("uniform", w.k, seed=2)
    alpha, iters, rel, outer = ctx.pcg_solve(dev(w.y), rtol=1e-8, max_iter=20000)
    a = alpha.cpu().numpy()
    K = ok.force_kernel_dense(w.R, w.sigma)
    res = np.linalg.norm(w.y - K @ a - w.lam * a) / np.linalg.norm(w.y)
    bound = 8 * EPS * np.linalg.norm(K, 2) * np.linalg.norm(a) / np.linalg.norm(w.y)
    assert rel <= 1e-8
    assert res <= 1e-8 + bound, (res, bound, iters)
    exact = osv.solve_exact(K, w.lam, w.y)
    assert np.linalg.norm(K @ (a - exact) + w.lam * (a - exact)) <= (2e-8 + 2 * bound) * np.linalg.norm(w.y)
    ctx.destroy()


def test_pcg_fp64_pivchol_matches_oracle_iterations():
    tmpl = synth.template(6, 4)
    R = synth.geometries(tmpl, 30, 0.1, 5)
    y = synth.morse_forces(R, tmpl).reshape(-1)
    sigma, lam, k = 5.0, 1e-6, 60
    ctx = gdml.kernel_setup(dev(R), sigma, lam)
    ctx.precond_build("pivchol", k)
    alpha, iters, rel, _ = ctx.pcg_solve(dev(y), rtol=1e-8)
    K = ok.force_kernel_dense(R, sigma)
    L, piv, _ = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k)
    LC = op.woodbury_core(L, lam)
    ref = osv.pcg(lambda v: K @ v + lam * v, lambda r: op.woodbury_apply(L, LC, lam, r), y, 1e-8, max_iter=20000)
    assert ref.converged and rel <= 1e-8
    assert abs(iters - ref.iters) <= max(3, 0.1 * ref.iters)
    ctx.destroy()


@pytest.mark.parametrize("prec,max_iters", [("fp64", 3), ("df64", 15), ("ozaki", 15)])
def test_full_rank_nystrom_converges_in_few_iterations(prec, max_iters):
    """k = rank(K): P = L Lt + lam I equals K + lam I up to the factor's rounding, so PCG
    needs a few steps where plain CG needs 154 (n = 90).  The DF64 and OZAKI forms store L
    in FP32: |K - L Lt| ~ 2^-24 |K| = 7e-8 against lam = 1e-6.  The bound 15 is CG's
    iteration bound for rtol 1e-8 with the preconditioned spectrum inside 1 +- 0.5."""
    tmpl = synth.template(5, 8)
    R = synth.geometries(tmpl, 6, 0.2, 9)
    y = synth.morse_forces(R, tmpl).reshape(-1)
    K = ok.force_kernel_dense(R, 2.0)
    rank = int(np.sum(np.linalg.eigvalsh(K) > 1e-10 * np.trace(K)))
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision=prec)
    ctx.precond_build("pivchol", rank)
    _, iters, rel, _ = ctx.pcg_solve(dev(y), rtol=1e-8)
    print(f"full-rank Nystrom PCG ({prec}): {iters} iterations, residual {rel:.2e}")
    assert rel <= 1e-8 and iters <= max_iters
    ctx.destroy()


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_zero_rhs_and_iteration_cap_and_bad_args(prec):
    w = synth.workload("ethanol9_m200", M=20)
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam, precision=prec)
    alpha, iters, rel, _ = ctx.pcg_solve(torch.zeros(w.n, dtype=torch.float64, device="cuda"))
    assert iters == 0 and rel == 0 and float(alpha.abs().max()) == 0.0
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_solve(dev(w.y), rtol=1e-12, max_iter=3)
    assert e.value.name == "ERR_NOT_CONVERGED"
    alpha, iters, rel, _ = ctx.pcg_solve(dev(w.y), rtol=1e-12, max_iter=3, raise_on_nonconvergence=False)
    assert iters == 3 and np.isfinite(rel) and rel > 1e-12  # plain CG may raise |r| early on
    with pytest.raises(gdml.GdmlError):
        ctx.precond_apply(dev(w.y))  # nothing built yet
    for bad in (0, w.n + 1):
        with pytest.raises(gdml.GdmlError) as e:
            ctx.precond_build("uniform", bad)
        assert e.value.name == "ERR_ARG"
    ctx.destroy()


@pytest.mark.parametrize("prec,k", [("ozaki", 400)])
def test_df_pivoted_cholesky_full_depth_replay_at_full_size(prec, k):
    """Algorithm 1 in the DF64/OZAKI form at n = 63,000 to k = 400: 256-row chunks of the
    fused Schur + finish pass, past m ~ 380 where it streams the first m columns evict-first.
    The oracle replays the GPU's pivot sequence (forced) and at EVERY step the GPU's pivot
    must be the residual diagonal's maximum up to what the FP32 storage of L perturbs
    (1e-6 of the largest diagonal); the residual traces must agree to that storage error."""
    w = synth.workload("aspirin21_m1000")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam, precision=prec)
    piv, tr = ctx.precond_build("pivchol", k, pivots=True, trace=True)
    ctx.destroy()
    gp = piv.cpu().numpy()
    d0 = ok.force_kernel_diag(w.R, w.sigma)
    diags = []
    L, rp, rtr = op.pivoted_cholesky(ok.column_getter(w.R, w.sigma), d0, k, forced=gp, diag_out=diags)
    assert np.array_equal(rp, gp) and len(diags) == k
    tol = 1e-6 * d0.max()
    worst = 0.0
    for m in range(k):
        dm = diags[m]
        dm[gp[:m]] = -np.inf
        worst = max(worst, dm.max() - dm[gp[m]])
        assert dm[gp[m]] >= dm.max() - tol, f"step {m}: pivot {gp[m]} is {dm.max() - dm[gp[m]]:.2e} below the max"
    print(f"{prec} Algorithm 1 replay, k={k}: largest shortfall of a GPU pivot {worst:.2e} (tol {tol:.2e})")
    # each stored l_ij is an FP32 rounding (2^-24 relative) and sum_j l_ij^2 <= K_ii, so every
    # residual diagonal may move by 2 2^-24 K_ii and the trace by 2^-23 tr(K)
    np.testing.assert_allclose(tr.cpu().numpy(), rtr, rtol=0, atol=2.0 ** -23 * d0.sum())


def test_headline_ozaki_solution_by_the_oracle():
    """aspirin21_m1000 in the OZAKI form with the pivoted-Cholesky preconditioner at k = 2000:
    the oracle's own FP64 matvec recomputes the true residual of the GPU's alpha."""
    w = synth.workload("aspirin21_m1000")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam, precision="ozaki")
    ctx.precond_build("pivchol", w.k)
    alpha, iters, rel, _ = ctx.pcg_solve(dev(w.y), rtol=1e-8)
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
    print(f"aspirin21_m1000 ozaki: {iters} iterations, GPU relres {rel:.2e}, oracle relres {res:.2e} "
          f"(bound {bound:.1e})")
    assert rel <= 1e-8 and res <= 1e-8 + bound
