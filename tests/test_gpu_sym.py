"""The symmetric (sGDML) force kernel on the GPU against the oracle (K_ab = sum_q J_a^T H(x_a, P_q x_b)
P_q J_b for a permutation group of the atoms; the oracle's form is pinned in test_oracle_sym.py).

* matvec in FP64 and OZAKI: |d|_2 <= 1e-12 |ref|_2 and max |d| <= 1e-10 max |ref| (as the plain
  kernel's matvec tests);
* preconditioner builds with the symmetric columns and diagonal: the uniform build's L_k element
  by element against the oracle's Nystrom factor, Algorithm 1's pivots replayed by the oracle;
* PCG to rtol = 1e-8 with the oracle's dense symmetric K recomputing the true residual;
* forces predicted from alpha against the dense symmetric kernel's cross blocks.
"""
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def group(N, name):
    """Permutation groups of the N atoms: a transposition, a 3-cycle, the Klein four-group on
    two disjoint transpositions, and S3 on atoms 0, 1, 2 (order 6)."""
    idn = list(range(N))

    def perm(mapping):
        p = list(idn)
        for a, b in mapping.items():
            p[a] = b
        return p
    if name == "swap":
        return [idn, perm({0: 1, 1: 0})]
    if name == "cycle":
        return [idn, perm({0: 1, 1: 2, 2: 0}), perm({0: 2, 1: 0, 2: 1})]
    if name == "klein":
        return [idn, perm({0: 1, 1: 0}), perm({2: 3, 3: 2}), perm({0: 1, 1: 0, 2: 3, 3: 2})]
    if name == "s3":
        import itertools
        return [perm(dict(zip((0, 1, 2), p))) for p in itertools.permutations((0, 1, 2))]
    raise ValueError(name)


def case(N, M, seed, noise=0.15):
    tmpl = synth.template(N, seed)
    R = synth.geometries(tmpl, M, noise, seed + 1)
    return R, synth.morse_forces(R, tmpl).reshape(-1)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("N,M,gname,sigma", [(5, 3, "swap", 1.0), (6, 7, "cycle", 1.5), (9, 60, "klein", 4.0),
                                             (9, 150, "s3", 6.0)])
def test_symmetric_matvec_matches_oracle(prec, N, M, gname, sigma):
    R, _ = case(N, M, 3)
    perms = group(N, gname)
    ctx = gdml.kernel_setup(dev(R), sigma, 1e-6, precision=prec, perms=perms)
    rng = np.random.default_rng(N + M)
    for _ in range(2):
        v = rng.standard_normal(R.size)
        got = ctx.matvec(dev(v)).cpu().numpy()
        ref = ok.matvec_sym(R, sigma, perms, v, 1e-6)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        emax = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"{prec} symmetric matvec N={N} M={M} S={len(perms)}: {err:.2e} (elementwise {emax:.2e})")
        assert err <= 1e-12 and emax <= 1e-10
    ctx.tc_check()
    ctx.destroy()


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_symmetric_nystrom_factor_matches_oracle(prec):
    """Uniform inducing columns: K_nk from the symmetric kernel columns, L_k = K_nk L_kk^-T (Eq. 5),
    element by element against the oracle (bound as in the plain kernel's test)."""
    N, M, k = 6, 40, 120
    R, _ = case(N, M, 5)
    perms = group(N, "cycle")
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision=prec, perms=perms)
    piv, _ = ctx.precond_build("uniform", k, seed=2, pivots=True)
    rank, jit = ctx.precond_info()
    Lg = ctx.precond_factor().cpu().numpy()
    ctx.destroy()
    S = piv.cpu().numpy()
    assert np.array_equal(S, op.select_uniform(R.size, k, 2))
    K = ok.force_kernel_dense_sym(R, 2.0, perms)
    Lr, eps = op.nystrom_factor(K[:, S], S)
    assert rank == k and jit == eps
    L_kk, _ = op.cholesky_jitter(K[np.ix_(S, S)])
    Linv = np.linalg.inv(L_kk)
    mag = np.abs(K[:, S]) @ np.abs(Linv).T + (np.abs(Lr) @ np.abs(L_kk).T) @ np.abs(Linv).T
    bound = (2.0 ** -24 if prec == "ozaki" else 0.0) * np.abs(Lr) + 4 * k * EPS * mag
    worst = (np.abs(Lg - Lr) / np.maximum(bound, 1e-300)).max()
    print(f"{prec} symmetric L_k: max |L_gpu - L_oracle| / bound = {worst:.3f}")
    assert worst <= 1.0


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_symmetric_pivoted_cholesky_replayed_by_the_oracle(prec):
    """Algorithm 1 on the symmetric kernel (its diagonal and columns): the oracle replays the GPU's
    pivots and each must be its step's residual-diagonal maximum (exactly up to FP64 rounding in
    FP64 contexts, up to the FP32 storage of L in OZAKI)."""
    N, M, k = 6, 30, 80
    R, _ = case(N, M, 7)
    perms = group(N, "klein")
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision=prec, perms=perms)
    piv, tr = ctx.precond_build("pivchol", k, pivots=True, trace=True)
    ctx.destroy()
    gp = piv.cpu().numpy()
    K = ok.force_kernel_dense_sym(R, 2.0, perms)
    diags = []
    _, rp, rtr = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k, forced=gp, diag_out=diags)
    tol = (1e-12 if prec == "fp64" else 1e-6) * np.diag(K).max()
    for m, dm in enumerate(diags):
        dm[gp[:m]] = -np.inf
        assert dm[gp[m]] >= dm.max() - tol, f"step {m}"
    np.testing.assert_allclose(tr.cpu().numpy(), rtr, rtol=0,
                               atol=(1e-12 if prec == "fp64" else 2.0 ** -23) * np.trace(K))


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_symmetric_pcg_and_prediction_by_the_oracle(prec):
    N, M = 6, 40
    R, y = case(N, M, 9)
    perms = group(N, "s3")
    sigma, lam = 2.0, 1e-8
    ctx = gdml.kernel_setup(dev(R), sigma, lam, precision=prec, perms=perms)
    ctx.precond_build("pivchol", 200)
    alpha, iters, rel, _ = ctx.pcg_solve(dev(y), rtol=1e-8)
    a = alpha.cpu().numpy()
    K = ok.force_kernel_dense_sym(R, sigma, perms)
    res = np.linalg.norm(y - K @ a - lam * a) / np.linalg.norm(y)
    bound = 8 * EPS * np.linalg.norm(K, 2) * np.linalg.norm(a) / np.linalg.norm(y)
    print(f"{prec} symmetric PCG: {iters} iterations, GPU relres {rel:.2e}, oracle relres {res:.2e}")
    assert rel <= 1e-8 and res <= 1e-8 + bound
    # prediction for query geometries: the symmetric kernel's cross blocks applied to alpha
    Rq = synth.geometries(synth.template(N, 9), 5, 0.2, 77)
    f = ctx.predict_forces(dev(Rq), alpha).cpu().numpy().reshape(-1)
    Kfull = ok.force_kernel_dense_sym(np.concatenate([Rq, R]), sigma, perms)
    nq = Rq.size
    ref = Kfull[:nq, nq:] @ a
    scale = (np.abs(Kfull[:nq, nq:]) @ np.abs(a)).max()
    assert np.abs(f - ref).max() <= 1e-12 * scale
    ctx.destroy()


def test_symmetry_arguments_are_checked():
    R, _ = case(5, 3, 1)
    idn = list(range(5))
    bad = {
        "not a permutation": [idn, [0, 0, 2, 3, 4]],
        "no identity": [[1, 0, 2, 3, 4]],
        "not closed": [idn, [1, 2, 0, 3, 4]],
        "repeated": [idn, idn],
    }
    for why, perms in bad.items():
        with pytest.raises(gdml.GdmlError) as e:
            gdml.kernel_setup(dev(R), 1.0, 1e-6, perms=perms)
        assert e.value.name == "ERR_ARG", why
    for prec in ("df64", "tf32", "bf16"):
        with pytest.raises(gdml.GdmlError) as e:
            gdml.kernel_setup(dev(R), 1.0, 1e-6, precision=prec, perms=[idn, [1, 0, 2, 3, 4]])
        assert e.value.name == "ERR_ARG"
    # the identity alone is the plain kernel
    c1 = gdml.kernel_setup(dev(R), 1.0, 1e-6, perms=[idn])
    c2 = gdml.kernel_setup(dev(R), 1.0, 1e-6)
    v = dev(np.random.default_rng(0).standard_normal(R.size))
    assert torch.equal(c1.matvec(v), c2.matvec(v))
    c1.destroy()
    c2.destroy()
