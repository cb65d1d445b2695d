"""Failure statuses of the C ABI on the GPU, each caused from the host -- no GPU fault, trap
or endless wait is provoked:

* GDML_ERR_NOT_SPD and the jitter retries of the K_kk factorisation (the reading of Eq. 5's
  "numerical considerations"): the library's Cholesky on caller matrices that are exactly
  singular (one retry) or indefinite (every retry fails), and a preconditioner whose
  inducing columns are all 3N columns of one geometry (K_kk = (c^2/3) J^T J contains the
  rigid motions of that geometry in its null space);
* GDML_ERR_BREAKDOWN of PCG (Eq. 2 needs p^T K_lambda p > 0): lambda replaced by a negative
  value through a test hook, so that K + lambda I is negative definite;
* GDML_ERR_TIMEOUT of the bounded device waits: a host-set poll limit of 0 makes every wait
  of the tcgen05 / TMA pipelines give up before its role issues any copy or MMA; the error
  word reports it and the context keeps working once the limit is restored;
* GDML_ERR_ARG for non-finite right-hand sides and geometries with coincident atoms.
"""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from oracle import precond as op
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


def small(M=12, N=6, seed=4):
    tmpl = synth.template(N, seed)
    R = synth.geometries(tmpl, M, 0.1, seed + 1)
    return R, synth.morse_forces(R, tmpl).reshape(-1)


def test_cholesky_jitter_retry_and_not_spd():
    # positive definite: no jitter, the factor of A itself
    A = np.array([[4.0, 2.0, 0.0], [2.0, 5.0, 1.0], [0.0, 1.0, 3.0]])
    L, eps = gdml.test_cholesky_jitter(dev(A))
    assert eps == 0.0
    np.testing.assert_allclose(L.cpu().numpy(), np.linalg.cholesky(A), rtol=0, atol=1e-15)
    # exactly singular: the first retry, eps = 1e-14 tr(A)/k, succeeds (as in the oracle)
    A = np.diag([2.0, 1.0, 0.0])
    L, eps = gdml.test_cholesky_jitter(dev(A))
    _, eps_ref = op.cholesky_jitter(A)
    assert eps == pytest.approx(1e-14 * np.trace(A) / 3, rel=1e-12) and eps == pytest.approx(eps_ref, rel=1e-12)
    L = L.cpu().numpy()
    np.testing.assert_allclose(L @ L.T, A + eps * np.eye(3), rtol=0, atol=1e-15)
    # indefinite: every retry up to 1e-6 tr/k fails; with tr <= 0 the rule has no scale and
    # fails at once
    for A in (np.diag([2.0, -1.0]), np.diag([1.0, -1.0]), np.diag([-1.0, -2.0])):
        with pytest.raises(gdml.GdmlError) as e:
            gdml.test_cholesky_jitter(dev(A))
        assert e.value.name == "ERR_NOT_SPD"
        with pytest.raises(np.linalg.LinAlgError):
            op.cholesky_jitter(A)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_inducing_block_of_one_geometry_is_factorised_with_jitter(prec):
    """All 3N columns of geometry 0 as inducing columns: K_kk = (c^2/3) J_0^T J_0 is singular
    (translations are exact null vectors of J_0).  The build must succeed -- with the jitter
    rule's eps in [1e-14, 1e-6] tr/k whenever its Cholesky meets the singularity -- and the
    preconditioner built on it must still take PCG to rtol."""
    R, y = small()
    M, N = R.shape[:2]
    sigma, lam = 2.0, 1e-6
    ctx = gdml.kernel_setup(dev(R), sigma, lam, precision=prec)
    scores = torch.zeros(M, dtype=torch.float64, device="cuda")
    scores[0] = 1.0
    piv = ctx.precond_build_scored(scores, 3 * N, pivots=True).cpu().numpy()
    rank, jit = ctx.precond_info()
    assert sorted(piv.tolist()) == list(range(3 * N)) and rank == 3 * N
    K = ok.force_kernel_dense(R, sigma)
    Kkk = K[np.ix_(piv, piv)]
    scale = np.trace(Kkk) / (3 * N)
    ev = np.linalg.eigvalsh(Kkk) / np.abs(Kkk).max()
    print(f"{prec}: jitter {jit:.3e} ({jit / scale:.1e} tr/k); K_kk eigenvalues / max|K_kk| from {ev[:4]}")
    assert abs(ev[:3]).max() <= 1e-13  # the three translations
    assert jit == 0.0 or 1e-14 * scale * (1 - 1e-9) <= jit <= 1e-6 * scale * (1 + 1e-9)
    z = ctx.precond_apply(dev(y)).cpu().numpy()
    assert np.all(np.isfinite(z))
    alpha, iters, rel, _ = ctx.pcg_solve(dev(y), rtol=1e-8)
    a = alpha.cpu().numpy()
    assert rel <= 1e-8
    assert np.linalg.norm(y - K @ a - lam * a) <= 2e-8 * np.linalg.norm(y)
    ctx.destroy()


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_pcg_breakdown_on_an_indefinite_operator(prec):
    R, y = small()
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision=prec)
    ctx.test_set_lambda(-1e3)  # |K| is O(1): K + lambda I is negative definite
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_solve(dev(y), rtol=1e-8)
    assert e.value.name == "ERR_BREAKDOWN"
    ctx.test_set_lambda(1e-6)  # the context solves normally again
    ctx.precond_build("pivchol", 40)
    alpha, iters, rel, _ = ctx.pcg_solve(dev(y), rtol=1e-8)
    assert rel <= 1e-8
    ctx.destroy()


def test_non_finite_inputs_are_rejected():
    R, y = small()
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6)
    bad = y.copy()
    bad[5] = np.nan
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_solve(dev(bad))
    assert e.value.name == "ERR_ARG"
    ctx.destroy()
    R2 = R.copy()
    R2[3, 2] = R2[3, 4]  # two atoms of geometry 3 at one place: 1/r is infinite
    with pytest.raises(gdml.GdmlError) as e:
        gdml.kernel_setup(dev(R2), 2.0, 1e-6)
    assert e.value.name == "ERR_ARG"
    R2 = R.copy()
    R2[0, 0, 1] = np.inf
    with pytest.raises(gdml.GdmlError) as e:
        gdml.kernel_setup(dev(R2), 2.0, 1e-6, precision="ozaki")
    assert e.value.name == "ERR_ARG"


@pytest.mark.parametrize("prec", ["ozaki", "bf16"])
def test_bounded_wait_timeout_is_reported_and_the_context_survives(prec):
    """Poll limit 0: the matvec's tcgen05 pipelines give up before issuing any copy or MMA,
    gdml_tc_check reports GDML_ERR_TIMEOUT, and with the limit restored the same context
    computes the matvec again (checked against the oracle)."""
    R, _ = small(M=40)
    sigma, lam = 2.0, 1e-6
    ctx = gdml.kernel_setup(dev(R), sigma, lam, precision=prec)
    v = np.random.default_rng(1).standard_normal(R.size)
    ref = ok.matvec(R, sigma, v, lam)
    try:
        gdml.test_set_wait_limit(0)
        ctx.matvec(dev(v))
        with pytest.raises(gdml.GdmlError) as e:
            ctx.tc_check()
        assert e.value.name == "ERR_TIMEOUT"
    finally:
        gdml.test_set_wait_limit(None)
    got = ctx.matvec(dev(v)).cpu().numpy()
    ctx.tc_check()
    tol = 1e-12 if prec == "ozaki" else 5e-2
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    ctx.destroy()


def test_staged_pass_timeout_is_reported_and_the_context_survives():
    """The TMA-staged Woodbury passes of an OZAKI context (n % 4 == 0): poll limit 0 makes
    their producer give up before its first copy; the apply reports GDML_ERR_TIMEOUT through
    gdml_tc_check and, with the limit restored, equals the apply computed before."""
    R, _ = small(M=40)
    assert R.size % 4 == 0
    ctx = gdml.kernel_setup(dev(R), 2.0, 1e-6, precision="ozaki")
    ctx.precond_build("pivchol", 60)
    r = dev(np.random.default_rng(2).standard_normal(R.size))
    z0 = ctx.precond_apply(r).cpu().numpy()
    ctx.tc_check()
    try:
        gdml.test_set_wait_limit(0)
        ctx.precond_apply(r)
        with pytest.raises(gdml.GdmlError) as e:
            ctx.tc_check()
        assert e.value.name == "ERR_TIMEOUT"
    finally:
        gdml.test_set_wait_limit(None)
    z1 = ctx.precond_apply(r).cpu().numpy()
    ctx.tc_check()
    assert np.array_equal(z0, z1)
    ctx.destroy()
