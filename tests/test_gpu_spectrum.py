"""The SVD preconditioner and the spectrum diagnostics on the GPU against the oracle
(Sec. 2.2, Sec. 4.1 / Fig. 3, App. A.1; the oracle's formulas are pinned in test_oracle_spectrum.py).

* SVD preconditioner: its factor is unique only up to a basis of each eigenspace, so the test
  checks what is unique -- L_k^T L_k = Sigma_k with Sigma_k the oracle's k largest eigenvalues
  of K, the eigen-relation K L_k = L_k Sigma_k with the oracle's dense K, and the residual
  trace -- each within the dense eigensolver's error (FP64 contexts) or the FP32 storage of
  L_k (OZAKI contexts);
* the Ritz values of the PCG run against the spectrum of the same P^-1 K_lam (P from the
  GPU's own stored factor) computed densely by the oracle: the largest within 1e-6, the
  smallest within 1e-6 (FP64) or inside the eigenvalue cluster at 1 (OZAKI), every Ritz value
  between them, and the SVD preconditioner's condition number no larger
  than any Nystrom preconditioner's (the bound pinned in the oracle tests);
* argument and call-order errors.
"""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from oracle import spectrum as osp
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu

SIGMA, LAM, K_IND = 2.0, 1e-6, 80


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


@pytest.fixture(scope="module")
def system():
    """N = 6 atoms, M = 100 geometries (n = 1800): small enough for dense eigensolves."""
    tm = synth.template(6, 31)
    R = synth.geometries(tm, 100, 0.1, 32)
    y = synth.morse_forces(R, tm).reshape(-1)
    K = ok.force_kernel_dense(R, SIGMA)
    w, _ = np.linalg.eigh(K)
    return R, y, K, w


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_svd_preconditioner_factor(system, prec):
    R, _, K, w = system
    n, k = K.shape[0], K_IND
    ctx = gdml.kernel_setup(dev(R), SIGMA, LAM, precision=prec)
    piv, tr = ctx.precond_build("svd", k, pivots=True, trace=True)
    rank, jit = ctx.precond_info()
    L = ctx.precond_factor().cpu().numpy()
    ctx.destroy()
    assert rank == k and jit == 0.0 and L.shape == (n, k)
    assert np.all(piv.cpu().numpy() == -1)
    sig = w[::-1][:k]
    smax = w[-1]
    # FP64: syevd's backward error ~ n eps |K|; OZAKI: L rounded to FP32 (relative 2^-24 per entry)
    tol = 1e-10 if prec == "fp64" else 2e-7
    G = L.T @ L
    np.testing.assert_allclose(np.diag(G), sig, rtol=0, atol=tol * smax)
    assert np.abs(G - np.diag(np.diag(G))).max() <= tol * smax
    resid = K @ L - L * sig
    assert np.abs(resid).max() <= tol * smax * np.abs(L).max() * 10
    # resid_trace[m] = sum of the eigenvalues below the m + 1 largest
    ref_tr = np.array([w[: n - 1 - m].sum() for m in range(k)])
    np.testing.assert_allclose(tr.cpu().numpy(), ref_tr, rtol=0, atol=1e-10 * np.trace(K))


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_pcg_ritz_values_match_the_preconditioned_spectrum(system, prec):
    R, y, K, _ = system
    ctx = gdml.kernel_setup(dev(R), SIGMA, LAM, precision=prec)
    conds = {}
    for rule in ("uniform", "rls", "pivchol", "svd"):
        ctx.precond_build(rule, K_IND, seed=2)
        L = ctx.precond_factor().cpu().numpy()
        _, iters, rel, _ = ctx.pcg_solve(dev(y), rtol=1e-10)
        tmin, tmax, m, top = ctx.pcg_spectrum(16)
        mu = osp.preconditioned_eigenvalues(K, LAM, L)
        print(f"{prec} {rule}: {iters} iterations ({m} recorded), theta [{tmin:.10f}, {tmax:.6e}], "
              f"mu [{mu.min():.10f}, {mu.max():.6e}]")
        assert rel <= 1e-10 and 1 <= m <= iters
        # the largest Ritz value approaches mu_max from below, the smallest mu_min from above.
        # Nystrom and SVD preconditioners put >= k eigenvalues at exactly 1 (FP64 factor); the
        # FP32-stored factor of OZAKI contexts spreads that cluster over ~1e-4, and the Lanczos
        # process resolves the cluster, not its lowest member.  OZAKI contexts apply P^-1 through
        # a k x k core with its own rounding, so their operator differs from the dense one by
        # ~1e-9 relative at the top of the spectrum
        assert mu.max() * (1 - 1e-6) <= tmax <= mu.max() * (1 + (1e-9 if prec == "fp64" else 1e-6))
        assert mu.min() - 1e-7 <= tmin <= mu.min() + (1e-6 if prec == "fp64" else 1e-3)
        assert top[0] == tmax and np.all(np.diff(top) <= 0)
        assert np.all((top >= tmin) & (top <= tmax))
        conds[rule] = tmax / tmin
    ctx.destroy()
    for rule in ("uniform", "rls", "pivchol"):
        assert conds["svd"] <= conds[rule] * (1 + 1e-6), conds


def test_spectrum_call_order_and_arguments(system):
    R, y, _, _ = system
    ctx = gdml.kernel_setup(dev(R), SIGMA, LAM)
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_spectrum()
    assert e.value.name == "ERR_STATE"
    ctx.pcg_solve(dev(y), rtol=1e-6)
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_spectrum(1025)
    assert e.value.name == "ERR_ARG"
    t0 = ctx.pcg_spectrum(3)
    assert t0[2] >= 1 and np.isfinite(t0[:2]).all()
    # a right-hand side of zeros takes no CG step: nothing recorded
    ctx.pcg_solve(torch.zeros_like(dev(y)))
    with pytest.raises(gdml.GdmlError) as e:
        ctx.pcg_spectrum()
    assert e.value.name == "ERR_STATE"
    ctx.destroy()
    # the SVD preconditioner is for small n only (a dense eigendecomposition of K)
    big = synth.geometries(synth.template(9, 1), 1000, 0.05, 2)  # n = 27000
    ctx = gdml.kernel_setup(dev(big), 10.0, 1e-6)
    with pytest.raises(gdml.GdmlError) as e:
        ctx.precond_build("svd", 10)
    assert e.value.name == "ERR_ARG"
    ctx.destroy()
