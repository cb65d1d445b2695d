"""Pins for the oracle's SVD preconditioner, preconditioned spectrum and PCG Lanczos matrix
(Sec. 2.2, Sec. 4.1 / Fig. 3, App. A.1), each against a route independent of its own code:
spectra fixed by construction, the Eckart-Young theorem, the lower bound every Nystrom
preconditioner obeys, and the Ritz values of an explicitly orthonormalised Krylov basis."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import kernel as ok
from oracle import precond as op
from oracle import solver as osv
from oracle import spectrum as osp


def spd_with_spectrum(sig, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((sig.size, sig.size)))
    return (Q * sig) @ Q.T, Q


def test_svd_factor_is_the_best_rank_k_approximation():
    """Eckart-Young: K_k = L_k L_k^T keeps the k largest eigenpairs of the constructed K, and
    |K - K_k|_2 = sigma_(k+1)."""
    sig = np.sort(np.random.default_rng(1).uniform(0.0, 5.0, 30))[::-1].copy()
    K, Q = spd_with_spectrum(sig, 2)
    for k in (1, 7, 29):
        L, s = osp.svd_factor(K, k)
        np.testing.assert_allclose(s, sig[:k], rtol=0, atol=1e-13 * sig[0])
        np.testing.assert_allclose(L @ L.T, (Q[:, :k] * sig[:k]) @ Q[:, :k].T, rtol=0, atol=1e-12 * sig[0])
        np.testing.assert_allclose(np.linalg.norm(K - L @ L.T, 2), sig[k], rtol=0, atol=1e-12 * sig[0])


def test_svd_preconditioned_spectrum_closed_form():
    """P = K_k + lam I removes the k dominant eigenvalues: spec(P^-1 K_lam) is 1 (k times) and
    (sigma_i + lam) / lam for the rest, so cond = (sigma_(k+1) + lam) / lam."""
    sig = np.concatenate([np.logspace(2, -3, 25), np.zeros(5)])
    K, _ = spd_with_spectrum(sig, 3)
    lam = 1e-2
    for k in (3, 10, 24):
        L, _ = osp.svd_factor(K, k)
        mu = osp.preconditioned_eigenvalues(K, lam, L)
        ref = np.sort(np.concatenate([np.ones(k), (sig[k:] + lam) / lam]))
        np.testing.assert_allclose(mu, ref, rtol=1e-9)
        assert osp.condition_number(mu) == pytest.approx((sig[k] + lam) / lam, rel=1e-9)


@pytest.fixture(scope="module")
def molecule():
    from paper_2212_12737_gb300 import synth
    R = synth.geometries(synth.template(6, 21), 12, 0.1, 22)
    return R, ok.force_kernel_dense(R, 2.0)


@pytest.mark.parametrize("rule", ["uniform", "rls", "pivchol"])
def test_every_nystrom_preconditioner_is_bounded_by_the_svd_one(molecule, rule):
    """For a Nystrom approximation K~ (0 <= K~ <= K, rank k) and P = K~ + lam I:
    * P^-1 K_lam e_s = e_s for every selected column s (K~ reproduces K's selected columns),
      so 1 is an eigenvalue of multiplicity >= k, and all eigenvalues are >= 1 (K_lam >= P);
    * some unit x lies in null(K~) and in the span of K's k + 1 dominant eigenvectors, where
      x^T K_lam x / x^T P x >= (sigma_(k+1) + lam) / lam; hence
      cond(P^-1 K_lam) >= (sigma_(k+1) + lam) / lam = cond for the SVD preconditioner.
    The paper observes this ordering (Fig. 3); here it is a theorem the oracle must obey."""
    R, K = molecule
    n = K.shape[0]
    lam, k = 1e-6, 40
    if rule == "uniform":
        S = op.select_uniform(n, k, 2)
    elif rule == "rls":
        S, _ = op.select_rls(lambda idx: K[:, idx], n, k, lam, 2)
    else:
        _, S, _ = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K).copy(), k)
    L, _ = op.nystrom_factor(K[:, S], S)
    mu = osp.preconditioned_eigenvalues(K, lam, L)
    scale = np.abs(K).max() / lam
    assert mu.min() >= 1.0 - 1e-7
    assert np.sum(np.abs(mu - 1.0) <= 1e-6) >= k
    Ls, sig = osp.svd_factor(K, k + 1)
    mu_svd = osp.preconditioned_eigenvalues(K, lam, Ls[:, :k])
    bound = (sig[k] + lam) / lam
    assert osp.condition_number(mu_svd) == pytest.approx(bound, rel=1e-6)
    assert osp.condition_number(mu) >= bound * (1 - 1e-9 * scale / bound)
    print(f"{rule}: cond {osp.condition_number(mu):.3e} >= SVD {bound:.3e}")


def krylov_ritz(A, Pinv, y, m):
    """Ritz values of Ahat = P^-1/2 A P^-1/2 on K_m(Ahat, P^-1/2 y), from an explicit
    orthonormal basis (QR of the Krylov matrix) -- no CG involved."""
    w, V = np.linalg.eigh(Pinv)
    Ph = (V * np.sqrt(w)) @ V.T
    Ah = Ph @ A @ Ph
    cols = [Ph @ y]
    for _ in range(m - 1):
        cols.append(Ah @ cols[-1])
    Kr = np.stack(cols, 1)
    Kr /= np.linalg.norm(Kr, axis=0)
    Q, _ = np.linalg.qr(Kr)
    return np.linalg.eigvalsh(Q.T @ Ah @ Q)


def test_lanczos_matrix_of_pcg_equals_the_krylov_projection():
    rng = np.random.default_rng(5)
    n = 30
    A, _ = spd_with_spectrum(np.logspace(0, -3, n), 6)
    B, _ = spd_with_spectrum(rng.uniform(0.5, 2.0, n), 7)
    y = rng.standard_normal(n)
    for m in (1, 3, 6):
        res = osv.pcg(lambda v: A @ v, lambda v: B @ v, y, rtol=1e-30, max_iter=m, max_restarts=0)
        assert len(res.gammas) == m
        theta = osp.ritz_values(res.gammas, res.betas)
        np.testing.assert_allclose(theta, krylov_ritz(A, B, y, m), rtol=1e-8)


def test_ritz_values_reach_the_extreme_eigenvalues():
    """Run to convergence: the extreme Ritz values equal the extreme eigenvalues of P^-1 A (from
    the construction of A with P = I), and every Ritz value lies between them."""
    sig = np.logspace(1, -2, 40)
    A, _ = spd_with_spectrum(sig, 8)
    y = np.random.default_rng(9).standard_normal(40)
    # finite-precision CG needs more than n steps here (85 for n = 40)
    res = osv.pcg(lambda v: A @ v, lambda v: v, y, rtol=1e-14, max_iter=400, max_restarts=0)
    theta = osp.ritz_values(res.gammas, res.betas)
    assert theta.max() == pytest.approx(sig[0], rel=1e-10)
    assert theta.min() == pytest.approx(sig[-1], rel=1e-8)
    assert theta.max() <= sig[0] * (1 + 1e-12) and theta.min() >= sig[-1] * (1 - 1e-12)


def test_planted_off_diagonal_error_is_caught(monkeypatch):
    """beta_j in place of sqrt(beta_j) on the off-diagonal must break the Krylov pin."""
    good = osp.lanczos_matrix

    def bad(gammas, betas):
        d, e = good(gammas, betas)
        return d, e * e * np.asarray(gammas)[:-1]

    monkeypatch.setattr(osp, "lanczos_matrix", bad)
    with pytest.raises(AssertionError):
        test_lanczos_matrix_of_pcg_equals_the_krylov_projection()


def test_recording_does_not_change_pcg():
    """The coefficients are recorded from the first run only; x and the residuals are those of
    the plain recurrence (checked against the dense solve)."""
    rng = np.random.default_rng(11)
    A, _ = spd_with_spectrum(np.logspace(0, -4, 50), 12)
    y = rng.standard_normal(50)
    res = osv.pcg(lambda v: A @ v, lambda v: v, y, rtol=1e-10, max_iter=500, max_restarts=0)
    x_ref = sla.solve(A, y, assume_a="pos")
    assert np.linalg.norm(res.x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    assert len(res.gammas) == res.iters and len(res.betas) == res.iters - 1
