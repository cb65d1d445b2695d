"""Pins for the oracle's random numbers, column selection, Nystrom factor and Woodbury apply (Sec. 3, Eqs. 3-5, Alg. 1)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.linalg import lapack

from oracle import kernel as ok
from oracle import philox
from oracle import precond as op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def spd(n, seed, decay=0.7):
    """Random SPD test matrix with a decaying spectrum."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * decay ** np.arange(n)) @ Q.T


# ---- Philox4x32-10 -------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(np.array([v[:4]], dtype=np.uint64), np.array([v[4:6]], dtype=np.uint64))
        assert [int(x) for x in out[0]] == v[6:]


def test_uniform_selection_distinct_and_unbiased():
    n, k, seeds = 40, 4, 3000
    counts = np.zeros(n)
    for s in range(seeds):
        S = op.select_uniform(n, k, s)
        assert len(set(S.tolist())) == k and S.min() >= 0 and S.max() < n
        counts[S] += 1
    from scipy.stats import chisquare
    assert chisquare(counts).pvalue > 1e-4


def test_uniform_selection_is_k_smallest_keys():
    u = philox.uniforms(1000, 7, philox.STREAM_UNIFORM)
    S = op.select_uniform(1000, 25, 7)
    assert np.array_equal(S, np.argsort(u, kind="stable")[:25])
    assert np.all((u > 0) & (u <= 1))


def test_weighted_selection_equal_weights_takes_largest_uniforms():
    u = philox.uniforms(500, 5, philox.STREAM_RLS_SAMPLE)
    S = op.select_weighted(np.full(500, 0.3), 20, 5)
    assert np.array_equal(S, np.argsort(-u, kind="stable")[:20])
    # zero weight is never picked while positive weights remain
    tau = np.ones(500); tau[::2] = 0.0
    assert np.all(op.select_weighted(tau, 100, 5) % 2 == 1)


def test_weighted_selection_first_pick_is_proportional_to_weight():
    """Efraimidis-Spirakis: the smallest key -ln(u_i)/tau_i is index i with probability
    tau_i / sum(tau).  Over many seeds the first pick's counts fit those probabilities (chi^2);
    a key with the wrong power of tau (e.g. -ln(u)/tau^2, giving tau^2 / sum tau^2) fails."""
    from scipy.stats import chisquare
    tau = np.array([1.0, 2.0, 3.0, 4.0, 10.0])
    seeds = 4000
    counts = np.zeros(tau.size)
    for s in range(seeds):
        counts[op.select_weighted(tau, 1, s)[0]] += 1
    assert chisquare(counts, seeds * tau / tau.sum()).pvalue > 1e-4
    assert chisquare(counts, seeds * tau ** 2 / (tau ** 2).sum()).pvalue < 1e-12
    # without replacement: the second pick, given the first, is proportional to the rest
    pair = np.zeros((tau.size, tau.size))
    for s in range(seeds):
        a, b = op.select_weighted(tau, 2, s)
        assert a != b
        pair[a, b] += 1
    first = 4  # the heaviest weight is picked first often enough to test its row
    rest = np.delete(np.arange(tau.size), first)
    row = pair[first, rest]
    assert chisquare(row, row.sum() * tau[rest] / tau[rest].sum()).pvalue > 1e-4


# ---- Woodbury and Nystrom (Eqs. 3-5) --------------------------------------

def test_woodbury_inverts_dense_p():
    rng = np.random.default_rng(4)
    L = rng.standard_normal((60, 9))
    for lam in (1e-3, 1e-8):
        LC = op.woodbury_core(L, lam)
        P = op.precond_matrix(L, lam)
        r = rng.standard_normal(60)
        z = op.woodbury_apply(L, LC, lam, r)
        # Eq. 4 subtracts nearly equal vectors and scales by 1/lam: its error
        # grows like eps * |L^T L| / lam, which sets the tolerance
        amp = max(1.0, np.linalg.norm(L, 2) ** 2 / lam)
        np.testing.assert_allclose(P @ z, r, rtol=0, atol=64 * np.finfo(float).eps * amp * np.linalg.norm(r))
        if lam >= 1e-3:
            ref = np.linalg.solve(P, r)
            np.testing.assert_allclose(z, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_nystrom_reproduces_inducing_columns(tiny):
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.2)
    S = op.select_uniform(K.shape[0], 12, 3)
    L, eps = op.nystrom_factor(K[:, S], S)
    assert eps == 0.0
    np.testing.assert_allclose((L @ L.T)[:, S], K[:, S], atol=1e-10 * np.abs(K).max())


def test_cholesky_jitter_retries_on_singular_block():
    A = np.ones((4, 4))  # rank 1
    L, eps = op.cholesky_jitter(A)
    assert eps > 0 and np.allclose(L @ L.T, A + eps * np.eye(4))


# ---- Algorithm 1: pivoted (incomplete) Cholesky ----------------------------

def test_pivoted_cholesky_full_rank_equals_lapack_dpstrf():
    A = spd(30, 5)
    L, piv, tr = op.pivoted_cholesky(lambda i: A[:, i], np.diag(A), 30)
    c, lp, rank, info = lapack.dpstrf(A, lower=1, tol=-1.0)
    assert rank == 30
    assert np.array_equal(piv, lp - 1)
    np.testing.assert_allclose(L[piv, :], np.tril(c), atol=1e-12)


def test_pivoted_cholesky_steps_match_explicit_schur_complements(tiny):
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.2)
    n, k = K.shape[0], 15
    L, piv, tr = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k)
    for m in range(k):
        P = piv[:m]
        Sch = K - K[:, P] @ np.linalg.solve(K[np.ix_(P, P)], K[P, :]) if m else K
        dS = np.diag(Sch).copy(); dS[P] = -np.inf
        assert piv[m] == int(np.argmax(dS)) or dS[piv[m]] >= dS.max() * (1 - 1e-9)
        rest = np.setdiff1d(np.arange(n), piv[:m + 1])
        assert abs(tr[m] - np.sum(np.diag(Sch)[rest] - (Sch[rest, piv[m]] ** 2) / Sch[piv[m], piv[m]])) <= 1e-9 * np.trace(K)
    assert np.all(np.diff(tr) <= 1e-15 * np.trace(K))
    assert piv[0] == int(np.argmax(np.diag(K)))
    np.testing.assert_allclose((L @ L.T)[:, piv], K[:, piv], atol=1e-10 * np.abs(K).max())


def test_pivoted_cholesky_forced_replay_reproduces_free_run(tiny):
    """Forcing Algorithm 1's own free choices reproduces it exactly (same factor, pivots,
    trace), and the recorded residual diagonals are those the free run took its argmax of;
    forcing a different (valid) column changes the factor and is checked like any other."""
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.2)
    k = 12
    diags = []
    L, piv, tr = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k, diag_out=diags)
    L2, piv2, tr2 = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k, forced=piv)
    assert np.array_equal(piv2, piv) and np.array_equal(L2, L) and np.array_equal(tr2, tr)
    assert len(diags) == k and np.array_equal(diags[0], np.diag(K))
    for m in range(k):
        dm = diags[m].copy()
        dm[piv[:m]] = -np.inf
        assert piv[m] == int(np.argmax(dm))
    other = list(piv)
    other[3] = int(np.setdiff1d(np.arange(K.shape[0]), piv)[0])
    L3, piv3, _ = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k, forced=other)
    assert np.array_equal(piv3, other)
    np.testing.assert_allclose((L3 @ L3.T)[:, piv3], K[:, piv3], atol=1e-10 * np.abs(K).max())
    with pytest.raises(ValueError):
        op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), 3, forced=[piv[0], piv[1], piv[0]])


def test_cholesky_jitter_rule():
    """The jitter reading of Eq. 5's factorisation: none for SPD, eps = 1e-14 tr/k for an
    exactly singular PSD matrix, failure for indefinite ones (also with tr <= 0)."""
    A = spd(6, 2)
    L, eps = op.cholesky_jitter(A)
    assert eps == 0.0 and np.allclose(L @ L.T, A, atol=1e-14)
    S = np.diag([3.0, 2.0, 1.0, 0.0])
    L, eps = op.cholesky_jitter(S)
    assert eps == pytest.approx(1e-14 * 6.0 / 4) and np.allclose(L @ L.T, S + eps * np.eye(4), atol=1e-15)
    for A in (np.diag([2.0, -1.0]), np.diag([1.0, -1.0]), np.diag([-1.0, -2.0]), np.zeros((2, 2))):
        with pytest.raises(np.linalg.LinAlgError):
            op.cholesky_jitter(A)


def test_nystrom_on_pivots_equals_incomplete_cholesky(tiny):
    """Sec. 3: Nystrom with the same inducing columns is the incomplete Cholesky."""
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.2)
    L, piv, _ = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), 10)
    Ln, _ = op.nystrom_factor(K[:, piv], piv)
    np.testing.assert_allclose(Ln @ Ln.T, L @ L.T, atol=1e-10 * np.abs(K).max())


def test_pivoted_cholesky_stops_at_numerical_rank():
    rng = np.random.default_rng(6)
    G = rng.standard_normal((20, 3))
    A = G @ G.T
    L, piv, tr = op.pivoted_cholesky(lambda i: A[:, i], np.diag(A), 20)
    assert L.shape[1] <= 20 and np.allclose(L @ L.T, A, atol=1e-10)


# ---- ridge leverage scores -------------------------------------------------

def test_ridge_leverage_scores_bounds_sum_and_nystrom_limit(tiny):
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.2)
    n = K.shape[0]
    lam = 1e-3
    tau = op.rls_exact(K, lam)
    ev = np.linalg.eigvalsh(K)
    assert np.all(tau >= -1e-12) and np.all(tau <= 1 + 1e-12)
    assert abs(tau.sum() - np.sum(ev / (ev + lam))) <= 1e-9 * n
    # with every column as pilot the estimate is exact (up to the jitter of a singular K_SS)
    piv = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), n)[1]
    full = piv[: np.sum(ev > 1e-10 * ev.max())]
    est = op.rls_nystrom(K[:, full], full, lam)
    np.testing.assert_allclose(est, tau, atol=1e-7)
    S = op.select_uniform(n, 10, 1)
    est = op.rls_nystrom(K[:, S], S, lam)
    assert np.all(est >= 0) and np.all(est <= 1 + 1e-12) and np.all(est <= tau + 1e-9)


def test_select_rls_returns_distinct_indices(tiny):
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.2)
    S, tau = op.select_rls(lambda idx: K[:, idx], K.shape[0], 8, 1e-6, 9)
    assert len(set(S.tolist())) == 8 and tau.shape == (K.shape[0],)
