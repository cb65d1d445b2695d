"""Oracle: Nystrom-type preconditioner (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

* P = L_k L_k^T + lam I_n                                  (Eq. 3)
* P^-1 = lam^-1 [I - L_k (lam I_k + L_k^T L_k)^-1 L_k^T]   (Eq. 4)
* Nystrom: K ~ K_nk K_kk^-1 K_nk^T, K_kk = L_kk L_kk^T,
  L_k = K_nk L_kk^-T                                       (Eq. 5)
* column selection (Sec. 3, "Column selection strategies"): uniform,
  ridge leverage scores tau_i = (K (K + lam I)^-1)_ii, incomplete (pivoted)
  Cholesky (App. A.2, Algorithm 1).

Readings where the paper is silent:
* uniform sampling is without replacement: the k smallest Philox keys;
* the "approximation" of ridge leverage scores is the Nystrom estimate from a
  uniform pilot set of size k: tau~_i = b_i^T (B^T B + lam I)^-1 b_i with
  B = K_nS L_S^-T; sampling without replacement proportional to tau~ takes
  the k smallest keys -ln(u_i)/tau~_i (Efraimidis-Spirakis);
* the K_kk factorisation retries with jitter eps = 1e-14 tr(K_kk)/k, times 10
  per retry, up to 1e-6 tr(K_kk)/k, when Cholesky fails;
* Algorithm 1 breaks ties in the argmax towards the lowest position, and
  stops early (returning the rank reached) when the largest residual
  diagonal is <= 0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import philox


def select_uniform(n: int, k: int, seed: int, stream: int = philox.STREAM_UNIFORM) -> np.ndarray:
    """Uniform column sampling (Sec. 3), without replacement: k distinct columns, the indices
    of the k smallest uniforms, ordered by key then index."""
    if not 0 < k <= n:
        raise ValueError("need 0 < k <= n")
    u = philox.uniforms(n, seed, stream)
    order = np.lexsort((np.arange(n), u))
    return order[:k].astype(np.int64)


def cholesky_jitter(A: np.ndarray) -> tuple[np.ndarray, float]:
    """Lower Cholesky factor of A, retrying with diagonal jitter (Eq. 5 reading): eps =
    1e-14 tr(A)/k, times 10 per retry, up to 1e-6 tr(A)/k.  A matrix whose trace is not
    positive gives the rule no scale (it cannot be a nonzero PSD block): it fails at once."""
    k = A.shape[0]
    scale = np.trace(A) / k
    eps = 0.0
    while True:
        try:
            L = np.linalg.cholesky(A + eps * np.eye(k))
            return L, eps
        except np.linalg.LinAlgError:
            if not (scale > 0.0 and np.isfinite(scale)):
                raise
            eps = 1e-14 * scale if eps == 0.0 else eps * 10.0
            if eps > 1e-6 * scale * 1.0000001:
                raise


def nystrom_factor(K_nk: np.ndarray, S: np.ndarray) -> tuple[np.ndarray, float]:
    """L_k = K_nk L_kk^-T with K_kk = K_nk[S] = L_kk L_kk^T (Eq. 5)."""
    L_kk, eps = cholesky_jitter(K_nk[S, :])
    L_k = sla.solve_triangular(L_kk, K_nk.T, lower=True).T
    return L_k, eps


def woodbury_core(L_k: np.ndarray, lam: float) -> np.ndarray:
    """Lower Cholesky factor of C = lam I_k + L_k^T L_k (Eq. 4)."""
    C = lam * np.eye(L_k.shape[1]) + L_k.T @ L_k
    return np.linalg.cholesky(C)


def woodbury_apply(L_k: np.ndarray, L_C: np.ndarray, lam: float, r: np.ndarray) -> np.ndarray:
    """z = P^-1 r = lam^-1 [r - L_k C^-1 L_k^T r] (Eq. 4)."""
    t = L_k.T @ r
    t = sla.solve_triangular(L_C, t, lower=True)
    t = sla.solve_triangular(L_C.T, t, lower=False)
    return (r - L_k @ t) / lam


def precond_matrix(L_k: np.ndarray, lam: float) -> np.ndarray:
    """Dense P = L_k L_k^T + lam I (Eq. 3); tiny cases only."""
    return L_k @ L_k.T + lam * np.eye(L_k.shape[0])


def pivoted_cholesky(get_col, d: np.ndarray, k: int, forced=None, diag_out: list | None = None):
    """Incomplete Cholesky with greedy diagonal pivoting (App. A.2, Algorithm 1).

    get_col(i) returns column i of K; d = diag(K).  Returns (L_k, pivots,
    trace) where trace[m] = sum of the residual diagonal after step m and
    pivots lists the chosen columns in order.  Stops early if the largest
    residual diagonal is not positive (rank reached).

    forced (optional): a sequence of column indices taken as the pivots of steps 0, 1, ...
    instead of the argmax (to replay another implementation's choices; a forced column must
    not have been chosen before).  diag_out (optional list): receives, before each step, the
    residual diagonal d as it stands (a copy), so a replay can compare each forced pivot
    with that step's maximum.
    """
    d = np.array(d, dtype=np.float64, copy=True)
    n = d.size
    perm = np.arange(n)
    pos = np.arange(n)  # position of each column in perm
    L = np.zeros((n, k), order="F")  # columns contiguous
    trace = []
    for m in range(k):
        if diag_out is not None:
            diag_out.append(d.copy())
        # pivot: largest residual diagonal among the not-yet-chosen positions
        rest = perm[m:]
        if forced is None:
            i = m + int(np.argmax(d[rest]))
        else:
            i = int(pos[int(forced[m])])
            if i < m:
                raise ValueError(f"forced pivot {forced[m]} at step {m} was chosen before")
        if d[perm[i]] <= 0.0:
            return L[:, :m], perm[:m].copy(), np.asarray(trace)
        perm[m], perm[i] = perm[i], perm[m]
        pos[perm[m]], pos[perm[i]] = m, i
        piv = perm[m]
        lmm = np.sqrt(d[piv])
        L[piv, m] = lmm
        col = get_col(piv)
        rest = perm[m + 1:]
        # Schur correction s = sum_{j < m} l_{piv, j} * l_{rest, j}, summed in
        # the order j = 0, 1, ..., m-1 (column m is still zero, so the sum to
        # j = m in the paper's listing is the same sum)
        s = np.zeros(n)
        for j in range(m):
            s += L[piv, j] * L[:, j]
        L[rest, m] = (col[rest] - s[rest]) / lmm
        d[rest] -= L[rest, m] ** 2
        trace.append(float(np.sum(d[rest])))
    return L, perm[:k].copy(), np.asarray(trace)


def rls_exact(K: np.ndarray, lam: float) -> np.ndarray:
    """Exact ridge leverage scores tau_i = (K (K + lam I)^-1)_ii (Sec. 3); tiny n."""
    n = K.shape[0]
    return np.diag(K @ np.linalg.inv(K + lam * np.eye(n))).copy()


def rls_nystrom(K_nS: np.ndarray, S: np.ndarray, lam: float) -> np.ndarray:
    """Nystrom estimate of the ridge leverage scores from pilot columns S (Sec. 3, leverage
    score sampling).

    B = K_nS L_S^-T (so B B^T is the Nystrom approximation of K) and
    tau~_i = b_i^T (B^T B + lam I)^-1 b_i.
    """
    B, _ = nystrom_factor(K_nS, S)
    G = np.linalg.cholesky(B.T @ B + lam * np.eye(B.shape[1]))
    Z = sla.solve_triangular(G, B.T, lower=True)
    return np.sum(Z * Z, axis=0)


def select_weighted(tau: np.ndarray, k: int, seed: int,
                    stream: int = philox.STREAM_RLS_SAMPLE) -> np.ndarray:
    """Weighted column sampling (Sec. 3): k distinct indices sampled without replacement with
    weights tau (Efraimidis-Spirakis).

    Key_i = -ln(u_i) / tau_i (inf if tau_i <= 0); the k smallest keys, ties by index.
    """
    n = tau.size
    u = philox.uniforms(n, seed, stream)
    with np.errstate(divide="ignore"):
        key = np.where(tau > 0.0, -np.log(u) / np.where(tau > 0.0, tau, 1.0), np.inf)
    order = np.lexsort((np.arange(n), key))
    return order[:k].astype(np.int64)


def select_rls(get_cols, n: int, k: int, lam: float, seed: int):
    """Ridge-leverage-score column selection (Sec. 3): pilot Nystrom estimate, then sampling.

    get_cols(S) returns K[:, S].  Returns (indices, tau~).
    """
    S0 = select_uniform(n, k, seed, philox.STREAM_RLS_PILOT)
    tau = rls_nystrom(get_cols(S0), S0, lam)
    return select_weighted(tau, k, seed), tau
