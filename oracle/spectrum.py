"""Oracle: the SVD preconditioner and the spectrum of the preconditioned matrix (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

* SVD preconditioner (Sec. 2.2 and App. A.1): K = U Sigma U^T is PSD, so its SVD is its
  eigendecomposition; the optimal rank-k approximation keeps the k dominant eigenpairs,
  K_k = U_k Sigma_k U_k^T, and P = K_k + lam I.  Written as P = L_k L_k^T + lam I with
  L_k = U_k Sigma_k^(1/2) it is applied by the same Woodbury identity (Eq. 4) as the
  Nystrom preconditioners.
* Preconditioned spectrum (Sec. 4.1, Fig. 3): the eigenvalues of P^-1 K_lam, which are those
  of the symmetric-definite pencil (K_lam, P); the condition number is their max / min.
* Lanczos matrix of PCG (a standard identity, e.g. Saad, "Iterative Methods for Sparse
  Linear Systems", Sec. 6.7.3): the CG step lengths gamma_j and ratios beta_j define the
  tridiagonal matrix T_m of the Lanczos process on P^-1 K_lam started from P^-1 y,
      T[0, 0] = 1 / gamma_0,  T[j, j] = 1 / gamma_j + beta_(j-1) / gamma_(j-1),
      T[j, j+1] = T[j+1, j] = sqrt(beta_j) / gamma_j,
  whose eigenvalues (Ritz values) lie in [mu_min, mu_max] of P^-1 K_lam and approach its
  extreme eigenvalues as the iteration proceeds.  This is how the library estimates the
  condition number from a solve at sizes where no dense eigendecomposition is possible.

Readings: where eigenvalues tie at the cut (sigma_k = sigma_(k+1)) the rank-k SVD
approximation is not unique; eigh's ascending order decides, and tests compare only
basis-independent quantities (eigenvalues, the eigen-relation, spectra of P^-1 K_lam).
Negative eigenvalues of K from rounding (K is PSD) are clamped to 0 in Sigma_k^(1/2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def svd_factor(K: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """(L_k, sigma_k): L_k = U_k Sigma_k^(1/2) (n x k) from the k largest eigenpairs of K,
    columns in descending eigenvalue order; sigma_k the k eigenvalues (App. A.1)."""
    w, U = np.linalg.eigh(K)
    idx = np.arange(K.shape[0] - 1, K.shape[0] - 1 - k, -1)
    sig = w[idx]
    return U[:, idx] * np.sqrt(np.maximum(sig, 0.0)), sig


def preconditioned_eigenvalues(K: np.ndarray, lam: float, L_k: np.ndarray) -> np.ndarray:
    """Ascending eigenvalues of P^-1 K_lam for P = L_k L_k^T + lam I (Eq. 3), from the
    symmetric-definite generalized eigenproblem K_lam x = mu P x."""
    n = K.shape[0]
    P = L_k @ L_k.T + lam * np.eye(n)
    return sla.eigh(K + lam * np.eye(n), P, eigvals_only=True)


def condition_number(mu: np.ndarray) -> float:
    """cond(P^-1 K_lam) = mu_max / mu_min of its (positive) eigenvalues."""
    return float(mu.max() / mu.min())


def lanczos_matrix(gammas, betas) -> tuple[np.ndarray, np.ndarray]:
    """Diagonal and off-diagonal of T_m from m CG step lengths gamma_0..gamma_(m-1) and the
    ratios beta_0..beta_(m-2) (the first m - 1 of any longer list are used)."""
    g = np.asarray(gammas, dtype=np.float64)
    m = g.size
    b = np.asarray(betas, dtype=np.float64)[: max(m - 1, 0)]
    diag = 1.0 / g
    diag[1:] += b / g[:-1]
    off = np.sqrt(b) / g[:-1]
    return diag, off


def ritz_values(gammas, betas) -> np.ndarray:
    """Ascending eigenvalues of T_m (the Ritz values of P^-1 K_lam after m PCG steps)."""
    d, e = lanczos_matrix(gammas, betas)
    if d.size == 0:
        return d
    return sla.eigh_tridiagonal(d, e, eigvals_only=True)
