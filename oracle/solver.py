"""Oracle: exact solve and preconditioned conjugate gradients (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

* K_lam alpha = y with K_lam = K + lam I                      (Eq. 1)
* P^-1 K_lam alpha = P^-1 y, solved by CG (Hestenes-Stiefel)  (Sec. 2.1, Eq. 2)

Readings where the paper is silent: x0 = 0; the stopping test is the
relative 2-norm residual |y - K_lam x| / |y| <= rtol; the recurrence
residual is checked against the true residual when it passes, and CG is
restarted from x (at most 3 times) if the true residual has not converged;
the iteration cap defaults to min(n, 20000).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla


def solve_exact(K: np.ndarray, lam: float, y: np.ndarray) -> np.ndarray:
    """Closed-form solve of Eq. 1 by dense Cholesky of K + lam I."""
    n = K.shape[0]
    c = sla.cho_factor(K + lam * np.eye(n), lower=True)
    return sla.cho_solve(c, y)


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float  # true relative residual |y - K_lam x| / |y|
    converged: bool
    restarts: int
    history: list
    # CG coefficients of the first run (before any restart): gamma_j = rho_j / p_j^T A p_j and
    # beta_j = rho_{j+1} / rho_j, the entries of the Lanczos matrix of P^-1 A (oracle.spectrum)
    gammas: list = dataclasses.field(default_factory=list)
    betas: list = dataclasses.field(default_factory=list)


def pcg(apply_A, apply_Pinv, y: np.ndarray, rtol: float = 1e-8, max_iter: int | None = None,
        max_restarts: int = 3) -> PCGResult:
    """Preconditioned CG (Sec. 2.1, Eq. 2) on A x = y (A = K_lam SPD, P^-1 SPD), x0 = 0."""
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    if max_iter is None:
        max_iter = min(n, 20000)
    ynorm = float(np.linalg.norm(y))
    x = np.zeros(n)
    if ynorm == 0.0:
        return PCGResult(x, 0, 0.0, True, 0, [], [], [])
    it = 0
    restarts = 0
    hist = []
    gammas, betas = [], []
    r = y.copy()
    while True:
        z = apply_Pinv(r)
        p = z.copy()
        rho = float(r @ z)
        while it < max_iter:
            q = apply_A(p)
            pq = float(p @ q)
            if not pq > 0.0:
                raise FloatingPointError("PCG breakdown: p^T A p <= 0")
            gamma = rho / pq
            if restarts == 0:
                gammas.append(gamma)
            x += gamma * p
            r -= gamma * q
            it += 1
            rel = float(np.linalg.norm(r)) / ynorm
            hist.append(rel)
            if rel <= rtol:
                break
            z = apply_Pinv(r)
            rho_new = float(r @ z)
            if restarts == 0:
                betas.append(rho_new / rho)
            p = z + (rho_new / rho) * p
            rho = rho_new
        r = y - apply_A(x)
        true_rel = float(np.linalg.norm(r)) / ynorm
        if true_rel <= rtol or it >= max_iter or restarts >= max_restarts:
            return PCGResult(x, it, true_rel, true_rel <= rtol, restarts, hist, gammas, betas)
        restarts += 1
