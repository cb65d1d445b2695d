"""Oracle: descriptor, Jacobian and the Matern-5/2 force kernel K (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

The paper (Sec. 2.1) uses the sGDML kernel: geometries are encoded by a
descriptor, K is PSD of size n = 3 d n_train and is made of 3d x 3d blocks,
one per pair of training geometries.  The kernel function itself is only
cited there; the reading used here is the GDML form without permutational
symmetries:

* descriptor  x_p = 1 / |R_i - R_j| for atom pairs i > j, p = i(i-1)/2 + j,
  D = N(N-1)/2;
* scalar kernel  kappa(x, x') = phi(|x - x'|), Matern-5/2
  phi(r) = (1 + c r + c^2 r^2 / 3) exp(-c r),  c = sqrt(5) / sigma;
* force kernel block  K_ab = grad_{R_a} grad_{R_b}^T kappa(x(R_a), x(R_b))
  = J_a^T H_ab J_b with the descriptor Jacobian J_a = dx_a / dR_a (D x 3N) and
  H_ab = d^2 kappa / dx_a dx_b^T = (c^2/3) e^{-c r} [(1 + c r) I - c^2 d d^T],
  d = x_a - x_b, r = |d|.

Vector index of a length-n vector: a*3N + 3*i + q (App. A, "Atomic
contribution": n -> (n_train, d, 3)).
"""
from __future__ import annotations

import numpy as np


def pair_index(N: int) -> tuple[np.ndarray, np.ndarray]:
    """Atom indices (i, j), i > j, of descriptor entry p = i(i-1)/2 + j (Sec. 2.1 descriptor)."""
    I, J = [], []
    for i in range(N):
        for j in range(i):
            I.append(i)
            J.append(j)
    return np.asarray(I, dtype=np.int64), np.asarray(J, dtype=np.int64)


def descriptor(R: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Inverse-distance descriptor X (M, D) and g (M, D, 3) = (R_i - R_j)/r^3 (Sec. 2.1).

    dx_p/dR_i = -g_p and dx_p/dR_j = +g_p for p = (i, j).
    """
    R = np.asarray(R, dtype=np.float64)
    I, J = pair_index(R.shape[1])
    diff = R[:, I, :] - R[:, J, :]
    r = np.sqrt(np.sum(diff * diff, axis=-1))
    return 1.0 / r, diff / (r**3)[..., None]


def jacobian(R: np.ndarray) -> np.ndarray:
    """Dense descriptor Jacobian J (M, D, 3N): J[a, p, 3i+q] = dx_{a,p}/dR_{a,i,q}; the J_a of
    K_ab = J_a^T H_ab J_b (Sec. 2.1)."""
    M, N, _ = R.shape
    I, J = pair_index(N)
    _, g = descriptor(R)
    D = I.size
    Jac = np.zeros((M, D, 3 * N))
    p = np.arange(D)
    for q in range(3):
        Jac[:, p, 3 * I + q] = -g[:, :, q]
        Jac[:, p, 3 * J + q] = g[:, :, q]
    return Jac


def matern52(r, sigma: float):
    """Scalar Matern-5/2 kernel phi(r), unit signal variance (the sGDML kernel cited in Sec. 2.1)."""
    c = np.sqrt(5.0) / sigma
    r = np.asarray(r, dtype=np.float64)
    return (1.0 + c * r + (c * r) ** 2 / 3.0) * np.exp(-c * r)


def hessian_block(xa: np.ndarray, xb: np.ndarray, sigma: float) -> np.ndarray:
    """H_ab = d^2 kappa(x_a, x_b) / dx_a dx_b^T (D x D), the middle factor of K_ab (Sec. 2.1)."""
    c = np.sqrt(5.0) / sigma
    d = xa - xb
    r = np.sqrt(d @ d)
    S = (c * c / 3.0) * np.exp(-c * r)
    return S * ((1.0 + c * r) * np.eye(d.size) - c * c * np.outer(d, d))


def force_kernel_dense(R: np.ndarray, sigma: float) -> np.ndarray:
    """Assemble the n x n force kernel K block by block (Sec. 2.1): K_ab = J_a^T H_ab J_b."""
    M, N, _ = R.shape
    X, _ = descriptor(R)
    Jac = jacobian(R)
    B = 3 * N
    K = np.empty((M * B, M * B))
    for a in range(M):
        for b in range(M):
            H = hessian_block(X[a], X[b], sigma)
            K[a * B:(a + 1) * B, b * B:(b + 1) * B] = Jac[a].T @ H @ Jac[b]
    return K


def force_kernel_column(R: np.ndarray, sigma: float, col: int) -> np.ndarray:
    """One column K[:, col] from its definition (used as get_col in Alg. 1)."""
    M, N, _ = R.shape
    B = 3 * N
    b, local = divmod(int(col), B)
    X, _ = descriptor(R)
    Jac = jacobian(R)
    out = np.empty(M * B)
    w = Jac[b][:, local]  # J_b e_local
    for a in range(M):
        out[a * B:(a + 1) * B] = Jac[a].T @ (hessian_block(X[a], X[b], sigma) @ w)
    return out


def column_getter(R: np.ndarray, sigma: float):
    """get_col(i) -> K[:, i] as in force_kernel_column, with the descriptor and
    Jacobian computed once (for Algorithm 1 on larger inputs)."""
    M, N, _ = R.shape
    B = 3 * N
    X, _ = descriptor(R)
    Jac = jacobian(R)

    def get_col(col):
        b, local = divmod(int(col), B)
        w = Jac[b][:, local]
        out = np.empty(M * B)
        for a in range(M):
            out[a * B:(a + 1) * B] = Jac[a].T @ (hessian_block(X[a], X[b], sigma) @ w)
        return out

    return get_col


def force_kernel_diag(R: np.ndarray, sigma: float) -> np.ndarray:
    """diag(K) (Sec. 2.1; the starting residual diagonal of Algorithm 1): K_aa = (c^2/3) J_a^T J_a
    since r = 0 on the diagonal block."""
    c = np.sqrt(5.0) / sigma
    Jac = jacobian(R)
    return ((c * c / 3.0) * np.sum(Jac * Jac, axis=1)).reshape(-1)


def matvec(R: np.ndarray, sigma: float, v: np.ndarray, lam: float = 0.0) -> np.ndarray:
    """Matrix-free (K + lam I) v (Sec. 2.1: CG needs only matrix-vector products).

    Steps: w_b = J_b v_b; u_a = sum_b H_ab w_b with H_ab applied from its
    definition, H_ab w = S_ab [(1 + c r_ab) w - c^2 d_ab (d_ab . w)];
    (K v)_a = J_a^T u_a.
    """
    M, N, _ = R.shape
    B = 3 * N
    c = np.sqrt(5.0) / sigma
    X, _ = descriptor(R)
    Jac = jacobian(R)
    V = np.asarray(v, dtype=np.float64).reshape(M, B)
    W = np.einsum("apk,ak->ap", Jac, V)
    U = np.empty_like(W)
    for a in range(M):
        d = X[a][None, :] - X  # (M, D): d_ab = x_a - x_b
        r = np.sqrt(np.sum(d * d, axis=1))
        S = (c * c / 3.0) * np.exp(-c * r)
        proj = np.sum(d * W, axis=1)  # d_ab . w_b
        U[a] = (S * (1.0 + c * r)) @ W - c * c * ((S * proj) @ d)
    out = np.einsum("apk,ap->ak", Jac, U).reshape(-1)
    return out + lam * np.asarray(v, dtype=np.float64)


def project(R: np.ndarray, v: np.ndarray) -> np.ndarray:
    """w_a = J_a v_a for every geometry (Sec. 2.1), from the two nonzeros of each row of J_a:
    w_{a,p} = -g_{a,p} . (v_{a,i} - v_{a,j}) for p = (i, j) (the entries jacobian() places).
    Returns W (M, D)."""
    M, N, _ = R.shape
    I, J = pair_index(N)
    _, g = descriptor(R)
    V = np.asarray(v, dtype=np.float64).reshape(M, N, 3)
    return -np.einsum("apq,apq->ap", g, V[:, I, :] - V[:, J, :])


def matvec_rows(R: np.ndarray, sigma: float, v: np.ndarray, rows, lam: float = 0.0) -> np.ndarray:
    """Blocks a in `rows` of (K + lam I) v (Sec. 2.1), from the same definition as matvec
    (all w_b = J_b v_b are needed, but only the H_ab of the sampled a):
    u_a = sum_b S_ab [(1 + c r_ab) w_b - c^2 d_ab (d_ab . w_b)], (K v)_a = J_a^T u_a.
    Returns an array of shape (len(rows), 3N)."""
    M, N, _ = R.shape
    B = 3 * N
    c = np.sqrt(5.0) / sigma
    X, _ = descriptor(R)
    W = project(R, v)
    V = np.asarray(v, dtype=np.float64).reshape(M, B)
    out = np.empty((len(rows), B))
    for t, a in enumerate(rows):
        d = X[a][None, :] - X  # (M, D): d_ab = x_a - x_b
        r = np.sqrt(np.einsum("bp,bp->b", d, d))
        S = (c * c / 3.0) * np.exp(-c * r)
        proj = np.einsum("bp,bp->b", d, W)  # d_ab . w_b
        u = (S * (1.0 + c * r)) @ W - c * c * ((S * proj) @ d)
        out[t] = jacobian(R[a:a + 1])[0].T @ u + lam * V[a]
    return out


def matvec_parallel(R: np.ndarray, sigma: float, v: np.ndarray, lam: float = 0.0,
                    workers: int | None = None) -> np.ndarray:
    """(K + lam I) v, the geometry blocks of matvec_rows shared out over worker processes
    (spawn start method: safe after a CUDA context exists in the caller; one BLAS thread per
    worker).  For the large systems where the single-process matvec takes minutes."""
    import multiprocessing as mp
    import os
    M = R.shape[0]
    workers = max(1, min(workers or os.cpu_count() or 1, M))
    chunks = [list(ch) for ch in np.array_split(np.arange(M), 2 * workers) if len(ch)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    try:
        for k in saved:
            os.environ[k] = "1"
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.starmap(matvec_rows, [(R, sigma, v, ch, lam) for ch in chunks])
    finally:
        for k, val in saved.items():
            if val is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = val
    return np.concatenate(parts).reshape(-1)


# ---- sGDML: permutational symmetries (Sec. 4.3, "Remarks on runtime": the kernel's forward
# pass grows with the number of symmetries) ------------------------------------------------
# A symmetry group of the molecule is given as S atom permutations sigma_q (sigma_q[i] = the
# atom that takes atom i's place).  Permuting the atoms of R_b permutes its descriptor entries:
# x(R_b^(q))_p = x(R_b)_{pi_q(p)} with pi_q(p) the pair index of (sigma_q(i), sigma_q(j)).  The
# symmetric scalar kernel is kappa_S(R_a, R_b) = sum_q kappa(x_a, P_q x_b) (no normalisation;
# the reading is stated in the design doc's R18), so its force kernel is
#   K_ab = sum_q J_a^T H(x_a, P_q x_b) P_q J_b,
# where P_q x_b and P_q J_b take rows pi_q(p) of x_b and J_b.

def pair_permutation(N: int, perm) -> np.ndarray:
    """pi(p) = pair index of (perm[i], perm[j]) for descriptor entry p = (i, j): x(R with atoms
    permuted by perm)_p = x(R)_pi(p)."""
    perm = np.asarray(perm, dtype=np.int64)
    I, J = pair_index(N)
    a, b = perm[I], perm[J]
    hi, lo = np.maximum(a, b), np.minimum(a, b)
    return hi * (hi - 1) // 2 + lo


def sym_kernel_value(Ra: np.ndarray, Rb: np.ndarray, sigma: float, perms) -> float:
    """kappa_S(R_a, R_b) = sum_q kappa(x(R_a), x(R_b with its atoms permuted by perm q)): the
    scalar symmetric kernel from atomic coordinates (used to pin its force kernel)."""
    xa = descriptor(Ra[None])[0][0]
    tot = 0.0
    for perm in perms:
        xb = descriptor(np.asarray(Rb)[np.asarray(perm)][None])[0][0]
        tot += float(matern52(np.linalg.norm(xa - xb), sigma))
    return tot


def force_kernel_dense_sym(R: np.ndarray, sigma: float, perms) -> np.ndarray:
    """Assemble the n x n symmetric force kernel block by block:
    K_ab = sum_q J_a^T H(x_a, P_q x_b) P_q J_b."""
    M, N, _ = R.shape
    X, _ = descriptor(R)
    Jac = jacobian(R)
    B = 3 * N
    pis = [pair_permutation(N, p) for p in perms]
    K = np.zeros((M * B, M * B))
    for a in range(M):
        for b in range(M):
            for pi in pis:
                H = hessian_block(X[a], X[b][pi], sigma)
                K[a * B:(a + 1) * B, b * B:(b + 1) * B] += Jac[a].T @ H @ Jac[b][pi]
    return K


def matvec_sym(R: np.ndarray, sigma: float, perms, v: np.ndarray, lam: float = 0.0) -> np.ndarray:
    """Matrix-free (K + lam I) v with the symmetric force kernel: w_b = J_b v_b;
    u_a = sum_q sum_b H(x_a, P_q x_b) P_q w_b, each H applied from its definition;
    (K v)_a = J_a^T u_a."""
    M, N, _ = R.shape
    B = 3 * N
    c = np.sqrt(5.0) / sigma
    X, _ = descriptor(R)
    W = project(R, v)
    V = np.asarray(v, dtype=np.float64).reshape(M, B)
    U = np.zeros_like(W)
    for pi in (pair_permutation(N, p) for p in perms):
        Xq, Wq = X[:, pi], W[:, pi]
        for a in range(M):
            d = X[a][None, :] - Xq  # d_ab = x_a - P_q x_b
            r = np.sqrt(np.einsum("bp,bp->b", d, d))
            S = (c * c / 3.0) * np.exp(-c * r)
            proj = np.einsum("bp,bp->b", d, Wq)
            U[a] += (S * (1.0 + c * r)) @ Wq - c * c * ((S * proj) @ d)
    out = np.empty((M, B))
    for a in range(M):
        out[a] = jacobian(R[a:a + 1])[0].T @ U[a] + lam * V[a]
    return out.reshape(-1)


def force_kernel_diag_sym(R: np.ndarray, sigma: float, perms) -> np.ndarray:
    """diag(K) of the symmetric force kernel: diag of sum_q J_a^T H(x_a, P_q x_a) P_q J_a."""
    M, N, _ = R.shape
    X, _ = descriptor(R)
    Jac = jacobian(R)
    B = 3 * N
    out = np.zeros((M, B))
    for pi in (pair_permutation(N, p) for p in perms):
        for a in range(M):
            out[a] += np.diag(Jac[a].T @ hessian_block(X[a], X[a][pi], sigma) @ Jac[a][pi])
    return out.reshape(-1)


def predict_forces(R_query: np.ndarray, R: np.ndarray, sigma: float, alpha: np.ndarray) -> np.ndarray:
    """Forces the trained model predicts for query geometries (Sec. 2.1: queried at a cost
    linear in the training set): f_q = sum_b K(q, b) alpha_b with the force-kernel block
    K(q, b) = J_q^T H(x_q, x_b) J_b of the query q against training geometry b.

    R_query: (Q, N, 3); R: (M, N, 3) training geometries; alpha: length 3 N M, the
    solution of Eq. 1.  Returns (Q, N, 3).
    """
    R_query = np.asarray(R_query, dtype=np.float64)
    M, N, _ = R.shape
    Q = R_query.shape[0]
    B = 3 * N
    Xq, _ = descriptor(R_query)
    Jq = jacobian(R_query)
    X, _ = descriptor(R)
    Jb = jacobian(R)
    A = np.asarray(alpha, dtype=np.float64).reshape(M, B)
    out = np.zeros((Q, B))
    for q in range(Q):
        for b in range(M):
            out[q] += Jq[q].T @ (hessian_block(Xq[q], X[b], sigma) @ (Jb[b] @ A[b]))
    return out.reshape(Q, N, 3)
