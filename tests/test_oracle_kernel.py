"""Pins for the oracle's descriptor and force kernel (Sec. 2.1), independent of its own formulas."""
import numpy as np
import pytest

from oracle import kernel as ok


def kappa_of_geometries(Ra, Rb, sigma):
    """kappa(x(R_a), x(R_b)) straight from the Matern-5/2 definition."""
    xa, _ = ok.descriptor(Ra[None])
    xb, _ = ok.descriptor(Rb[None])
    r = np.linalg.norm(xa[0] - xb[0])
    c = np.sqrt(5.0) / sigma
    return (1 + c * r + c * c * r * r / 3) * np.exp(-c * r)


def test_descriptor_jacobian_matches_finite_differences(tiny):
    R, _ = tiny
    Jac = ok.jacobian(R)
    h = 1e-6
    for a in range(R.shape[0]):
        for col in range(R.shape[1] * 3):
            i, q = divmod(col, 3)
            Rp = R[a].copy(); Rp[i, q] += h
            Rm = R[a].copy(); Rm[i, q] -= h
            fd = (ok.descriptor(Rp[None])[0][0] - ok.descriptor(Rm[None])[0][0]) / (2 * h)
            np.testing.assert_allclose(Jac[a][:, col], fd, rtol=1e-6, atol=1e-9)


def test_matern52_against_sklearn():
    sk = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(0)
    A = rng.standard_normal((7, 4))
    B = rng.standard_normal((5, 4))
    for sigma in (0.5, 3.0):
        ref = sk.Matern(length_scale=sigma, nu=2.5)(A, B)
        r = np.linalg.norm(A[:, None] - B[None], axis=-1)
        np.testing.assert_allclose(ok.matern52(r, sigma), ref, rtol=1e-13)
    assert ok.matern52(0.0, 1.0) == 1.0


def test_force_kernel_matches_mixed_second_differences(tiny):
    """K_ab[(i,q),(j,s)] = d^2 kappa / dR_a,iq dR_b,js by central differences."""
    R, _ = tiny
    sigma = 1.0  # small length scale: every term of the Hessian matters
    K = ok.force_kernel_dense(R, sigma)
    M, N, _ = R.shape
    B = 3 * N
    h = 1e-4
    rng = np.random.default_rng(1)
    for a, b in [(0, 0), (0, 1), (2, 1)]:
        for _ in range(12):
            u, v = rng.integers(0, B, size=2)
            eu = np.zeros(B); eu[u] = h
            ev = np.zeros(B); ev[v] = h
            Ra, Rb = R[a].reshape(-1), R[b].reshape(-1)

            def f(du, dv):
                return kappa_of_geometries((Ra + du).reshape(N, 3), (Rb + dv).reshape(N, 3), sigma)

            fd = (f(eu, ev) - f(eu, -ev) - f(-eu, ev) + f(-eu, -ev)) / (4 * h * h)
            assert abs(K[a * B + u, b * B + v] - fd) <= 1e-6 * np.abs(K).max(), (a, b, u, v)


def test_force_kernel_symmetric_psd_and_rigid_null_space(tiny):
    R, _ = tiny
    M, N, _ = R.shape
    K = ok.force_kernel_dense(R, 2.0)
    assert np.array_equal(K, K.T) or np.abs(K - K.T).max() <= 1e-15 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert ev.min() >= -1e-13 * ev.max()
    # K annihilates translations and infinitesimal rotations of each geometry
    B = 3 * N
    for a in range(M):
        for q in range(3):
            t = np.zeros(M * B); t[a * B + q:(a + 1) * B:3] = 1.0
            assert np.linalg.norm(K @ t) <= 1e-12 * ev.max() * np.linalg.norm(t)
            w = np.zeros(3); w[q] = 1.0
            rot = np.zeros(M * B); rot[a * B:(a + 1) * B] = np.cross(w, R[a]).reshape(-1)
            assert np.linalg.norm(K @ rot) <= 1e-12 * ev.max() * np.linalg.norm(rot)
    # and nothing else: null space dimension 6M (App. A.1: l ~ 6 n_train)
    assert np.sum(ev < 1e-10 * ev.max()) == 6 * M


def test_single_geometry_closed_form(tiny):
    R, _ = tiny
    sigma = 1.7
    J = ok.jacobian(R[:1])[0]
    np.testing.assert_allclose(ok.force_kernel_dense(R[:1], sigma), (5 / (3 * sigma**2)) * J.T @ J, rtol=1e-13)


def test_matrix_free_matvec_column_and_diag_match_dense(tiny):
    R, _ = tiny
    sigma, lam = 1.3, 1e-3
    K = ok.force_kernel_dense(R, sigma)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(K.shape[0])
    ref = K @ v + lam * v
    np.testing.assert_allclose(ok.matvec(R, sigma, v, lam), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    for col in (0, 7, K.shape[0] - 1):
        np.testing.assert_allclose(ok.force_kernel_column(R, sigma, col), K[:, col], atol=1e-14 * np.abs(K).max())
    np.testing.assert_allclose(ok.force_kernel_diag(R, sigma), np.diag(K), rtol=1e-13)


def test_descriptor_order_does_not_change_k(tiny, monkeypatch):
    R, _ = tiny
    K = ok.force_kernel_dense(R, 1.5)
    I, J = ok.pair_index(R.shape[1])
    perm = np.random.default_rng(3).permutation(I.size)
    monkeypatch.setattr(ok, "pair_index", lambda N: (I[perm], J[perm]))
    np.testing.assert_allclose(ok.force_kernel_dense(R, 1.5), K, atol=1e-15 * np.abs(K).max())


def test_atom_relabelling_permutes_k(tiny):
    """Relabelling atoms the same way in every geometry permutes rows/columns of K."""
    R, _ = tiny
    M, N, _ = R.shape
    K = ok.force_kernel_dense(R, 1.5)
    pa = np.array([3, 0, 4, 1, 2])
    Kp = ok.force_kernel_dense(R[:, pa, :], 1.5)
    idx = np.array([a * 3 * N + 3 * pa[i] + q for a in range(M) for i in range(N) for q in range(3)])
    np.testing.assert_allclose(Kp, K[np.ix_(idx, idx)], atol=1e-14 * np.abs(K).max())


def test_planted_sign_error_is_caught(tiny, monkeypatch):
    """A flipped sign of the d d^T term must break the finite-difference pin."""
    R, _ = tiny
    good = ok.hessian_block

    def bad(xa, xb, sigma):
        c = np.sqrt(5.0) / sigma
        d = xa - xb
        return good(xa, xb, sigma) + 2 * (c * c / 3) * np.exp(-c * np.linalg.norm(d)) * c * c * np.outer(d, d)

    monkeypatch.setattr(ok, "hessian_block", bad)
    with pytest.raises(AssertionError):
        test_force_kernel_matches_mixed_second_differences((R, None))


def test_sampled_rows_equal_full_matvec(tiny):
    R, _ = tiny
    v = np.random.default_rng(4).standard_normal(R.size)
    full = ok.matvec(R, 1.3, v, 1e-4).reshape(R.shape[0], -1)
    np.testing.assert_allclose(ok.matvec_rows(R, 1.3, v, [2, 0], 1e-4), full[[2, 0]], rtol=0,
                               atol=1e-14 * np.abs(full).max())


def test_projection_equals_dense_jacobian_product(tiny):
    """project(): J_a v_a from the two nonzeros per Jacobian row equals the dense J_a v_a."""
    R, _ = tiny
    v = np.random.default_rng(4).standard_normal(R.size)
    Jac = ok.jacobian(R)
    dense = np.einsum("apk,ak->ap", Jac, v.reshape(R.shape[0], -1))
    np.testing.assert_allclose(ok.project(R, v), dense, rtol=0, atol=1e-14 * np.abs(dense).max())


def test_parallel_matvec_equals_dense_k(tiny):
    """matvec_parallel (row blocks in spawned worker processes) equals (K + lam I) v with K
    assembled densely, and the serial matvec."""
    from paper_2212_12737_gb300 import synth
    R = synth.geometries(synth.template(6, 3), 9, 0.2, 4)
    v = np.random.default_rng(5).standard_normal(R.size)
    K = ok.force_kernel_dense(R, 1.7)
    ref = K @ v + 1e-3 * v
    got = ok.matvec_parallel(R, 1.7, v, 1e-3, workers=2)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(got, ok.matvec(R, 1.7, v, 1e-3), rtol=0, atol=1e-13 * np.abs(ref).max())
