"""Pins for the oracle's symmetric (sGDML) force kernel: K_ab = sum_q J_a^T H(x_a, P_q x_b) P_q J_b
for a permutation group of the atoms, independent of its own formulas (finite differences of
the scalar kernel computed from permuted coordinates, the plain kernel, group structure)."""
import numpy as np
import pytest

from oracle import kernel as ok

ID5 = [0, 1, 2, 3, 4]
SWAP01 = [ID5, [1, 0, 2, 3, 4]]
CYCLE012 = [ID5, [1, 2, 0, 3, 4], [2, 0, 1, 3, 4]]
KLEIN = [ID5, [1, 0, 2, 3, 4], [0, 1, 2, 4, 3], [1, 0, 2, 4, 3]]


def test_pair_permutation_moves_descriptor_entries(tiny):
    """x(R with atoms permuted)_p = x(R)_pi(p), from the descriptor of the permuted coordinates."""
    R, _ = tiny
    for perm in (SWAP01[1], CYCLE012[1], KLEIN[3]):
        pi = ok.pair_permutation(5, perm)
        assert sorted(pi.tolist()) == list(range(10))
        X, _ = ok.descriptor(R)
        Xp, _ = ok.descriptor(R[:, perm, :])
        np.testing.assert_array_equal(Xp, X[:, pi])


def test_identity_group_is_the_plain_kernel(tiny):
    R, _ = tiny
    np.testing.assert_array_equal(ok.force_kernel_dense_sym(R, 1.2, [ID5]), ok.force_kernel_dense(R, 1.2))


@pytest.mark.parametrize("group", [SWAP01, CYCLE012, KLEIN])
def test_symmetric_kernel_is_the_mixed_hessian_of_the_symmetrised_scalar_kernel(tiny, group):
    """K_ab[(i,q),(j,s)] = d^2 kappa_S / dR_a,iq dR_b,js by central differences, with kappa_S
    evaluated from permuted atomic coordinates (not from the oracle's P_q, J or H)."""
    R, _ = tiny
    sigma = 1.0
    K = ok.force_kernel_dense_sym(R, sigma, group)
    M, N, _ = R.shape
    B = 3 * N
    h = 1e-4
    rng = np.random.default_rng(2)
    for a, b in [(0, 0), (0, 1), (2, 1)]:
        for _ in range(10):
            u, v = rng.integers(0, B, size=2)
            eu = np.zeros(B); eu[u] = h
            ev = np.zeros(B); ev[v] = h
            Ra, Rb = R[a].reshape(-1), R[b].reshape(-1)

            def f(du, dv):
                return ok.sym_kernel_value((Ra + du).reshape(N, 3), (Rb + dv).reshape(N, 3), sigma, group)

            fd = (f(eu, ev) - f(eu, -ev) - f(-eu, ev) + f(-eu, -ev)) / (4 * h * h)
            assert abs(K[a * B + u, b * B + v] - fd) <= 1e-6 * np.abs(K).max(), (a, b, u, v)


@pytest.mark.parametrize("group", [SWAP01, CYCLE012, KLEIN])
def test_symmetric_kernel_is_symmetric_psd_and_invariant_for_a_group(tiny, group):
    R, _ = tiny
    K = ok.force_kernel_dense_sym(R, 1.2, group)
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() >= -1e-12 * np.abs(K).max()
    # kappa_S(R_a, R_b) does not change when R_b's atoms are permuted by a group element
    for perm in group:
        assert abs(ok.sym_kernel_value(R[0], R[1][perm], 1.2, group) - ok.sym_kernel_value(R[0], R[1], 1.2, group)) \
            <= 1e-14 * len(group)


def test_a_set_that_is_not_a_group_breaks_symmetry(tiny):
    """Without closure under composition K_ab != K_ba^T: the library accepts groups only."""
    R, _ = tiny
    K = ok.force_kernel_dense_sym(R, 1.2, [ID5, [1, 2, 0, 3, 4]])
    assert np.abs(K - K.T).max() > 1e-6 * np.abs(K).max()


@pytest.mark.parametrize("group", [SWAP01, KLEIN])
def test_symmetric_matvec_and_diagonal_equal_the_dense_kernel(tiny, group):
    R, _ = tiny
    K = ok.force_kernel_dense_sym(R, 1.3, group)
    v = np.random.default_rng(4).standard_normal(R.size)
    ref = K @ v + 1e-4 * v
    np.testing.assert_allclose(ok.matvec_sym(R, 1.3, group, v, 1e-4), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(ok.force_kernel_diag_sym(R, 1.3, group), np.diag(K), rtol=0,
                               atol=1e-14 * np.abs(K).max())
