"""Pins for the oracle's exact solve (Eq. 1) and PCG (Sec. 2.1, Eq. 2), plus the input generator."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import kernel as ok
from oracle import precond as op
from oracle import solver as osv
from paper_2212_12737_gb300 import synth


@pytest.fixture(scope="module")
def system():
    tmpl = synth.template(6, 21)
    R = synth.geometries(tmpl, 6, 0.2, 22)
    y = synth.morse_forces(R, tmpl).reshape(-1)
    K = ok.force_kernel_dense(R, 2.0)
    return R, y, K


def test_exact_solve_matches_numpy_solve(system):
    R, y, K = system
    lam = 1e-4
    a = osv.solve_exact(K, lam, y)
    ref = np.linalg.solve(K + lam * np.eye(K.shape[0]), y)
    np.testing.assert_allclose(a, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert np.linalg.norm(y - K @ a - lam * a) <= 1e-12 * np.linalg.norm(y)


def test_pcg_iterates_match_scipy_cg(system):
    """x_j after j PCG steps equals SciPy's preconditioned CG after j steps."""
    R, y, K = system
    lam = 1e-3
    n = K.shape[0]
    L, piv, _ = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), 8)
    LC = op.woodbury_core(L, lam)
    A = lambda v: K @ v + lam * v
    Pinv = lambda r: op.woodbury_apply(L, LC, lam, r)
    for j in (1, 4, 10):
        ours = osv.pcg(A, Pinv, y, rtol=1e-30, max_iter=j, max_restarts=0)
        ref, _ = spla.cg(spla.LinearOperator((n, n), matvec=A), y, rtol=1e-30, atol=0.0, maxiter=j,
                         M=spla.LinearOperator((n, n), matvec=Pinv))
        assert ours.iters == j
        np.testing.assert_allclose(ours.x, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_pcg_with_p_equal_k_lambda_converges_in_one_step(system):
    """App. A.1: when all eigenvalues are equal, CG converges after one step."""
    R, y, K = system
    lam = 1e-4
    Kl = K + lam * np.eye(K.shape[0])
    res = osv.pcg(lambda v: Kl @ v, lambda r: np.linalg.solve(Kl, r), y, rtol=1e-10)
    assert res.iters == 1 and res.converged


def test_pcg_converges_to_exact_solution_with_monotone_energy_error(system):
    R, y, K = system
    lam = 1e-6
    n = K.shape[0]
    Kl = K + lam * np.eye(n)
    exact = osv.solve_exact(K, lam, y)
    S = op.select_uniform(n, 20, 2)
    L, _ = op.nystrom_factor(K[:, S], S)
    LC = op.woodbury_core(L, lam)
    errs = []
    for j in range(1, 40):
        res = osv.pcg(lambda v: Kl @ v, lambda r: op.woodbury_apply(L, LC, lam, r), y, rtol=1e-30,
                      max_iter=j, max_restarts=0)
        e = res.x - exact
        errs.append(float(e @ Kl @ e))
    assert np.all(np.diff(errs) <= 1e-9 * errs[0])
    res = osv.pcg(lambda v: Kl @ v, lambda r: op.woodbury_apply(L, LC, lam, r), y, rtol=1e-9)
    assert res.converged and res.relres <= 1e-9
    assert np.linalg.norm(Kl @ (res.x - exact)) <= 1e-8 * np.linalg.norm(y)


def test_full_rank_nystrom_preconditioner_converges_in_few_steps(system):
    """A preconditioner that captures the whole range of K leaves only lam-level work."""
    R, y, K = system
    lam = 1e-6
    n = K.shape[0]
    Kl = K + lam * np.eye(n)
    L, piv, tr = op.pivoted_cholesky(lambda i: K[:, i], np.diag(K), n)
    d_ok = np.sum(np.linalg.eigvalsh(K) > 1e-10 * np.trace(K))
    L = L[:, :d_ok]
    LC = op.woodbury_core(L, lam)
    res = osv.pcg(lambda v: Kl @ v, lambda r: op.woodbury_apply(L, LC, lam, r), y, rtol=1e-8)
    assert res.converged and res.iters <= 3


def test_pcg_reports_non_convergence(system):
    R, y, K = system
    res = osv.pcg(lambda v: K @ v + 1e-10 * v, lambda r: r, y, rtol=1e-12, max_iter=3, max_restarts=0)
    assert not res.converged and res.iters == 3


def test_pcg_restarts_when_the_recurrence_residual_drifts():
    """The restart branch: one corrupted product makes the recurrence residual r disagree
    with y - A x; when r passes rtol the true residual does not, and PCG must restart from x
    (then converge to the exact solution); with no restarts allowed it must report failure."""
    rng = np.random.default_rng(5)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * np.linspace(1.0, 50.0, n)) @ Q.T
    y = rng.standard_normal(n)
    x_star = np.linalg.solve(A, y)

    def make_apply():
        calls = {"n": 0}

        def apply_A(v):
            calls["n"] += 1
            out = A @ v
            if calls["n"] == 3:  # one wrong product inside the first CG run
                out = out + 1e-3 * np.linalg.norm(out) * rng.standard_normal(n)
            return out
        return apply_A

    res = osv.pcg(make_apply(), lambda r: r, y, rtol=1e-10, max_iter=500, max_restarts=3)
    assert res.restarts >= 1 and res.converged and res.relres <= 1e-10
    np.testing.assert_allclose(res.x, x_star, rtol=0, atol=1e-8 * np.abs(x_star).max())
    res0 = osv.pcg(make_apply(), lambda r: r, y, rtol=1e-10, max_iter=500, max_restarts=0)
    assert res0.restarts == 0 and not res0.converged and res0.relres > 1e-10


# ---- generator (inputs, not method) ---------------------------------------

def test_morse_forces_are_minus_energy_gradient_and_rigid_free():
    tmpl = synth.template(7, 3)
    R = synth.geometries(tmpl, 2, 0.1, 4)
    F = synth.morse_forces(R, tmpl)
    h = 1e-6
    for a in range(2):
        for i in range(7):
            for q in range(3):
                Rp = R.copy(); Rp[a, i, q] += h
                Rm = R.copy(); Rm[a, i, q] -= h
                fd = -(synth.morse_energy(Rp, tmpl)[a] - synth.morse_energy(Rm, tmpl)[a]) / (2 * h)
                assert abs(F[a, i, q] - fd) <= 1e-6 * max(1.0, abs(fd))
    np.testing.assert_allclose(F.sum(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(R, F).sum(axis=1), 0.0, atol=1e-12)


def test_template_min_distance_and_labels_orthogonal_to_null_space():
    for N in (9, 21, 42):
        t = synth.template(N, 0)
        d = np.linalg.norm(t[:, None] - t[None], axis=-1)[np.triu_indices(N, 1)]
        assert d.min() >= 1.0 and np.all(np.linalg.norm(t, axis=1) <= N ** (1 / 3) + 1e-12)
    tmpl = synth.template(5, 1)
    R = synth.geometries(tmpl, 3, 0.1, 2)
    y = synth.morse_forces(R, tmpl).reshape(-1)
    K = ok.force_kernel_dense(R, 3.0)
    ev, U = np.linalg.eigh(K)
    null = U[:, ev < 1e-10 * ev.max()]
    assert null.shape[1] == 18
    assert np.linalg.norm(null.T @ y) <= 1e-10 * np.linalg.norm(y)
