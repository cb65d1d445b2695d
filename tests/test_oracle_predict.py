"""Pins of the oracle's force prediction f_q = sum_b J_q^T H(x_q, x_b) J_b alpha_b
(Sec. 2.1) against what the model and the mathematics fix, without its Hessian blocks:

* at the training geometries the prediction is K alpha = y - lambda alpha (Eq. 1);
* it is the gradient, in the query coordinates, of the model's energy
  E(R*) = sum_b grad_{x_b} kappa(x*, x_b) . (J_b alpha_b), taken here by a complex-step
  derivative of the scalar Matern-5/2 function and central differences;
* rotating the query rotates the forces, translating it changes nothing, and the
  predicted net force vanishes.
"""
import numpy as np
import pytest

from oracle import kernel as ok
from oracle import solver as osv
from paper_2212_12737_gb300 import synth

SIGMA = 2.0


@pytest.fixture(scope="module")
def model():
    tmpl = synth.template(5, 3)
    R = synth.geometries(tmpl, 6, 0.2, 4)
    Rq = synth.geometries(tmpl, 3, 0.25, 11)
    alpha = np.random.default_rng(1).standard_normal(R.size)
    return R, Rq, alpha


def phi(r, sigma):
    """Matern-5/2 as a function of (possibly complex) r, for the complex-step derivative."""
    c = np.sqrt(5.0) / sigma
    return (1.0 + c * r + (c * r) ** 2 / 3.0) * np.exp(-c * r)


def energy(Rq1, R, alpha, sigma):
    """sum_b d/dt kappa(x(Rq1), x_b + t w_b) at t = 0, w_b = J_b alpha_b (complex step, h = 1e-30)."""
    xq = ok.descriptor(Rq1[None])[0][0]
    X, _ = ok.descriptor(R)
    Jb = ok.jacobian(R)
    M, N, _ = R.shape
    W = np.einsum("apk,ak->ap", Jb, alpha.reshape(M, 3 * N))
    h = 1e-30
    e = 0.0
    for b in range(M):
        d = xq - (X[b] + 1j * h * W[b])
        e += phi(np.sqrt(np.sum(d * d)), sigma).imag / h
    return e


def test_phi_is_the_oracle_matern(model):
    r = np.linspace(0.0, 5.0, 11)
    np.testing.assert_allclose(phi(r, SIGMA), ok.matern52(r, SIGMA), rtol=1e-15, atol=0)


def test_prediction_at_training_geometries_is_y_minus_lambda_alpha(model):
    R, _, _ = model
    y = np.random.default_rng(2).standard_normal(R.size)
    lam = 1e-3
    K = ok.force_kernel_dense(R, SIGMA)
    alpha = osv.solve_exact(K, lam, y)
    f = ok.predict_forces(R, R, SIGMA, alpha).reshape(-1)
    np.testing.assert_allclose(f, y - lam * alpha, rtol=0, atol=1e-9 * np.abs(y).max())


def test_prediction_is_the_gradient_of_the_model_energy(model):
    R, Rq, alpha = model
    f = ok.predict_forces(Rq, R, SIGMA, alpha)
    h = 1e-5
    for q in range(Rq.shape[0]):
        g = np.empty(Rq.shape[1:])
        for i in range(Rq.shape[1]):
            for k in range(3):
                Rp, Rm = Rq[q].copy(), Rq[q].copy()
                Rp[i, k] += h
                Rm[i, k] -= h
                g[i, k] = (energy(Rp, R, alpha, SIGMA) - energy(Rm, R, alpha, SIGMA)) / (2 * h)
        np.testing.assert_allclose(f[q], g, rtol=0, atol=1e-7 * np.abs(g).max())


def test_rotation_equivariance_translation_invariance_and_zero_net_force(model):
    R, Rq, alpha = model
    f = ok.predict_forces(Rq, R, SIGMA, alpha)
    Qm, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((3, 3)))
    f_rot = ok.predict_forces(Rq @ Qm.T, R, SIGMA, alpha)
    np.testing.assert_allclose(f_rot, f @ Qm.T, rtol=0, atol=1e-12 * np.abs(f).max())
    f_tr = ok.predict_forces(Rq + np.array([0.3, -1.2, 2.0]), R, SIGMA, alpha)
    np.testing.assert_allclose(f_tr, f, rtol=0, atol=1e-12 * np.abs(f).max())
    assert np.abs(f.sum(axis=1)).max() <= 1e-12 * np.abs(f).max()


def test_planted_hessian_error_is_caught(model, monkeypatch):
    """Dropping the c^2 d d^T term of H leaves K symmetric and the net force zero, but the
    prediction is then no longer the energy's gradient."""
    R, Rq, alpha = model
    good = ok.predict_forces(Rq[:1], R, SIGMA, alpha)

    def bad(xa, xb, sigma):
        c = np.sqrt(5.0) / sigma
        r = np.sqrt(np.sum((xa - xb) ** 2))
        return (c * c / 3.0) * np.exp(-c * r) * (1.0 + c * r) * np.eye(xa.size)

    monkeypatch.setattr(ok, "hessian_block", bad)
    assert np.abs(ok.predict_forces(Rq[:1], R, SIGMA, alpha) - good).max() > 1e-3 * np.abs(good).max()
