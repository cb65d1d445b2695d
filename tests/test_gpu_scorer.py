"""Learned inducing-column scorer: BF16 MLP kernels (the five contractions on the tcgen05
tensor cores) against a PyTorch CPU FP32 reference with the same forward BF16 roundings
(straight-through gradients). The GPU's backward pass also rounds the back-propagated
gradients to BF16 (they are tensor-core operands): relative 2^-9 per entry, well inside the
gradient tolerance. Then the RLS labels against the oracle, and the learned selection with
pivoted Cholesky as fallback and referee."""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from oracle import precond as op
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2212_12737_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    gdml.load()


def bf(x):
    """round to BF16 in the forward pass, identity in the backward pass"""
    return x + (x.to(torch.bfloat16).to(torch.float32) - x).detach()


def reference_loss(p, X, y, D, H, mu, sd, ym, ysd):
    i = 0
    W1 = p[i:i + H * D].view(H, D); i += H * D
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].view(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    w3 = p[i:i + H]; i += H
    b3 = p[i:i + 1]
    Xs = bf(((X - mu) / sd).float())
    Z1 = Xs @ bf(W1).T + b1
    A1 = bf(torch.nn.functional.gelu(Z1))
    Z2 = A1 @ bf(W2).T + b2
    A2 = bf(torch.nn.functional.gelu(Z2))
    out = A2 @ bf(w3) + b3
    ys = ((y - ym) / ysd).float()
    return torch.mean((out - ys) ** 2)


def test_mlp_loss_and_gradient_match_cpu_reference():
    rng = np.random.default_rng(0)
    B, D, H = 96, 36, 64
    X = rng.standard_normal((B, D)) * 0.3 + 1.0
    y = X[:, :5].sum(1) + 0.1 * rng.standard_normal(B)
    s = gdml.Scorer(D, H, seed=3)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    s.fit_scaling(Xd, yd)
    loss, g = s.grad(Xd, yd)
    p = s.params().cpu().requires_grad_(True)
    mu = torch.from_numpy(X.mean(0)).float()
    sd = torch.from_numpy(X.std(0)).float()
    ref = reference_loss(p, torch.from_numpy(X), torch.from_numpy(y), D, H, mu, sd, float(y.mean()), float(y.std()))
    ref.backward()
    assert abs(loss - ref.item()) <= 2e-3 * ref.item()
    gg = g.cpu()
    assert float(torch.linalg.norm(gg - p.grad) / torch.linalg.norm(p.grad)) <= 2e-2
    # finite differences on the FP32 output bias (not rounded in the forward pass)
    h = 1e-3
    q = s.params()
    q[-1] += h
    s.set_params(q)
    lp, _ = s.grad(Xd, yd)
    q[-1] -= 2 * h
    s.set_params(q)
    lm, _ = s.grad(Xd, yd)
    assert abs((lp - lm) / (2 * h) - float(gg[-1])) <= 1e-2 * abs(float(gg[-1])) + 1e-4
    s.destroy()


def test_mlp_training_fits_a_smooth_target():
    rng = np.random.default_rng(1)
    B, D = 512, 36
    X = rng.standard_normal((B, D))
    y = np.tanh(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    s = gdml.Scorer(D, 256, seed=1)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    s.fit_scaling(Xd, yd)
    l0, _ = s.grad(Xd, yd)
    s.train(Xd, yd, epochs=60, batch=128, lr=1e-3)
    l1, _ = s.grad(Xd, yd)
    pred = s.predict(Xd).cpu().numpy()
    assert l1 < 0.1 * l0
    assert np.corrcoef(pred, y)[0, 1] > 0.95
    s.destroy()


def test_rls_scores_match_oracle_estimate():
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, 1e-4)
    tau = ctx.rls_scores(100, seed=2).cpu().numpy()
    K = ok.force_kernel_dense(w.R, w.sigma)
    S0 = op.select_uniform(w.n, 100, 2, 1)
    ref = op.rls_nystrom(K[:, S0], S0, 1e-4)
    assert np.all(tau >= -1e-12) and np.all(tau <= 1 + 1e-9)
    np.testing.assert_allclose(tau, ref, rtol=0, atol=1e-8)
    ctx.destroy()


def test_exact_rls_labels_match_the_oracle():
    """Exact per-geometry labels (dense eigendecomposition in the library) against the oracle's
    tau = diag(K (K + lam I)^-1) from a dense inverse, summed over each geometry's 3N columns.
    lam = 1e-4 keeps the scores' sensitivity to the eigenvalues' rounding (~n eps |K| / lam)
    far below the tolerance."""
    tm = synth.template(9, 5)
    R = synth.geometries(tm, 120, 0.1, 6)
    lam = 1e-4
    ctx = gdml.kernel_setup(torch.from_numpy(R).cuda(), 10.0, lam)
    got = gdml.geometry_labels(ctx, exact=True).cpu().numpy()
    est = gdml.geometry_labels(ctx, k=400, seed=2).cpu().numpy()
    ctx.destroy()
    K = ok.force_kernel_dense(R, 10.0)
    tau = op.rls_exact(K, lam)
    ref = tau.reshape(120, 27).sum(axis=1)
    print(f"exact labels: max |gpu - oracle| = {np.abs(got - ref).max():.2e}; Nystrom estimate k=400 "
          f"differs by {np.abs(est - ref).max():.2e}")
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-7)
    assert np.all(est <= ref + 1e-6)  # the Nystrom estimate never exceeds the exact scores


def test_learned_selection_solves_with_pivchol_as_referee():
    train = [synth.make_workload(f"t{s}", 9, 200, 0.05, 10.0, 1e-10, 200, "uniform", template_seed=0,
                                 noise_seed=100 + s) for s in range(4)]
    Xs, ys = [], []
    for w in train:
        c = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam)
        Xs.append(c.descriptors())
        ys.append(gdml.geometry_labels(c, 200))
        c.destroy()
    X = torch.cat(Xs)
    y = torch.cat(ys)
    s = gdml.Scorer(X.shape[1], 256, seed=0)
    s.fit_scaling(X, y)
    s.train(X, y, epochs=40, batch=256, lr=1e-3)
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam)
    yd = torch.from_numpy(w.y).cuda()
    ctx.precond_build("pivchol", 200)
    _, it_pc, rel_pc, _ = ctx.pcg_solve(yd)
    piv = ctx.precond_build_scored(s.predict(ctx.descriptors()), 200, pivots=True)
    assert len(set(piv.cpu().tolist())) == 200
    # the learned preconditioner on its own (no referee cap), then through the referee
    _, it_l, rel_l, _ = ctx.pcg_solve(yd, raise_on_nonconvergence=False)
    a, it, rel, used = gdml.solve_learned(ctx, s, yd, 200, referee_iters=it_pc)
    print(f"learned selection: {it_l} iterations vs pivoted Cholesky {it_pc} (ratio {it_l / it_pc:.2f}); "
          f"referee chose {used}")
    assert rel <= 1e-8
    # the referee keeps the learned preconditioner exactly when it converged within 1.5x
    assert used == ("learned" if (rel_l <= 1e-8 and it_l <= 1.5 * it_pc) else "pivchol")
    if used == "learned":
        assert it == it_l
    ctx.destroy()
    s.destroy()
