"""Many uneven systems in one graph launch, and the split-K autotuner, against
per-system solves and the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
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


def systems():
    rng = np.random.default_rng(7)
    out = []
    for s in range(6):
        N = int(rng.choice([5, 7, 9]))
        M = int(rng.integers(20, 121))
        sigma = float(rng.choice([2.0, 5.0, 10.0]))
        lam = float(rng.choice([1e-8, 1e-6]))
        w = synth.make_workload(f"b{s}", N, M, 0.1, sigma, lam, max(1, M // 10) * 3, "uniform",
                                template_seed=100 + s, noise_seed=200 + s)
        out.append(w)
    return out


def test_batched_solve_matches_per_system_solves_and_oracle():
    ws = systems()
    ctxs, ys = [], []
    for w in ws:
        c = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam)
        c.precond_build("uniform", w.k, seed=2)
        ctxs.append(c)
        ys.append(torch.from_numpy(w.y).cuda())
    alphas, iters, rels = gdml.pcg_solve_batched(ctxs, ys, rtol=1e-8)
    for w, c, y, a, it, rel in zip(ws, ctxs, ys, alphas, iters, rels):
        single, it1, rel1, _ = c.pcg_solve(y, rtol=1e-8)
        assert it == it1 and abs(rel - rel1) <= 1e-12 * max(rel1, 1e-300)
        assert torch.equal(a, single)  # same kernels, same order: bitwise equal
        an = a.cpu().numpy()
        K = ok.force_kernel_dense(w.R, w.sigma)
        res = np.linalg.norm(w.y - K @ an - w.lam * an) / np.linalg.norm(w.y)
        bound = 8 * np.finfo(float).eps * np.linalg.norm(K, 2) * np.linalg.norm(an) / np.linalg.norm(w.y)
        assert rel <= 1e-8 and res <= 1e-8 + bound
        c.destroy()


def test_batched_solve_rejects_bad_batches():
    w = systems()[0]
    c = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam)
    y = torch.from_numpy(w.y).cuda()
    with pytest.raises(gdml.GdmlError):
        gdml.pcg_solve_batched([c, c], [y, y])  # a context twice
    t = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision="tf32")
    with pytest.raises(gdml.GdmlError):
        gdml.pcg_solve_batched([t], [y])  # tensor-core contexts are refined one by one
    c.destroy()
    t.destroy()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_autotune_keeps_results_and_caches(prec, tmp_path):
    w = synth.workload("ethanol9_m200")
    c = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision=prec)
    v = torch.from_numpy(np.random.default_rng(0).standard_normal(w.n)).cuda()
    ref = c.matvec(v).clone()
    cache = str(tmp_path / "tune.json")
    choice = c.autotune(cache)
    assert choice >= 1
    got = c.matvec(v)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) <= tol
    c2 = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision=prec)
    assert c2.autotune(cache) == choice  # read back from the cache
    c.destroy()
    c2.destroy()
