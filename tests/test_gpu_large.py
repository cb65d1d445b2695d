"""The 630,000-unknown system (N=42 atoms, M=5000 geometries, D=861): the GPU
matvec in FP64 / DF64 / TF32 / BF16 against the oracle on sampled geometry
blocks (the full oracle matvec would take minutes), and basic invariants."""
import numpy as np
import pytest
import torch

from oracle import kernel as ok
from paper_2212_12737_gb300 import gdml, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2212_12737_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return synth.workload("mol42_m5000")


@pytest.fixture(scope="module")
def sampled(big):
    w = big
    v = np.random.default_rng(11).standard_normal(w.n)
    rows = [0, 1234, 2500, 4999]
    ref = ok.matvec_rows(w.R, w.sigma, v, rows, w.lam)
    return v, rows, ref


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("df64", 1e-12), ("ozaki", 1e-12), ("tf32", 5e-3),
                                      ("bf16", 5e-2)])
def test_full_size_matvec_on_sampled_blocks(big, sampled, prec, tol):
    w = big
    v, rows, ref = sampled
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).cuda(), w.sigma, w.lam, precision=prec)
    got = ctx.matvec(torch.from_numpy(v).cuda()).cpu().numpy().reshape(w.M, -1)[rows]
    ctx.tc_check()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    emax = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"{prec} matvec at n={w.n}: relative error on sampled blocks {err:.2e} (elementwise {emax:.2e})")
    assert err <= tol
    if tol <= 1e-12:  # the FP64-class forms: elementwise too
        assert emax <= 1e-10
    ctx.destroy()


def test_full_size_rls_solve_reaches_rtol_by_the_oracle(big):
    """The 630,000-unknown system end to end in the OZAKI form: the leverage-score
    preconditioner at k = 5000 (pilot Nystrom factor, its core and the scores on the sliced
    tensor cores), PCG to a relative residual of 1e-8, and the oracle's own FP64 matvec
    recomputing the true residual of the GPU's alpha.  The evaluation error of that check
    is bounded by 8 eps |K|_2 |alpha| / |y|, with |K|_2 from a power iteration."""
    w = big
    eps = np.finfo(float).eps
    R, y = torch.from_numpy(w.R).cuda(), torch.from_numpy(w.y).cuda()
    ctx = gdml.kernel_setup(R, w.sigma, w.lam, precision="ozaki")
    tau = ctx.rls_scores(w.k, seed=2).cpu().numpy()
    assert tau.min() >= -1e-9 and tau.max() <= 1.0 + 1e-9 and tau.sum() <= w.k * (1.0 + 1e-9)
    piv, _ = ctx.precond_build("rls", w.k, seed=2, pivots=True)
    p = piv.cpu().numpy()
    assert len(np.unique(p)) == w.k and p.min() >= 0 and p.max() < w.n
    rank, _ = ctx.precond_info()
    assert rank == w.k
    alpha, iters, rel, _ = ctx.pcg_solve(y, rtol=1e-8, max_iter=20000)
    ctx.tc_check()
    v = torch.from_numpy(np.random.default_rng(3).standard_normal(w.n)).cuda()
    for _ in range(30):
        v = ctx.matvec(v, add_lambda=False)
        knorm = float(torch.linalg.norm(v))
        v = v / knorm
    ctx.destroy()
    a = alpha.cpu().numpy()
    res = np.linalg.norm(w.y - ok.matvec_parallel(w.R, w.sigma, a, w.lam)) / np.linalg.norm(w.y)
    bound = 8 * eps * knorm * np.linalg.norm(a) / np.linalg.norm(w.y)
    print(f"n={w.n} rls k={w.k}: {iters} PCG iterations, GPU relres {rel:.2e}, oracle relres {res:.2e} "
          f"(evaluation bound {bound:.1e})")
    assert rel <= 1e-8
    assert res <= 1e-8 + bound
