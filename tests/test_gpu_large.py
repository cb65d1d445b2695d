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
    print(f"{prec} matvec at n={w.n}: relative error on sampled blocks {err:.2e}")
    assert err <= tol
    ctx.destroy()
