"""Force prediction f_q = sum_b J_q^T H(x_q, x_b) J_b alpha_b (Sec. 2.1) through the C ABI
against the FP64 oracle.  Both sides are FP64 with different summation orders:
max |df| <= 1e-10 max |f|.  At the training geometries the prediction is K alpha, the
FP64 matvec without lambda, to 1e-12."""
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
    from paper_2212_12737_gb300 import build
    import os
    if not os.path.exists(build.LIB):
        build.build()
    gdml.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("Q", [1, 37])
def test_predicted_forces_match_the_oracle(prec, Q):
    tmpl = synth.template(7, 5)
    R = synth.geometries(tmpl, 150, 0.1, 6)
    Rq = synth.geometries(tmpl, Q, 0.12, 9)
    alpha = np.random.default_rng(3).standard_normal(R.size)
    ctx = gdml.kernel_setup(dev(R), 3.0, 1e-6, precision=prec)
    f = ctx.predict_forces(dev(Rq), dev(alpha)).cpu().numpy()
    ref = ok.predict_forces(Rq, R, 3.0, alpha)
    err = np.abs(f - ref).max() / np.abs(ref).max()
    print(f"predicted forces vs FP64 oracle ({prec}, Q = {Q}): {err:.2e}")
    assert err <= 1e-10
    ctx.destroy()


def test_prediction_at_the_training_set_is_the_matvec():
    w = synth.workload("ethanol9_m200")
    ctx = gdml.kernel_setup(dev(w.R), w.sigma, w.lam)
    alpha = dev(np.random.default_rng(4).standard_normal(w.n))
    f = ctx.predict_forces(dev(w.R), alpha).reshape(-1)
    kv = ctx.matvec_fp64(alpha, add_lambda=False)
    rel = float((f - kv).abs().max() / kv.abs().max())
    print(f"prediction at the training set vs K alpha: {rel:.2e}")
    assert rel <= 1e-12
    with pytest.raises(ValueError):
        ctx.predict_forces(dev(w.R[:, :5]), alpha)
    with pytest.raises(ValueError):
        ctx.predict_forces(dev(w.R), alpha[:-1])
    ctx.destroy()
