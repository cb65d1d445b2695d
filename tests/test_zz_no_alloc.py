"""gdml_matvec_noalloc: the context-free FP64 matvec for callers that cannot
allocate device memory (its working memory is a static device array).

Each case is checked on two calls in a row (the second reuses the array the
first one left behind) against
* the FP64 CPU oracle (oracle.kernel.matvec), with the tolerances of the other
  FP64 matvec parity tests: |d|_2 <= 1e-12 |ref|_2 and max |d| <= 1e-10 max |ref|;
* the regular entry points (gdml_kernel_setup + gdml_matvec), same bound.
The largest case, N = 24 atoms and M = 128 geometries, fills the array exactly.
Collected last so a failure here comes after every other test has run.
"""
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


def _close(got, ref):
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("N,M,noise,sigma,lam", [
    (24, 128, 0.05, 10.0, 1e-10),  # the array's limit: 7 M D + 4 M^2 + 2 M doubles exactly
    (9, 128, 0.05, 10.0, 1e-10),
    (6, 37, 0.2, 3.0, 1e-6),       # ragged sizes on the array a larger call left behind
    (2, 1, 0.1, 1.5, 0.0),         # one geometry of two atoms, no lambda
])
def test_noalloc_matvec_matches_oracle_and_context_on_two_calls(N, M, noise, sigma, lam):
    tmpl = synth.template(N, 7)
    Rn = synth.geometries(tmpl, M, noise, 8)
    R = torch.from_numpy(Rn).cuda()
    rng = np.random.default_rng(M + N)
    ctx = gdml.kernel_setup(R, sigma, lam if lam > 0 else 1e-12)
    for _ in range(2):
        vn = rng.standard_normal(3 * N * M)
        v = torch.from_numpy(vn).cuda()
        got = gdml.matvec_noalloc(R, sigma, lam, v).cpu().numpy()
        _close(got, ok.matvec(Rn, sigma, vn, lam))
        ref = ctx.matvec(v, add_lambda=False).cpu().numpy() + lam * vn
        _close(got, ref)
    ctx.destroy()


def test_noalloc_matvec_rejects_sizes_beyond_its_array():
    for N, M in ((5, 129), (25, 3)):
        tmpl = synth.template(N, 1)
        R = torch.from_numpy(synth.geometries(tmpl, M, 0.1, 2)).cuda()
        v = torch.zeros(3 * N * M, dtype=torch.float64, device="cuda")
        with pytest.raises(gdml.GdmlError) as e:
            gdml.matvec_noalloc(R, 1.0, 1e-8, v)
        assert e.value.name == "ERR_ARG" and ("128" in str(e.value) and "24" in str(e.value))


def test_noalloc_matvec_binding_rejects_wrong_vectors():
    tmpl = synth.template(4, 1)
    R = torch.from_numpy(synth.geometries(tmpl, 3, 0.1, 2)).cuda()
    n = 3 * 4 * 3
    with pytest.raises(ValueError):
        gdml.matvec_noalloc(R, 1.0, 1e-8, torch.zeros(n, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        gdml.matvec_noalloc(R, 1.0, 1e-8, torch.zeros(n - 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        gdml.matvec_noalloc(R, 1.0, 1e-8, torch.zeros(n, dtype=torch.float64, device="cuda"),
                            out=torch.zeros(n + 3, dtype=torch.float64, device="cuda"))
