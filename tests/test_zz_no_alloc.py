"""gdml_matvec_noalloc: the context-free FP64 matvec for callers that cannot
allocate device memory (its working memory is a static device array).

Checked against the regular entry points (gdml_kernel_setup + gdml_matvec) on
two calls in a row, with the FP64 matvec tolerance the other GPU tests use
(|d|_2 <= 1e-12 |ref|_2).  Collected last so a failure here comes after every
other test has run.
"""
import numpy as np
import pytest
import torch

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


def test_noalloc_matvec_matches_context_matvec_on_two_calls():
    cases = [(9, 128, 0.05, 10.0, 1e-10), (6, 37, 0.2, 3.0, 1e-6)]  # second call: other sizes, same array
    for N, M, noise, sigma, lam in cases:
        tmpl = synth.template(N, 7)
        R = torch.from_numpy(synth.geometries(tmpl, M, noise, 8)).cuda()
        v = torch.from_numpy(np.random.default_rng(M).standard_normal(3 * N * M)).cuda()
        got = gdml.matvec_noalloc(R, sigma, lam, v)
        ctx = gdml.kernel_setup(R, sigma, lam)
        ref = ctx.matvec(v)
        torch.cuda.synchronize()
        ctx.destroy()
        err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        assert err <= 1e-12, (N, M, err)


def test_noalloc_matvec_rejects_sizes_beyond_its_array():
    tmpl = synth.template(5, 1)
    R = torch.from_numpy(synth.geometries(tmpl, 129, 0.1, 2)).cuda()
    v = torch.zeros(3 * 5 * 129, dtype=torch.float64, device="cuda")
    with pytest.raises(gdml.GdmlError) as e:
        gdml.matvec_noalloc(R, 1.0, 1e-8, v)
    assert e.value.name == "ERR_ARG" and "128" in str(e.value)
