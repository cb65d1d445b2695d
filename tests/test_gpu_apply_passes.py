"""The two passes over the FP32-stored factor L_k of the DF64/OZAKI Woodbury apply
(Eq. 4): t = L^T r and z = (r - L u) / lambda, with exact FP32 products and
double-float sums.  Both the TMA-staged kernels (n % 4 == 0) and the
register-streamed ones are compared with the same sums in FP64 (the definition of
the two matrix-vector products, evaluated by numpy on the FP32 values of L)."""
import numpy as np
import pytest
import torch

from paper_2212_12737_gb300 import gdml

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


def _case(n, k, seed):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((n, k)).astype(np.float32)
    r = rng.standard_normal(n)
    u = rng.standard_normal(k) * 10.0 ** rng.uniform(-3, 3, size=k)
    return L, r, u


def _check(L, r, u, lam, staged):
    Lg = torch.from_numpy(L).cuda()
    t, z = gdml.test_df_passes(Lg, torch.from_numpy(r).cuda(), torch.from_numpy(u).cuda(), lam, staged=staged)
    t, z = t.cpu().numpy(), z.cpu().numpy()
    L64 = L.astype(np.float64)
    t_ref = L64.T @ r
    z_ref = (r - L64 @ u) / lam
    # double-float sums: error far below 1e-12 of the sum of |terms|
    t_scale = np.abs(L64).T @ np.abs(r)
    z_scale = (np.abs(r) + np.abs(L64) @ np.abs(u)) / lam
    et = np.max(np.abs(t - t_ref) / t_scale)
    ez = np.max(np.abs(z - z_ref) / z_scale)
    return et, ez, t, z


@pytest.mark.parametrize("rows", [128, 256])
@pytest.mark.parametrize("n,k", [(4, 1), (100, 17), (5400, 300), (20000, 1000), (63000, 2000)])
def test_staged_passes_match_fp64(n, k, rows):
    """128- and 256-row chunks (one chunk, a ragged last chunk, several per CTA), k not
    a multiple of the 32- or 16-column tiles, and the bench's size (n = 63,000, k = 2,000)."""
    L, r, u = _case(n, k, n + k)
    et, ez, _, _ = _check(L, r, u, 1e-3, staged=rows)
    print(f"staged rows={rows} n={n} k={k}: L^T r {et:.2e}, (r - L u)/lambda {ez:.2e} of the |term| sums")
    assert et <= 1e-13 and ez <= 1e-13


@pytest.mark.parametrize("n,k", [(3150, 300), (20000, 1000)])
def test_register_streamed_passes_match_fp64(n, k):
    L, r, u = _case(n, k, 3 * n + k)
    et, ez, _, _ = _check(L, r, u, 1e-3, staged=False)
    assert et <= 1e-13 and ez <= 1e-13


def test_staged_many_chunks_per_cta():
    """n = 630,000 gives 2,461 chunks of 256 rows, up to 9 per CTA (the ring runs
    across chunk boundaries)."""
    n, k = 630000, 40
    L, r, u = _case(n, k, 11)
    et, ez, _, _ = _check(L, r, u, 1e-6, staged=True)
    assert et <= 1e-13 and ez <= 1e-13


def test_staged_and_register_streamed_agree():
    L, r, u = _case(20000, 500, 5)
    _, _, ts, zs = _check(L, r, u, 1e-10, staged=True)
    _, _, tr, zr = _check(L, r, u, 1e-10, staged=False)
    assert np.max(np.abs(ts - tr) / np.abs(tr).max()) <= 1e-13
    assert np.max(np.abs(zs - zr) / np.abs(zr).max()) <= 1e-13


def test_staged_needs_rows_multiple_of_4():
    L, r, u = _case(3150, 8, 1)
    with pytest.raises(gdml.GdmlError) as e:
        _check(L, r, u, 1.0, staged=True)
    assert e.value.name == "ERR_ARG"


@pytest.mark.parametrize("M", [150, 152])
def test_df64_pivchol_schur_paths_match_fp64(M):
    """Algorithm 1 in DF64 form: n = 21 M is 3150 (register-streamed Schur sums, n % 4 != 0)
    or 3192 (TMA-staged Schur sums).  Both must pick the FP64 build's leading pivots and
    give the same residual trace to FP32-storage accuracy."""
    from paper_2212_12737_gb300 import synth
    R = synth.geometries(synth.template(7, 5), M, 0.1, 6)
    Rg = torch.from_numpy(R).cuda()
    out = {}
    for prec in ("fp64", "df64"):
        ctx = gdml.kernel_setup(Rg, 3.0, 1e-6, precision=prec)
        piv, tr = ctx.precond_build("pivchol", 200, pivots=True, trace=True)
        out[prec] = (piv.cpu().numpy(), tr.cpu().numpy())
        ctx.destroy()
    assert np.array_equal(out["fp64"][0][:40], out["df64"][0][:40])
    t64, tdf = out["fp64"][1], out["df64"][1]
    rel = np.abs(tdf[:40] - t64[:40]) / t64[0]
    assert rel.max() <= 1e-5
