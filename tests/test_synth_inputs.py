"""The seeded synthetic inputs: reproducible from their seeds, with the shapes and parameters
of the workloads the tests and the benchmark use (N atoms, M geometries, n = 3 N M,
D = N (N - 1) / 2), and a batched suite with the stated ranges."""
import numpy as np
import pytest

from paper_2212_12737_gb300 import synth

TABLE = {  # name: N, M, n, D, sigma, lambda, k, selection
    "ethanol9_m200": (9, 200, 5400, 36, 10.0, 1e-10, 100, "uniform"),
    "aspirin21_m1000": (21, 1000, 63000, 210, 20.0, 1e-10, 2000, "pivchol"),
}


@pytest.mark.parametrize("name", sorted(TABLE))
def test_workload_shapes_and_parameters(name):
    N, M, n, D, sigma, lam, k, select = TABLE[name]
    w = synth.workload(name)
    assert w.R.shape == (M, N, 3) and w.y.shape == (n,) and w.n == n
    assert N * (N - 1) // 2 == D
    assert (w.sigma, w.lam, w.k, w.select) == (sigma, lam, k, select)
    assert np.isfinite(w.R).all() and np.isfinite(w.y).all()


def test_workloads_are_reproducible_from_their_seeds():
    a, b = synth.workload("ethanol9_m200"), synth.workload("ethanol9_m200")
    assert np.array_equal(a.R, b.R) and np.array_equal(a.y, b.y)
    c = synth.workload("ethanol9_m200", noise_seed=2)
    assert not np.array_equal(a.R, c.R)


def test_geometries_fluctuate_around_one_template():
    tmpl = synth.template(9, 0)
    R = synth.geometries(tmpl, 500, 0.05, 1)
    dev = R - tmpl[None]
    assert abs(dev.std() - 0.05) < 0.005 and abs(dev.mean()) < 0.005


def test_batched_suite_ranges():
    suite = synth.batched_suite(count=16, mmax=400)
    assert len(suite) == 16
    for w in suite:
        assert w.N in (9, 12, 15, 21, 42) and 100 <= w.M <= 400
        assert w.sigma in (5.0, 10.0, 20.0, 40.0) and w.lam in (1e-10, 1e-8)
        assert w.k == max(1, w.M // 10) and w.select == "uniform"
    again = synth.batched_suite(count=16, mmax=400)
    assert all(np.array_equal(x.R, y.R) for x, y in zip(suite, again))
