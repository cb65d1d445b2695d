"""gdml_rule_of_thumb_k (host arithmetic in the C library, no GPU needed) against the
oracle's brute-force argmin of the runtime model (Sec. 4.3, Eqs. 7-8, Table 1).

Bit-exact integer parity, except where the model's costs at floor(k*) and ceil(k*)
tie to within 1e-13 relative: there both answers are correct and either is accepted,
since the two sides evaluate the power with different pow routines."""
import math
import os

import numpy as np
import pytest

from oracle import rule_of_thumb as rot

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rule_of_thumb_table1.txt")


@pytest.fixture(scope="module")
def gdml():
    from paper_2212_12737_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2212_12737_gb300 import gdml as g
    try:
        g.load()
    except OSError as e:  # no CUDA runtime to link against on this machine
        pytest.skip(f"cannot dlopen: {e}")
    return g


def table1():
    rows = {}
    for line in open(GOLDEN):
        if not line.startswith("#") and line.strip():
            name, _atoms, m, k_min = line.split()
            rows[name] = (float(m), float(k_min))
    return rows


def agrees(k_lib, n, m, k_min):
    k_ref = rot.k_rule_of_thumb(n, m, k_min)
    if k_lib == k_ref:
        return True
    c_lib, c_ref = (float(rot.runtime_model(k, n, m, k_min)) for k in (k_lib, k_ref))
    return abs(k_lib - k_ref) == 1 and abs(c_lib - c_ref) <= 1e-13 * c_ref


def test_binding_table_is_table_1(gdml):
    assert gdml.ROT_PARAMS == table1()


@pytest.mark.parametrize("molecule", sorted(table1()))
@pytest.mark.parametrize("n", [1, 2, 50, 5400, 31000, 63000, 157500, 504000])
def test_table_1_rows_match_the_oracle(gdml, molecule, n):
    m, k_min = table1()[molecule]
    assert agrees(gdml.rule_of_thumb_k(n, molecule), n, m, k_min)


def test_random_parameters_match_the_oracle(gdml):
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(np.exp(rng.uniform(0.0, np.log(2e5))))
        m = float(rng.uniform(0.3, 3.0))
        k_min = float(np.exp(rng.uniform(np.log(1e-2), np.log(1e4))))
        k = gdml.rule_of_thumb_k(n, m=m, k_min=k_min)
        assert 1 <= k <= n
        assert agrees(k, n, m, k_min), (n, m, k_min, k)


@pytest.mark.parametrize("n", [10 ** 8, 10 ** 12, 2 ** 62])
def test_sizes_beyond_brute_force_are_discrete_minima(gdml, n):
    """No overflow for huge n: the answer is floor or ceil of Eq. 8's closed form and no
    neighbour costs less (evaluated here in FP64)."""
    k = gdml.rule_of_thumb_k(n, m=1.0, k_min=100.0)
    ks = (100.0 * n * float(n) / 2.0) ** (1.0 / 3.0)
    assert k in (math.floor(ks), math.ceil(ks))
    c = lambda x: (100.0 / x) + (x / n) ** 2
    assert c(k) <= c(k - 1) * (1 + 1e-15) and c(k) <= c(k + 1) * (1 + 1e-15)


def test_default_row_at_the_aspirin_system_size(gdml):
    assert gdml.rule_of_thumb_k(63000) == 5833


@pytest.mark.parametrize("args", [(0, 1.0, 100.0), (-5, 1.0, 100.0), (100, 0.0, 100.0), (100, -1.0, 100.0),
                                  (100, float("nan"), 100.0), (100, 1.0, 0.0), (100, 1.0, float("inf")),
                                  (100, float("inf"), 100.0)])
def test_bad_arguments_are_rejected(gdml, args):
    n, m, k_min = args
    with pytest.raises(gdml.GdmlError) as e:
        gdml.rule_of_thumb_k(n, m=m, k_min=k_min)
    assert e.value.name == "ERR_ARG" and "rule_of_thumb_k" in str(e.value)
