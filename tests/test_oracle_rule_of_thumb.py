"""Pins of the rule-of-thumb oracle (Sec. 4.3, Eqs. 7-8, Table 1) against what the
paper and the mathematics fix: Table 1's printed parameters, the stationary-point
closed form of Eq. 8, the end points of the runtime model, and its scaling in n."""
import math
import os

import numpy as np
import pytest

from oracle import rule_of_thumb as rot

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rule_of_thumb_table1.txt")


def table1():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, _atoms, m, k_min = line.split()
        rows[name] = (float(m), float(k_min))
    return rows


def closed_form(n, m, k_min):
    """Eq. 8's right-hand side: the stationary point of the model over real k."""
    return (k_min ** m * m * n * n / 2.0) ** (1.0 / (2.0 + m))


def test_oracle_table_is_table_1():
    assert rot.TABLE1 == table1()


CASES = [(n, m, k) for n in (50, 1000, 5400, 31000, 63000, 157500, 500000)
         for (m, k) in table1().values()] + [(63000, 2.5, 7.0), (1000, 0.2, 900.0), (20, 1.0, 5000.0)]


@pytest.mark.parametrize("n,m,k_min", CASES)
def test_argmin_is_floor_or_ceil_of_the_closed_form(n, m, k_min):
    """The model is convex in k > 0, so its integer minimiser over [1, n] is floor or ceil of
    the real stationary point (clamped), whichever costs less."""
    k = rot.k_rule_of_thumb(n, m, k_min)
    ks = closed_form(n, m, k_min)
    cands = sorted({min(max(c, 1), n) for c in (math.floor(ks), math.ceil(ks))})
    assert k in cands
    cost = [float(rot.runtime_model(c, n, m, k_min)) for c in cands]
    assert float(rot.runtime_model(k, n, m, k_min)) == pytest.approx(min(cost), rel=1e-14)


@pytest.mark.parametrize("n,m,k_min", [(63000, 1.0, 100.0), (31000, 1.14, 236.0), (500000, 0.73, 89.0)])
def test_minimum_is_a_discrete_local_minimum_and_the_derivative_changes_sign(n, m, k_min):
    k = rot.k_rule_of_thumb(n, m, k_min)
    c = lambda x: float(rot.runtime_model(x, n, m, k_min))
    assert c(k) <= c(k - 1) and c(k) <= c(k + 1)
    # d cost / dk = -m k_min^m k^-(m+1) + 2 k / n^2: negative below the optimum, positive above
    d = lambda x: -m * k_min ** m * x ** (-m - 1) + 2 * x / n ** 2
    assert d(k - 1) < 0 < d(k + 1)


def test_default_row_at_the_aspirin_system_size():
    """m = 1, k_min = 100 at n = 63000: k* = (100 n^2 / 2)^(1/3) = 5832.89, so k = 5833."""
    assert rot.k_rule_of_thumb(63000) == 5833
    assert abs(closed_form(63000, 1.0, 100.0) - 5832.889) < 1e-3


@pytest.mark.parametrize("m,k_min", [(1.0, 100.0), (1.14, 236.0), (0.73, 89.0)])
def test_model_recovers_the_closed_form_cost_at_both_ends(m, k_min):
    """Sec. 4.3: at k = k_min the PCG term is 1 and at k = n the build term is 1, so both ends
    cost about as much as the cubic closed-form solve.  At the stationary point the build
    term is m/2 times the PCG term, so the optimum costs (1 + m/2) (k_min / k*)^m."""
    n = 63000
    assert rot.runtime_model(k_min, n, m, k_min) == pytest.approx(1.0 + (k_min / n) ** 2, rel=1e-15)
    assert rot.runtime_model(n, n, m, k_min) == pytest.approx(1.0 + (k_min / n) ** m, rel=1e-15)
    ks = closed_form(n, m, k_min)
    assert rot.runtime_model(ks, n, m, k_min) == pytest.approx((1.0 + m / 2.0) * (k_min / ks) ** m, rel=1e-13)
    k = rot.k_rule_of_thumb(n, m, k_min)
    assert rot.runtime_model(k, n, m, k_min) == pytest.approx(rot.runtime_model(ks, n, m, k_min), rel=1e-6)


def test_scaling_in_n():
    """k* grows like n^(2/(2+m)): 8x the kernel size gives 4x the columns at m = 1."""
    for m in (1.0, 0.5, 2.0):
        k1 = rot.k_rule_of_thumb(10000, m, 50.0)
        k8 = rot.k_rule_of_thumb(80000, m, 50.0)
        ratio = 8.0 ** (2.0 / (2.0 + m))
        assert abs(k8 / k1 - ratio) <= (1.0 + ratio) / k1  # each k within 1 of its k*


def test_clamped_to_one_and_n():
    assert rot.k_rule_of_thumb(1, 1.0, 100.0) == 1
    assert rot.k_rule_of_thumb(30, 1.0, 5000.0) == 30  # k* > n: every k is worse than n
    assert rot.k_rule_of_thumb(10 ** 6, 1.0, 1e-15) == 1  # k* = (1e-15 n^2 / 2)^(1/3) < 1


def test_bad_arguments_raise():
    for args in ((0, 1.0, 100.0), (100, 0.0, 100.0), (100, 1.0, -1.0)):
        with pytest.raises(ValueError):
            rot.k_rule_of_thumb(*args)


def test_planted_exponent_error_is_caught(monkeypatch):
    """A build term (k / n) instead of (k / n)^2 moves the optimum off Eq. 8's closed form."""
    monkeypatch.setattr(rot, "runtime_model", lambda k, n, m, k_min: (k_min / np.asarray(k, float)) ** m
                        + np.asarray(k, float) / n)
    k = rot.k_rule_of_thumb(63000, 1.0, 100.0)
    assert k not in (math.floor(closed_form(63000, 1.0, 100.0)), math.ceil(closed_form(63000, 1.0, 100.0)))
