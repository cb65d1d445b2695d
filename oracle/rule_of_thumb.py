"""Oracle: preconditioner size from the runtime model (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 4.3 models the cost of a preconditioned solve as the k^2 n of building the
preconditioner plus the PCG cost, whose normalised iteration count falls as a power
law (k_min / k)^m in the number k of inducing columns:

* runtime[k] ~ n^3 [ (k_min / k)^m + (k / n)^2 ]                        (Eq. 7)
* k_RoT = the k in [1, n] that minimises runtime[k]                    (Eq. 8)

with (m, k_min) per molecule from Table 1 and the default row m = 1,
k_min = 100.  Here k_RoT is that definition written out: the integer argmin
of Eq. 7 over every k in [1, n], found by evaluating all of them.  The
stationary-point closed form that Eq. 8 also states is a pin (a test), not
part of this module.

Readings where the paper is silent:
* k is an integer in [1, n]; ties between two integers go to the smaller k;
* the n^3 factor of Eq. 7 is dropped (it does not move the minimum).
"""
from __future__ import annotations

import numpy as np

# Table 1: molecule -> (m, k_min), measured at n = 31k; "default" is the row the
# paper recommends for molecules without fitted parameters.
TABLE1 = {
    "default": (1.0, 100.0),
    "ethanol": (0.87, 10.0),
    "uracil": (1.07, 32.0),
    "toluene": (1.01, 44.0),
    "aspirin": (1.14, 236.0),
    "azobenzene": (1.02, 62.0),
    "catcher": (1.02, 316.0),
    "nanotube": (0.73, 89.0),
}


def runtime_model(k, n: int, m: float, k_min: float):
    """Eq. 7 without its n^3 factor: (k_min / k)^m + (k / n)^2 (k may be an array)."""
    k = np.asarray(k, dtype=np.float64)
    return (k_min / k) ** m + (k / n) ** 2


def k_rule_of_thumb(n: int, m: float = 1.0, k_min: float = 100.0) -> int:
    """Eq. 8: the integer k in [1, n] with the smallest Eq. 7 cost (first one on a tie)."""
    if n < 1 or not (m > 0) or not (k_min > 0):
        raise ValueError("need n >= 1, m > 0, k_min > 0")
    ks = np.arange(1, n + 1, dtype=np.float64)
    return int(np.argmin(runtime_model(ks, n, m, k_min))) + 1
