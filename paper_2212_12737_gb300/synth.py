"""Seeded synthetic molecular workloads (inputs only).

The paper trains on molecular-dynamics geometries with ab-initio force
labels (Sec. 4, MD17/MD22).  Those datasets are not available here, so this
module draws stand-in inputs with the same shapes and structure:

* one rigid "template" molecule of N atoms, drawn by random sequential
  addition inside a ball of radius N**(1/3) Angstrom with a minimum pair
  distance of 1.0 Angstrom;
* M geometries = template + isotropic Gaussian noise (std ``noise`` Angstrom
  per coordinate), mimicking near-equilibrium MD sampling;
* force labels y = F = -grad E of a Morse pair potential
  E = sum_{i<j} De * (1 - exp(-a (r_ij - r0_ij)))**2 with De = 1, a = 1/A
  and r0 = template distances.

Vector layout of y (and of every length-n vector of the method): index
``a*3N + 3*i + q`` for geometry a, atom i and Cartesian coordinate q, i.e.
the reshape n -> (n_train, d, 3) of App. A ("Atomic contribution").

This module holds none of the method's arithmetic (no descriptor, kernel,
preconditioner or solver); it is shared by the CPU oracle's tests and by the
GPU path's tests and benchmark so that both see identical inputs.
"""
from __future__ import annotations

import dataclasses
import numpy as np

MORSE_DE = 1.0
MORSE_A = 1.0


def template(N: int, seed: int, min_dist: float = 1.0) -> np.ndarray:
    """Random sequential addition of N atoms in a ball of radius N**(1/3)."""
    rng = np.random.default_rng([seed, 0x7E1])
    radius = 1.0 * N ** (1.0 / 3.0)
    atoms: list[np.ndarray] = []
    tries = 0
    while len(atoms) < N:
        tries += 1
        if tries > 1_000_000:
            raise RuntimeError("template: could not place atoms")
        p = rng.uniform(-radius, radius, size=3)
        if p @ p > radius * radius:
            continue
        if atoms and np.min(np.linalg.norm(np.asarray(atoms) - p, axis=1)) < min_dist:
            continue
        atoms.append(p)
    return np.asarray(atoms, dtype=np.float64)


def geometries(tmpl: np.ndarray, M: int, noise: float, seed: int) -> np.ndarray:
    """M noisy copies of the template, shape (M, N, 3), Angstrom."""
    rng = np.random.default_rng([seed, 0x9E0])
    return tmpl[None, :, :] + noise * rng.standard_normal((M, tmpl.shape[0], 3))


def morse_forces(R: np.ndarray, tmpl: np.ndarray) -> np.ndarray:
    """Analytic Morse forces F = -dE/dR, shape (M, N, 3)."""
    N = tmpl.shape[0]
    r0 = np.linalg.norm(tmpl[:, None, :] - tmpl[None, :, :], axis=-1)
    diff = R[:, :, None, :] - R[:, None, :, :]  # (M, N, N, 3): R_i - R_j
    r = np.linalg.norm(diff, axis=-1)
    np.einsum("mii->mi", r)[...] = 1.0  # avoid 0/0 on the diagonal
    ex = np.exp(-MORSE_A * (r - r0[None]))
    dEdr = 2.0 * MORSE_DE * MORSE_A * (1.0 - ex) * ex
    idx = np.arange(N)
    dEdr[:, idx, idx] = 0.0
    return -np.einsum("mij,mijq->miq", dEdr / r, diff)


def morse_energy(R: np.ndarray, tmpl: np.ndarray) -> np.ndarray:
    """Morse energy per geometry, shape (M,)."""
    N = tmpl.shape[0]
    iu = np.triu_indices(N, 1)
    r0 = np.linalg.norm(tmpl[:, None, :] - tmpl[None, :, :], axis=-1)[iu]
    r = np.linalg.norm(R[:, :, None, :] - R[:, None, :, :], axis=-1)[:, iu[0], iu[1]]
    return np.sum(MORSE_DE * (1.0 - np.exp(-MORSE_A * (r - r0))) ** 2, axis=1)


@dataclasses.dataclass
class Workload:
    """One kernel system: geometries R (M,N,3), labels y (n,), sigma, lambda."""

    name: str
    R: np.ndarray
    y: np.ndarray
    sigma: float
    lam: float
    k: int
    select: str  # "uniform" | "rls" | "pivchol"

    @property
    def M(self) -> int:
        return self.R.shape[0]

    @property
    def N(self) -> int:
        return self.R.shape[1]

    @property
    def n(self) -> int:
        return 3 * self.M * self.N


def make_workload(name: str, N: int, M: int, noise: float, sigma: float, lam: float,
                  k: int, select: str, template_seed: int = 0, noise_seed: int = 1) -> Workload:
    tmpl = template(N, template_seed)
    R = geometries(tmpl, M, noise, noise_seed)
    y = morse_forces(R, tmpl).reshape(-1)
    return Workload(name, R, y, sigma, lam, k, select)


# The paper-shaped workloads (atom counts of ethanol / aspirin / a 42-atom
# molecule; kernel sizes n = 5.4k, 63k and 630k).
WORKLOADS = {
    "ethanol9_m200": dict(N=9, M=200, noise=0.05, sigma=10.0, lam=1e-10, k=100, select="uniform"),
    "aspirin21_m1000": dict(N=21, M=1000, noise=0.05, sigma=20.0, lam=1e-10, k=2000, select="pivchol"),
    "mol42_m5000": dict(N=42, M=5000, noise=0.1, sigma=30.0, lam=1e-9, k=5000, select="rls"),
}


def workload(name: str, **override) -> Workload:
    cfg = dict(WORKLOADS[name])
    cfg.update(override)
    return make_workload(name, **cfg)


def batched_suite(count: int = 64, seed: int = 42, mmax: int = 2000) -> list[Workload]:
    """Many uneven systems: N in {9,12,15,21,42}, M in [100, mmax] (2000 by default),
    sigma in {5,10,20,40}, lambda in {1e-10, 1e-8}, uniform k = M // 10."""
    rng = np.random.default_rng([seed, 0xBA7])
    out = []
    for s in range(count):
        N = int(rng.choice([9, 12, 15, 21, 42]))
        M = int(rng.integers(100, 2001))
        M = 100 + (M - 100) * (mmax - 100) // 1900 if mmax < 2000 else M
        sigma = float(rng.choice([5.0, 10.0, 20.0, 40.0]))
        lam = float(rng.choice([1e-10, 1e-8]))
        out.append(make_workload(f"batch{s}", N, M, 0.05, sigma, lam, max(1, M // 10), "uniform",
                                 template_seed=1000 + s, noise_seed=2000 + s))
    return out
