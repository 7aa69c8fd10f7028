"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the method: only the random locations and
random vectors of the workloads.  Locations are uniform in the unit square,
as in the paper's synthetic experiments (Sec. 5: locations in [0,1]^2, data
drawn as Z = L xi with xi ~ N(0, I)).  The moisture / real-location data sets
the paper also uses are not available; these draws stand in for them.

Seeds: locations of workload c use ``1000 + c``; its random vector ``2000 + c``.
"""
from __future__ import annotations

import numpy as np

# The workloads, by their sizes and parameters.
WORKLOADS = {
    # n=2000: exponential Matern, plain FP64 H-matrix vs the dense oracle.
    "n2000_nu0.5_eps1e-7": dict(index=1, n=2000, sigma2=1.0, ell=0.1, nu=0.5, nugget=1e-4,
                                leaf=32, eta=2.0, eps=1e-7, z="dense_factor"),
    # n=65,536: the closed-form nu=3/2 kernel and a general-nu Bessel kernel.
    "n65536_nu1.5_eps1e-6": dict(index=2, n=65536, sigma2=1.0, ell=0.05, nu=1.5, nugget=1e-4,
                                 leaf=64, eta=2.0, eps=1e-6, z="normal"),
    "n65536_nu0.325_eps1e-6": dict(index=2, n=65536, sigma2=1.0, ell=0.05, nu=0.325, nugget=1e-4,
                                   leaf=64, eta=2.0, eps=1e-6, z="normal"),
    # n=524,288: the throughput workload.
    "n524288_nu0.5_eps1e-5": dict(index=3, n=524288, sigma2=1.0, ell=0.0864, nu=0.5, nugget=1e-4,
                                  leaf=64, eta=2.0, eps=1e-5, z="normal"),
    "n524288_nu0.5_eps1e-7": dict(index=3, n=524288, sigma2=1.0, ell=0.0864, nu=0.5, nugget=1e-4,
                                  leaf=64, eta=2.0, eps=1e-7, z="normal"),
}


def points(n: int, seed: int) -> np.ndarray:
    """n uniform locations in [0,1]^2, shape (n, 2), float64, row-major."""
    return np.random.default_rng(seed).random((n, 2))


def normal(n: int, seed: int) -> np.ndarray:
    """n independent N(0, 1) draws, float64."""
    return np.random.default_rng(seed).standard_normal(n)


def workload_points(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return points(w["n"], 1000 + w["index"])


def workload_normal(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return normal(w["n"], 2000 + w["index"])


def theta_jitter(base: dict, k: int, seed: int = 77) -> dict:
    """The k-th of a sequence of parameter sets within +-5 % of ``base``
    (sigma2, ell, nu), used to vary theta between timed evaluations."""
    rng = np.random.default_rng(seed + k)
    f = 1.0 + 0.05 * (2.0 * rng.random(3) - 1.0)
    out = dict(base)
    out["sigma2"] = base["sigma2"] * f[0]
    out["ell"] = base["ell"] * f[1]
    out["nu"] = base["nu"] * f[2]
    return out
