"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds NO arithmetic of the k-nearest-neighbour method: it only
draws points.  Every array comes from numpy's Philox counter-based generator
keyed by an explicit seed, so the same call gives the same bytes on every
host (x86 or Arm) and the GPU path and the oracle always see identical input.

The paper does not state the distribution of its timing workloads
(Sec. 3, Table 1); the recipes below are the synthetic stand-ins, each with
the shapes of the paper's experiments or of the workload it names.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def uniform(rows: int, d: int, seed: int) -> np.ndarray:
    """rows x d float32 points, i.i.d. uniform in [0, 1)."""
    return rng(seed).random((int(rows), int(d)), dtype=np.float32)


def gaussian_mixture(rows: int, d: int, n_centres: int, sigma: float,
                     seed_centres: int, seed_points: int) -> np.ndarray:
    """rows x d float32 points: a centre drawn uniformly from n_centres centres
    (the centres themselves uniform in [0,1)^d), plus N(0, sigma^2) per
    coordinate.  The centres depend only on seed_centres, so queries drawn
    with another seed_points come from the same mixture."""
    centres = rng(seed_centres).random((int(n_centres), int(d)), dtype=np.float32)
    g = rng(seed_points)
    which = g.integers(0, n_centres, size=int(rows))
    noise = g.standard_normal((int(rows), int(d)), dtype=np.float32) * np.float32(sigma)
    return (centres[which] + noise).astype(np.float32)


def lattice(side: int, d: int, spacing: float = 1.0) -> np.ndarray:
    """All points of {0, 1, .., side-1}^d (times spacing) in row-major order:
    the point with coordinates (x_0, .., x_{d-1}) has index
    sum_t x_t * side^(d-1-t)."""
    axes = [np.arange(side, dtype=np.float32) * np.float32(spacing)] * d
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in grid], axis=1).astype(np.float32)


# Named workloads.  Sizes follow Table 1 of the paper (N = n = m, D, k = 20)
# and the larger synthetic workloads of the precision, batching and serving
# forms.  Seeds are fixed here so every consumer regenerates identical data.
WORKLOADS = {
    "uniform_n1200_d8_k20": dict(m=1200, n=1200, d=8, k=20, seed_r=1, seed_q=2,
                                 dist="uniform"),
    "uniform_n38400_d96_k20": dict(m=38400, n=38400, d=96, k=20, seed_r=3, seed_q=4,
                                   dist="uniform"),
    "mixture_m1048576_n16384_d128_k100": dict(m=1048576, n=16384, d=128, k=100,
                                              n_centres=1024, sigma=0.05,
                                              seed_centres=7, seed_r=8, seed_q=9,
                                              dist="mixture"),
    # serving: a resident reference set; requests draw their queries from a
    # seeded pool (uniform, like the references)
    "serve_m4194304_d96": dict(m=4194304, d=96, seed_r=6, seed_q=60, pool=65536,
                               dist="uniform"),
}


def workload_refs(name: str) -> np.ndarray:
    """The reference set of a named workload."""
    w = WORKLOADS[name]
    return uniform(w["m"], w["d"], w["seed_r"])


def workload(name: str):
    """(R, Q, k) for a named workload."""
    w = WORKLOADS[name]
    if w["dist"] == "uniform":
        R = uniform(w["m"], w["d"], w["seed_r"])
        Q = uniform(w["n"], w["d"], w["seed_q"])
    else:
        R = gaussian_mixture(w["m"], w["d"], w["n_centres"], w["sigma"],
                             w["seed_centres"], w["seed_r"])
        Q = gaussian_mixture(w["n"], w["d"], w["n_centres"], w["sigma"],
                             w["seed_centres"], w["seed_q"])
    return R, Q, w["k"]
