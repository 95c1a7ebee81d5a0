"""The seeded input recipes (paper_0804_1448_gb300/inputs.py): deterministic
per seed, the stated distributions and shapes.  No GPU."""
import numpy as np

from paper_0804_1448_gb300 import inputs


def test_uniform_is_deterministic_and_in_the_unit_cube():
    a = inputs.uniform(500, 7, seed=11)
    b = inputs.uniform(500, 7, seed=11)
    c = inputs.uniform(500, 7, seed=12)
    assert a.dtype == np.float32 and a.shape == (500, 7) and a.flags["C_CONTIGUOUS"]
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(float(a.mean()) - 0.5) < 0.02


def test_mixture_points_sit_near_their_centres():
    sigma, d = 0.05, 16
    X = inputs.gaussian_mixture(4000, d, 32, sigma, seed_centres=5, seed_points=6)
    centres = inputs.rng(5).random((32, d), dtype=np.float32)
    dist = np.sqrt(((X[:, None, :] - centres[None, :, :]) ** 2).sum(-1)).min(1)
    # the nearest centre is the own one at sigma*sqrt(d) on average
    assert abs(float(np.median(dist)) - sigma * np.sqrt(d)) < 0.25 * sigma * np.sqrt(d)
    # another point seed draws from the same centres
    Y = inputs.gaussian_mixture(1000, d, 32, sigma, seed_centres=5, seed_points=7)
    dist_y = np.sqrt(((Y[:, None, :] - centres[None, :, :]) ** 2).sum(-1)).min(1)
    assert float(np.median(dist_y)) < 2 * sigma * np.sqrt(d)


def test_lattice_indexing():
    L = inputs.lattice(5, 2)
    assert L.shape == (25, 2)
    assert L[5 * 3 + 4].tolist() == [3.0, 4.0]        # (x0, x1) -> x0 * side + x1


def test_named_workloads():
    R, Q, k = inputs.workload("uniform_n1200_d8_k20")
    assert R.shape == (1200, 8) and Q.shape == (1200, 8) and k == 20
    assert not np.array_equal(R, Q)
    w = inputs.WORKLOADS["uniform_n38400_d96_k20"]
    assert (w["m"], w["n"], w["d"], w["k"]) == (38400, 38400, 96, 20)
    w = inputs.WORKLOADS["mixture_m1048576_n16384_d128_k100"]
    assert (w["m"], w["n"], w["d"], w["k"], w["n_centres"], w["sigma"]) == \
        (1048576, 16384, 128, 100, 1024, 0.05)
    assert inputs.WORKLOADS["serve_m4194304_d96"]["m"] == 4194304
