"""Pins of the Mahalanobis oracle (oracle.knn_mahalanobis): the quadratic form
of Sec. 2.1's Mahalanobis distance checked against things outside itself --
hand-derived lattice lists, the Euclidean oracle (M = I), a weighted sum
written out (diagonal M), the Euclidean distance of transformed points
(M = A^T A) and scaling.  A planted mistake (off-diagonal terms dropped) must
fail at least one pin.  No GPU."""
import os

import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mahalanobis_lattice.txt")


def golden_cases():
    cases, cur = [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            word, *rest = line.split()
            if word == "case":
                cur = {"name": rest[0]}
                cases.append(cur)
            elif word == "matrix":
                cur["M"] = np.array([float(x) for x in rest]).reshape(2, 2)
            elif word == "keys":
                cur["keys"] = np.array([float(x) for x in rest])
            elif word == "idx":
                cur["idx"] = np.array([int(x) for x in rest])
    return cases


def lattice():
    return np.array([[x, y] for x in range(5) for y in range(5)], dtype=np.float32)


def spd(d, seed):
    g = np.random.Generator(np.random.Philox(seed))
    A = g.standard_normal((d, d))
    return A, A.T @ A + 0.1 * np.eye(d)


def hand_pins_pass(mutant=0):
    R = lattice()
    q = np.array([[2, 2]], dtype=np.float32)
    for c in golden_cases():
        dist, idx = oracle.knn_mahalanobis(R, q, c["M"], 25, mutant=mutant)
        if not (np.array_equal(idx[0], c["idx"]) and np.allclose(dist[0] ** 2, c["keys"], rtol=1e-12)):
            return False
    return True


def transformed_pin_passes(mutant=0):
    d = 6
    A, _ = spd(d, 11)
    R = inputs.uniform(300, d, seed=12)
    Q = inputs.uniform(7, d, seed=13)
    dist, idx = oracle.knn_mahalanobis(R, Q, A.T @ A, 10, mutant=mutant)
    Rt = R.astype(np.float64) @ A.T
    Qt = Q.astype(np.float64) @ A.T
    full = np.sqrt(((Qt[:, None, :] - Rt[None, :, :]) ** 2).sum(-1))
    ref_idx = np.argsort(full, axis=1, kind="stable")[:, :10]
    ref = np.take_along_axis(full, ref_idx, axis=1)
    return np.array_equal(idx, ref_idx) and np.allclose(dist, ref, rtol=1e-10)


@pytest.mark.parametrize("case", [c["name"] for c in golden_cases()])
def test_hand_derived_lattices(case):
    c = next(x for x in golden_cases() if x["name"] == case)
    dist, idx = oracle.knn_mahalanobis(lattice(), np.array([[2, 2]], dtype=np.float32), c["M"], 25)
    np.testing.assert_array_equal(idx[0], c["idx"])
    np.testing.assert_allclose(dist[0] ** 2, c["keys"], rtol=1e-12)


def test_identity_matrix_is_the_euclidean_oracle():
    R = inputs.uniform(400, 9, seed=21)
    Q = inputs.uniform(13, 9, seed=22)
    d1, i1 = oracle.knn(R, Q, 20, "l2")
    d2, i2 = oracle.knn_mahalanobis(R, Q, np.eye(9), 20)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(d1, d2)        # same arithmetic: bit-identical


def test_diagonal_matrix_is_a_weighted_sum():
    R = inputs.uniform(300, 5, seed=23)
    Q = inputs.uniform(4, 5, seed=24)
    w = np.array([0.5, 2.0, 1.0, 3.0, 0.25])
    dist, idx = oracle.knn_mahalanobis(R, Q, np.diag(w), 300)
    diff = Q.astype(np.float64)[:, None, :] - R.astype(np.float64)[None, :, :]
    full = np.sqrt((w * diff ** 2).sum(-1))
    np.testing.assert_allclose(dist, np.take_along_axis(full, idx, axis=1), rtol=1e-13)
    assert np.all(np.diff(dist, axis=1) >= 0)


def test_gram_matrix_equals_euclidean_of_transformed_points():
    assert transformed_pin_passes()


def test_scaling_the_matrix_by_four_doubles_the_distances():
    R = inputs.uniform(200, 4, seed=25)
    Q = inputs.uniform(5, 4, seed=26)
    _, M = spd(4, 27)
    d1, i1 = oracle.knn_mahalanobis(R, Q, M, 15)
    d2, i2 = oracle.knn_mahalanobis(R, Q, 4.0 * M, 15)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(d2, 2.0 * d1)


def test_pins_catch_the_dropped_off_diagonal_mutant():
    assert hand_pins_pass(0) and transformed_pin_passes(0)
    assert not (hand_pins_pass(5) and transformed_pin_passes(5)), "mutant 5 slipped through"
