"""The Sec. 2.2 applications' host arithmetic (paper_0804_1448_gb300/apps.py)
against closed forms, on neighbour distances from the oracle.  No GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import apps, inputs


def oracle_self_rho(R, k):
    """rho_k(y_i): distance to the k-th nearest OTHER point (oracle)."""
    dist, idx = oracle.knn(R, R, k + 1, "l2")
    out = np.empty(R.shape[0])
    for i in range(R.shape[0]):
        keep = [s for s in range(k + 1) if idx[i, s] != i][:k]
        out[i] = dist[i, keep[k - 1]]
    return out


def test_digamma_at_integers():
    g = apps.EULER_GAMMA
    assert apps.digamma_int(1) == pytest.approx(-g, abs=1e-15)
    assert apps.digamma_int(2) == pytest.approx(1 - g, abs=1e-15)
    assert apps.digamma_int(5) == pytest.approx(25 / 12 - g, abs=1e-14)
    special = pytest.importorskip("scipy.special")
    for k in range(1, 60):
        assert apps.digamma_int(k) == pytest.approx(float(special.digamma(k)), abs=1e-12)


def test_unit_ball_volumes():
    assert math.exp(apps.log_unit_ball(1)) == pytest.approx(2.0)
    assert math.exp(apps.log_unit_ball(2)) == pytest.approx(math.pi)
    assert math.exp(apps.log_unit_ball(3)) == pytest.approx(4 * math.pi / 3)
    assert math.exp(apps.log_unit_ball(4)) == pytest.approx(math.pi ** 2 / 2)


def test_entropy_of_the_unit_square_is_near_zero():
    R = inputs.uniform(4000, 2, seed=501)
    H = apps.entropy_from_rho(oracle_self_rho(R, 4), 2, 4)
    assert abs(H) < 0.06                     # true entropy 0; edge effects bias it slightly


def test_entropy_of_a_gaussian():
    sigma, d = 0.5, 3
    R = (np.random.Generator(np.random.Philox(502)).standard_normal((4000, d)) * sigma).astype(np.float32)
    H = apps.entropy_from_rho(oracle_self_rho(R, 4), d, 4)
    assert H == pytest.approx(0.5 * d * math.log(2 * math.pi * math.e * sigma ** 2), abs=0.06)


def test_printed_and_goria_forms_agree_in_one_dimension():
    R = inputs.uniform(2000, 1, seed=503)
    rho = oracle_self_rho(R, 3)
    assert apps.entropy_from_rho(rho, 1, 3, "printed") == pytest.approx(
        apps.entropy_from_rho(rho, 1, 3, "goria"), abs=1e-12)


def test_majority_vote():
    labels = np.array([[3, 1, 3, 2, 1], [7, 7, 7, 0, 0], [5, 4, 4, 5, 9]])
    np.testing.assert_array_equal(apps.majority_vote(labels), [1, 7, 4])   # ties -> smaller
