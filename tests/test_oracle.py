"""Pins for the CPU oracle (no GPU).

The oracle restates the brute-force algorithm of Sec. 2.1 (compute every
distance, sort, keep the k smallest).  The paper prints no worked example, so
these tests pin it to things that do not come from the oracle itself:
hand-derived lattice neighbour lists (tests/golden/), exact brute force over
all orderings on tiny dyadic inputs, an independent library computation
(scipy distances + numpy lexsort), closed forms and invariants.  The last test
builds deliberately broken oracles and checks that these pins catch each one.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_neighbours.txt")


def read_golden():
    cases, cur = [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, *rest = line.split()
            if head == "case":
                cur = {"name": rest[0]}
                cases.append(cur)
            elif head in ("side", "dim"):
                cur[head] = int(rest[0])
            elif head == "metric":
                cur[head] = rest[0]
            elif head in ("query", "keys"):
                cur[head] = [float(x) for x in rest]
            elif head == "idx":
                cur[head] = [int(x) for x in rest]
    return cases


# --------------------------------------------------------------------------
# 1. hand-derived lattice cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", read_golden(), ids=lambda c: c["name"])
def test_golden_lattice(case, lib=0):
    check_golden(case, mutant=0)


def check_golden(case, mutant=0):
    R = inputs.lattice(case["side"], case["dim"])
    Q = np.array([case["query"]], dtype=np.float32)
    m = R.shape[0]
    assert len(case["idx"]) == m
    dist, idx = oracle.knn(R, Q, m, case["metric"], mutant=mutant)
    keys = np.array(case["keys"])
    want = np.sqrt(keys) if case["metric"] == "l2" else keys
    assert idx[0].tolist() == case["idx"]
    np.testing.assert_array_equal(dist[0], want)
    # every prefix (k < m) is the same list cut short
    for k in (1, 2, 5, m - 1):
        dk, ik = oracle.knn(R, Q, k, case["metric"], mutant=mutant)
        assert ik[0].tolist() == case["idx"][:k]


# --------------------------------------------------------------------------
# 2. exact brute force over all orderings on tiny dyadic inputs
# --------------------------------------------------------------------------
def exact_key(q, r, metric):
    diffs = [Fraction(float(a)) - Fraction(float(b)) for a, b in zip(q, r)]
    if metric == "l2":
        return sum(x * x for x in diffs)
    if metric == "l1":
        return sum(abs(x) for x in diffs)
    return max(abs(x) for x in diffs)


def brute_force_order(q, R, metric):
    """The lexicographically smallest sequence of (key, index) over all m!
    orderings of the references -- i.e. the sorted list, found without
    sorting."""
    keys = [exact_key(q, r, metric) for r in R]
    best = None
    for perm in itertools.permutations(range(len(R))):
        seq = [(keys[j], j) for j in perm]
        if best is None or seq < best:
            best = seq
    return best


def tiny_cases(seed, count):
    g = np.random.default_rng(seed)
    for _ in range(count):
        m = int(g.integers(1, 7))
        d = int(g.integers(1, 4))
        # multiples of 1/4 in [-1, 1]: exact in float32 and double, many ties
        R = (g.integers(-4, 5, size=(m, d)) / 4.0).astype(np.float32)
        Q = (g.integers(-4, 5, size=(2, d)) / 4.0).astype(np.float32)
        yield R, Q


@pytest.mark.parametrize("metric", ["l2", "l1", "linf"])
def test_brute_force_permutations(metric):
    check_brute_force(metric, mutant=0)


def check_brute_force(metric, mutant=0, seed=11, count=25):
    for R, Q in tiny_cases(seed, count):
        m = R.shape[0]
        dist, idx = oracle.knn(R, Q, m, metric, mutant=mutant)
        for i in range(Q.shape[0]):
            best = brute_force_order(Q[i], R, metric)
            assert idx[i].tolist() == [j for _, j in best]
            want = [math.sqrt(float(kv)) if metric == "l2" else float(kv) for kv, _ in best]
            np.testing.assert_array_equal(dist[i], np.array(want))


# --------------------------------------------------------------------------
# 3. independent library computation (scipy.spatial distances + lexsort)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("metric,name", [("l2", "euclidean"), ("l1", "cityblock"),
                                         ("linf", "chebyshev")])
def test_matches_scipy_full_sort(metric, name):
    check_scipy(metric, name, mutant=0)


def check_scipy(metric, name, mutant=0):
    from scipy.spatial.distance import cdist
    R = inputs.uniform(300, 7, seed=21)
    Q = inputs.uniform(40, 7, seed=22)
    m = R.shape[0]
    dist, idx = oracle.knn(R, Q, m, metric, mutant=mutant)
    D = cdist(Q.astype(np.float64), R.astype(np.float64), name)
    for i in range(Q.shape[0]):
        order = np.lexsort((np.arange(m), D[i]))
        assert idx[i].tolist() == order.tolist()
        np.testing.assert_allclose(dist[i], D[i][order], rtol=1e-13, atol=0)


# --------------------------------------------------------------------------
# 4. invariants and special cases
# --------------------------------------------------------------------------
def test_self_neighbour_is_zero_with_smallest_duplicate():
    R = inputs.uniform(200, 5, seed=31)
    R[150] = R[40]          # a duplicate: index 40 must win the tie
    Q = R[[40, 150, 7]].copy()
    for metric in ("l2", "l1", "linf"):
        dist, idx = oracle.knn(R, Q, 3, metric)
        assert dist[:, 0].tolist() == [0.0, 0.0, 0.0]
        assert idx[0, :2].tolist() == [40, 150]
        assert idx[1, :2].tolist() == [40, 150]
        assert idx[2, 0] == 7


def test_permutation_invariance():
    R = inputs.uniform(500, 12, seed=41)
    Q = inputs.uniform(30, 12, seed=42)
    perm = np.random.default_rng(43).permutation(500)
    for metric in ("l2", "l1"):
        d0, i0 = oracle.knn(R, Q, 25, metric)
        d1, i1 = oracle.knn(R[perm], Q, 25, metric)
        np.testing.assert_array_equal(d0, d1)
        np.testing.assert_array_equal(i0, perm[i1])


def test_non_decreasing_and_prefix():
    R = inputs.uniform(800, 16, seed=51)
    Q = inputs.uniform(50, 16, seed=52)
    d_big, i_big = oracle.knn(R, Q, 60, "l2")
    assert np.all(np.diff(d_big, axis=1) >= 0)
    for k in (1, 7, 20, 59):
        d_k, i_k = oracle.knn(R, Q, k, "l2")
        np.testing.assert_array_equal(i_k, i_big[:, :k])
        np.testing.assert_array_equal(d_k, d_big[:, :k])


def test_scaling_by_two_is_exact():
    R = inputs.uniform(300, 9, seed=61)
    Q = inputs.uniform(20, 9, seed=62)
    for metric in ("l2", "l1", "linf"):
        d1, i1 = oracle.knn(R, Q, 15, metric)
        d2, i2 = oracle.knn(2 * R, 2 * Q, 15, metric)
        np.testing.assert_array_equal(i1, i2)
        np.testing.assert_array_equal(2 * d1, d2)


def test_one_dimension_is_sorting_abs_difference():
    R = inputs.uniform(257, 1, seed=71)
    Q = inputs.uniform(9, 1, seed=72)
    for metric in ("l2", "l1", "linf"):
        dist, idx = oracle.knn(R, Q, 257, metric)
        for i in range(9):
            a = np.abs(Q[i, 0].astype(np.float64) - R[:, 0].astype(np.float64))
            order = np.lexsort((np.arange(257), a))
            assert idx[i].tolist() == order.tolist()
            np.testing.assert_array_equal(dist[i], a[order])


def test_norm_inequalities():
    d = 10
    R = inputs.uniform(400, d, seed=81)
    Q = inputs.uniform(10, d, seed=82)
    m = R.shape[0]
    out = {}
    for metric in ("l2", "l1", "linf"):
        dist, idx = oracle.knn(R, Q, m, metric)
        full = np.empty_like(dist)
        np.put_along_axis(full, idx.astype(np.int64), dist, axis=1)
        out[metric] = full
    tol = 1e-12
    assert np.all(out["l2"] <= out["l1"] * (1 + tol))
    assert np.all(out["l1"] <= math.sqrt(d) * out["l2"] * (1 + tol))
    assert np.all(out["linf"] <= out["l2"] * (1 + tol))
    assert np.all(out["l2"] <= math.sqrt(d) * out["linf"] * (1 + tol))


def test_all_identical_points():
    R = np.full((50, 4), 0.25, dtype=np.float32)
    Q = np.array([[0.25] * 4, [1.0] * 4], dtype=np.float32)
    dist, idx = oracle.knn(R, Q, 10, "l2")
    assert idx.tolist() == [list(range(10))] * 2
    assert dist[0].tolist() == [0.0] * 10
    np.testing.assert_array_equal(dist[1], np.full(10, 1.5))   # sqrt(4 * 0.75^2)


def test_single_reference():
    R = np.array([[3.0, 4.0]], dtype=np.float32)
    Q = np.array([[0.0, 0.0]], dtype=np.float32)
    dist, idx = oracle.knn(R, Q, 1, "l2")
    assert idx.tolist() == [[0]] and dist.tolist() == [[5.0]]
    dist, idx = oracle.knn(R, Q, 1, "l1")
    assert dist.tolist() == [[7.0]]


def test_invalid_arguments_are_rejected():
    R = inputs.uniform(5, 3, seed=1)
    Q = inputs.uniform(2, 3, seed=2)
    with pytest.raises(ValueError):
        oracle.knn(R, Q, 6, "l2")     # k > m
    with pytest.raises(ValueError):
        oracle.knn(R, Q, 0, "l2")     # k < 1
    with pytest.raises(ValueError):
        oracle.knn(R, inputs.uniform(2, 4, seed=2), 1, "l2")


def test_subset_and_pairs_agree_with_full():
    R = inputs.uniform(300, 6, seed=91)
    Q = inputs.uniform(40, 6, seed=92)
    d, i = oracle.knn(R, Q, 8, "l2")
    sel = np.array([39, 0, 17])
    ds, is_ = oracle.knn_subset(R, Q, sel, 8, "l2")
    np.testing.assert_array_equal(ds, d[sel])
    np.testing.assert_array_equal(is_, i[sel])
    keys = oracle.key_pairs(R, Q, np.repeat(sel, 8), is_.reshape(-1), "l2")
    np.testing.assert_array_equal(np.sqrt(keys), ds.reshape(-1))


def test_thread_count_is_per_call():
    # the result does not depend on the thread count, and a call's count does
    # not stay behind for the next one (the single-core timing runs between
    # all-core ones)
    R = inputs.uniform(500, 5, seed=93)
    Q = inputs.uniform(64, 5, seed=94)
    before = oracle.max_threads()
    d1, i1 = oracle.knn(R, Q, 10, "l1", nthreads=1)
    assert oracle.max_threads() == before
    d3, i3 = oracle.knn(R, Q, 10, "l1", nthreads=3)
    np.testing.assert_array_equal(d1, d3)
    np.testing.assert_array_equal(i1, i3)
    M = np.eye(5)
    oracle.knn_mahalanobis(R, Q, M, 4, nthreads=1)
    assert oracle.max_threads() == before


# --------------------------------------------------------------------------
# 5. the pins catch planted mistakes
# --------------------------------------------------------------------------
def pins_pass(mutant):
    try:
        for case in read_golden():
            check_golden(case, mutant=mutant)
        for metric in ("l2", "l1", "linf"):
            check_brute_force(metric, mutant=mutant, count=10)
        check_scipy("l2", "euclidean", mutant=mutant)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutant", [1, 2, 3, 4],
                         ids=["dropped_term", "wrong_sign", "reversed_tiebreak",
                              "swapped_operands"])
def test_pins_catch_planted_mistakes(mutant):
    assert pins_pass(0)
    assert not pins_pass(mutant), f"mutant {mutant} slipped through the pins"
