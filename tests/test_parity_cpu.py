"""The parity rule every GPU test applies (tests/parity.py), checked on the
CPU against results built from the oracle: what it must accept (the oracle
itself, reorderings inside near-tie runs, another member of a run that crosses
the k-th position, distances within tolerance) and what it must reject."""
import numpy as np
import pytest

import oracle
import parity
from paper_0804_1448_gb300 import inputs


def case(k=10, m=400, d=6, seed=11):
    R = inputs.uniform(m, d, seed=seed)
    Q = inputs.uniform(4, d, seed=seed + 1)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, m), "l2")
    return o_dist, o_idx, k, m


def row_ok(g_dist, g_idx, o_dist, o_idx, k, m):
    return parity.check_row(g_dist, g_idx, o_dist, o_idx, k, m) is None


def test_runs_groups_near_equal_neighbours():
    row = np.array([1.0, 1.0 + 5e-7, 1.0 + 9e-7, 2.0, 3.0, 3.0])
    assert parity.runs(row) == [(0, 2), (3, 3), (4, 5)]
    assert parity.runs(np.array([0.0, 0.0, 1.0])) == [(0, 1), (2, 2)]


def test_accepts_the_oracle_itself():
    o_dist, o_idx, k, m = case()
    rows, exact = parity.compare(o_dist[:, :k].astype(np.float32), o_idx[:, :k], o_dist, o_idx, k, m)
    assert rows == exact == o_idx.shape[0]


def test_accepts_reordering_inside_a_run_and_boundary_members():
    o_dist = np.array([0.5, 1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 3.0])
    o_idx = np.array([7, 3, 1, 9, 4, 8, 2, 6])
    m, k = 50, 5
    assert row_ok(o_dist[:k], [7, 9, 3, 1, 4], o_dist, o_idx, k, m)      # run 1..3 reordered
    assert row_ok(o_dist[:k], [7, 3, 1, 9, 2], o_dist, o_idx, k, m)      # run 4..6 crosses k
    assert row_ok(o_dist[:k], [7, 3, 1, 9, 8], o_dist, o_idx, k, m)


@pytest.mark.parametrize("mutate", ["wrong_member", "swap_across_runs", "duplicate", "out_of_range",
                                    "distance_off", "outside_boundary_run"])
def test_rejects_planted_mistakes(mutate):
    o_dist = np.array([0.5, 1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 3.0])
    o_idx = np.array([7, 3, 1, 9, 4, 8, 2, 6])
    m, k = 50, 5
    g_dist = o_dist[:k].astype(np.float32).copy()
    g_idx = list(o_idx[:k])
    if mutate == "wrong_member":
        g_idx[1] = 11                       # not a reference of this run
    elif mutate == "swap_across_runs":
        g_idx[0], g_idx[1] = g_idx[1], g_idx[0]
    elif mutate == "duplicate":
        g_idx[4] = g_idx[3]
    elif mutate == "out_of_range":
        g_idx[4] = m
    elif mutate == "distance_off":
        g_dist[2] *= 1 + 3e-5
    elif mutate == "outside_boundary_run":
        g_idx[4] = 6                        # the next run's member at the k-th slot
    assert not row_ok(g_dist, g_idx, o_dist, o_idx, k, m)


def test_distance_tolerance_is_relative():
    o_dist, o_idx, k, m = case(seed=21)
    g = o_dist[:, :k].astype(np.float64) * (1 + 0.5 * parity.REL_DIST)
    parity.compare(g, o_idx[:, :k], o_dist, o_idx, k, m)
    with pytest.raises(AssertionError):
        parity.compare(o_dist[:, :k] * (1 + 2 * parity.REL_DIST), o_idx[:, :k], o_dist, o_idx, k, m)


def test_oracle_k_leaves_room_for_boundary_runs():
    assert parity.oracle_k(20, 38400) == 52
    assert parity.oracle_k(20, 30) == 30


def test_recall_and_max_relative_error():
    o_dist, o_idx, k, m = case(seed=31)
    assert parity.recall(o_idx[:, :k], o_idx, k) == 1.0
    g = o_idx[:, :k].copy()
    g[0, k - 1] = m - 1 if m - 1 not in o_idx[0, :k] else m - 2   # one wrong neighbour in one row
    assert parity.recall(g, o_idx, k) == pytest.approx(1.0 - 1.0 / (k * g.shape[0]))
    assert parity.max_rel_err(o_dist[:, :k], o_dist, k) == 0.0
    d = o_dist[:, :k].copy()
    d[2, 3] *= 1 + 4e-6
    assert parity.max_rel_err(d, o_dist, k) == pytest.approx(4e-6, rel=1e-6)


def test_recall_matches_the_set_definition():
    """The vectorised recall counts, per row, the returned indices that are
    among the oracle's k (a repeated index once), as a set intersection does."""
    rng = np.random.default_rng(5)
    k, rows = 7, 300
    o = np.stack([rng.choice(60, k, replace=False) for _ in range(rows)])
    g = rng.integers(0, 60, size=(rows, k))            # repeats and misses included
    want = np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(g, o)])
    assert parity.recall(g, o, k) == pytest.approx(want, abs=1e-12)


def test_compare_finds_one_bad_row_among_many():
    """Rows equal to the oracle take the vectorised path; a planted mistake in
    one row out of many is still reported, with its row number."""
    o_dist, o_idx, k, m = case(k=8, m=300, seed=41)
    reps = 500
    od = np.tile(o_dist, (reps, 1))
    oi = np.tile(o_idx, (reps, 1))
    g_dist = od[:, :k].astype(np.float32).copy()
    g_idx = oi[:, :k].copy()
    assert parity.compare(g_dist, g_idx, od, oi, k, m) == (od.shape[0], od.shape[0])
    bad = 1234
    g_idx[bad, 0] = next(j for j in range(m) if j not in set(oi[bad, :k + 2].tolist()))
    with pytest.raises(AssertionError, match=f"row {bad}:"):
        parity.compare(g_dist, g_idx, od, oi, k, m)
