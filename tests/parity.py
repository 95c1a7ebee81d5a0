"""Comparison of a k-nearest-neighbour result with the oracle's (test helper).

The rule:
  * indices must equal the oracle's exactly, except inside runs of near-equal
    oracle distances (consecutive distances within REL_TIE relative of each
    other): inside such a run any order is accepted, and where a run crosses
    the k-th position any of its members may fill the remaining slots;
  * every returned distance must be within REL_DIST relative of the oracle's
    distance at the same position;
  * returned indices must be distinct within a row.
"""
from __future__ import annotations

import numpy as np

REL_TIE = 1e-6
REL_DIST = 1e-5


def runs(dist_row: np.ndarray, rel: float = REL_TIE):
    """[(a, b)] inclusive index ranges of near-tie runs of a sorted row."""
    out, a = [], 0
    for p in range(1, len(dist_row) + 1):
        if p == len(dist_row) or dist_row[p] - dist_row[p - 1] > rel * max(dist_row[p], 1e-300):
            out.append((a, p - 1))
            a = p
    return out


def check_row(g_dist, g_idx, o_dist, o_idx, k, m):
    """Return None if row passes, else a message.  o_* hold the oracle's first
    K >= k entries (K > k whenever k < m so a boundary run is visible)."""
    g_idx = [int(x) for x in g_idx[:k]]
    if len(set(g_idx)) != k:
        return f"duplicate indices {g_idx}"
    if any(j < 0 or j >= m for j in g_idx):
        return f"index out of range {g_idx}"
    for a, b in runs(o_dist):
        if a >= k:
            break
        end = min(b + 1, k)
        got = set(g_idx[a:end])
        # a run that reaches the end of the oracle's K entries allows only the
        # members shown (oracle_k asks for 32 spare entries)
        allowed = set(int(x) for x in o_idx[a:b + 1])
        if not got <= allowed:
            return (f"positions {a}..{end - 1}: got {sorted(got)} not within oracle run "
                    f"{sorted(allowed)}")
    err = np.abs(np.asarray(g_dist[:k], np.float64) - o_dist[:k])
    tol = REL_DIST * np.abs(o_dist[:k])
    bad = np.nonzero(err > tol)[0]
    if len(bad):
        p = int(bad[0])
        return f"distance at {p}: got {g_dist[p]!r} oracle {o_dist[p]!r}"
    return None


def compare(g_dist, g_idx, o_dist, o_idx, k, m, max_report=5):
    """Assert-style check of all rows; returns (n_rows, n_exact_index_rows).

    Rows whose k indices equal the oracle's first k, in order, and whose
    distances are all within REL_DIST pass check_row by construction (every
    run then holds exactly the oracle's members, the oracle's indices are
    distinct and in range); they are accepted in one vectorised pass and only
    the other rows go through check_row."""
    g_dist = np.asarray(g_dist)
    g_idx = np.asarray(g_idx)
    o_dist = np.asarray(o_dist)
    o_idx = np.asarray(o_idx)
    n = g_idx.shape[0]
    if n == 0:
        return 0, 0
    same = np.all(g_idx[:, :k] == o_idx[:, :k], axis=1)
    err = np.abs(np.asarray(g_dist[:, :k], np.float64) - o_dist[:, :k])
    close = np.all(err <= REL_DIST * np.abs(o_dist[:, :k]), axis=1)
    errors = []
    for i in np.nonzero(~(same & close))[0]:
        msg = check_row(g_dist[i], g_idx[i], o_dist[i], o_idx[i], k, m)
        if msg:
            errors.append(f"row {int(i)}: {msg}")
            if len(errors) >= max_report:
                break
    assert not errors, "\n".join(errors)
    return n, int(np.count_nonzero(same))


def oracle_k(k: int, m: int) -> int:
    """How many oracle entries to request so boundary runs are visible."""
    return min(m, k + 32)


def max_rel_err(g_dist, o_dist, k):
    g = np.asarray(g_dist[:, :k], np.float64)
    o = o_dist[:, :k]
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(o > 0, np.abs(g - o) / o, np.abs(g - o))
    return float(np.max(r)) if r.size else 0.0


def recall(g_idx, o_idx, k):
    """Mean fraction of the oracle's k indices present in the returned k."""
    g = np.sort(np.asarray(g_idx)[:, :k].astype(np.int64), axis=1)
    o = np.sort(np.asarray(o_idx)[:, :k].astype(np.int64), axis=1)
    if g.shape[0] == 0:
        return 1.0
    # a repeated returned index counts once: repeats become negative values
    # no oracle index can equal
    rep = np.zeros_like(g, dtype=bool)
    rep[:, 1:] = g[:, 1:] == g[:, :-1]
    g = np.where(rep, -1 - np.arange(k, dtype=np.int64)[None, :], g)
    # count the common members of each pair of rows by merging them (rows
    # offset so that values of different rows never meet)
    off = (np.arange(g.shape[0], dtype=np.int64) * (2 ** 33))[:, None]
    both = np.concatenate([g + off, o + off], axis=1).ravel()
    both.sort()
    common = np.count_nonzero(both[1:] == both[:-1])
    return common / (k * g.shape[0])


# (workload, form) -> (rows checked, recall@k, max relative distance error),
# filled by the GPU tests and printed at the end of the run by conftest.py
SUMMARY: dict[str, tuple[int, float, float]] = {}


def record(name, g_dist, g_idx, o_dist, o_idx, k):
    """Store the recall and the largest relative distance error of a checked
    result under `name`, for the end-of-run summary, and return them."""
    rec = recall(g_idx, o_idx, k)
    err = max_rel_err(np.asarray(g_dist), np.asarray(o_dist), k)
    SUMMARY[name] = (int(np.asarray(g_idx).shape[0]), rec, err)
    return rec, err
