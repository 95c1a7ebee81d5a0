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
    """Assert-style check of all rows; returns (n_rows, n_exact_index_rows)."""
    g_dist = np.asarray(g_dist)
    g_idx = np.asarray(g_idx)
    errors = []
    exact = 0
    for i in range(g_idx.shape[0]):
        msg = check_row(g_dist[i], g_idx[i], o_dist[i], o_idx[i], k, m)
        if msg:
            errors.append(f"row {i}: {msg}")
            if len(errors) >= max_report:
                break
        if np.array_equal(g_idx[i, :k], o_idx[i, :k]):
            exact += 1
    assert not errors, "\n".join(errors)
    return g_idx.shape[0], exact


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
    tot = 0.0
    for a, b in zip(np.asarray(g_idx)[:, :k], np.asarray(o_idx)[:, :k]):
        tot += len(set(a.tolist()) & set(b.tolist())) / k
    return tot / len(g_idx)
