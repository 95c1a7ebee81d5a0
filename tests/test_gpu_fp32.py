"""Parity of the float32 CUDA-core path with the oracle (needs a GB300).

Every case calls the C ABI through the ctypes binding and compares with the
oracle element by element under the rule of tests/parity.py.  Shapes span
several tiles with ragged tails (queries per CTA 64, references per tile 128,
coordinates per stage 16), k = 1 and k = m, duplicates, lattices full of
exact ties (which exercise the float64 re-check and the exact fallback).  The
full n = m = 38400, d = 96 workload, every row, is in
tests/test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_1448_gb300 import knn as mod
    return mod


def run_case(knn, R, Q, k, metric, device_io=True):
    import torch
    idx_ = knn.Index(0, "fp32")
    if device_io:
        idx_.set_reference(torch.from_numpy(R).cuda())
        dist, ind = idx_.search(torch.from_numpy(Q).cuda(), k, metric)
        torch.cuda.synchronize()
        out = dist.cpu().numpy(), ind.cpu().numpy()
    else:
        idx_.set_reference(R)
        out = idx_.search(Q, k, metric)
    st = idx_.stats()
    idx_.close()
    return out[0], out[1], st


def check(knn, R, Q, k, metric, device_io=True):
    m = R.shape[0]
    g_dist, g_idx, st = run_case(knn, R, Q, k, metric, device_io)
    ko = parity.oracle_k(k, m)
    o_dist, o_idx = oracle.knn(R, Q, ko, metric)
    rows, exact = parity.compare(g_dist, g_idx, o_dist, o_idx, k, m)
    return rows, exact, st


@pytest.mark.parametrize("metric", ["l2", "l1", "linf"])
def test_uniform_n1200_d8_k20(knn, metric):
    R, Q, k = inputs.workload("uniform_n1200_d8_k20")
    rows, exact, _ = check(knn, R, Q, k, metric)
    assert rows == 1200


@pytest.mark.parametrize("metric", ["l2", "l1", "linf"])
@pytest.mark.parametrize("n,m,d,k", [
    (1, 1, 1, 1),            # single point
    (7, 300, 3, 5),          # n below one query tile
    (130, 1000, 33, 20),     # ragged in every dimension
    (257, 129, 16, 129),     # k = m, m one past a tile
    (65, 4099, 7, 1),        # k = 1, many splits
    (100, 2000, 96, 64),
    (50, 700, 200, 100),     # d over several stages, large k
    (300, 1500, 64, 10),     # small-set select, selection in registers (48 per lane)
    (40, 3000, 37, 30),      # small-set select, radix selection, rows not whole float4s
])
def test_ragged_shapes(knn, metric, n, m, d, k):
    R = inputs.uniform(m, d, seed=1000 + m)
    Q = inputs.uniform(n, d, seed=2000 + n)
    check(knn, R, Q, k, metric)


def test_host_and_device_io_agree(knn):
    R = inputs.uniform(3000, 24, seed=5)
    Q = inputs.uniform(333, 24, seed=6)
    d1, i1, _ = run_case(knn, R, Q, 17, "l2", device_io=True)
    d2, i2, _ = run_case(knn, R, Q, 17, "l2", device_io=False)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(d1, d2)


def test_queries_drawn_from_reference(knn):
    R = inputs.uniform(5000, 12, seed=15)
    Q = R[::37].copy()
    for metric in ("l2", "l1", "linf"):
        g_dist, g_idx, _ = run_case(knn, R, Q, 10, metric)
        assert np.all(g_dist[:, 0] == 0.0)
        np.testing.assert_array_equal(g_idx[:, 0], np.arange(0, 5000, 37))
        check(knn, R, Q, 10, metric)


def test_lattice_ties(knn):
    """Integer lattice: distances tie in large groups; indices must follow
    the smaller-index rule exactly."""
    R = inputs.lattice(9, 3)            # 729 points
    Q = inputs.lattice(9, 3)[::5] + np.float32(0.5) * (np.arange(3) == 0)
    for metric in ("l2", "l1", "linf"):
        for k in (1, 6, 27, 100):
            m = R.shape[0]
            g_dist, g_idx, _ = run_case(knn, R, Q, k, metric)
            o_dist, o_idx = oracle.knn(R, Q, k, metric)
            np.testing.assert_array_equal(g_idx, o_idx)
            np.testing.assert_allclose(g_dist, o_dist, rtol=1e-6, atol=0)


def near_tie_ladder(d, metric, n_q=12, rungs=48, m_far=1500, step=3e-6, seed=123):
    """For every query, `rungs` references on shells around it whose
    distances (squared for l2) step by `step` relative: float32 distances of
    neighbouring rungs are within float32 rounding of one another, while the
    float64 order is fixed (step > the parity rule's tie tolerance), so every
    position must match the oracle.  Far references fill the rest."""
    rng = np.random.default_rng(seed)
    Q = inputs.uniform(n_q, d, seed=seed)
    rows = [inputs.uniform(m_far, d, seed=seed + 1) * np.float32(4.0) + np.float32(3.0)]
    for i in range(n_q):
        u = rng.standard_normal((rungs, d))
        if metric == "l2":
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            s = 0.5 * np.sqrt(1.0 + step * np.arange(rungs))
        elif metric == "l1":
            u /= np.abs(u).sum(axis=1, keepdims=True)
            s = 0.5 * (1.0 + step * np.arange(rungs))
        else:
            u /= np.abs(u).max(axis=1, keepdims=True)
            s = 0.5 * (1.0 + step * np.arange(rungs))
        rows.append((Q[i].astype(np.float64) + s[:, None] * u).astype(np.float32))
    R = np.concatenate(rows)
    perm = np.random.default_rng(seed + 2).permutation(R.shape[0])
    return np.ascontiguousarray(R[perm]), Q


@pytest.mark.parametrize("metric", ["l2", "l1", "linf"])
@pytest.mark.parametrize("d", [96, 33])
def test_near_tie_ladder_exact_order(knn, metric, d):
    """Distances 3e-6 apart: beyond float32's resolution at this d, so the
    float-float re-check (d = 96: eight lanes per entry; d = 33: one lane)
    decides the order, which must be the oracle's at every position."""
    R, Q = near_tie_ladder(d, metric)
    k = 30
    g_dist, g_idx, st = run_case(knn, R, Q, k, metric)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), metric)
    parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])
    assert st["recheck_entries"] > 0


@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_expanded_euclidean_far_from_the_origin(knn, offset):
    """The float32 Euclidean select (m > 4096) ranks lower bounds of the
    expanded distance, with coordinates taken relative to a reference of the
    split: a point cloud translated far from the origin (coordinates near
    1000, spread 1) keeps the bound's slack at the scale of the spread, so no
    query needs the exact fallback, and the result is the oracle's."""
    R = inputs.uniform(6000, 32, seed=881) + np.float32(offset)
    Q = inputs.uniform(300, 32, seed=882) + np.float32(offset)
    k = 20
    g_dist, g_idx, st = run_case(knn, R, Q, k, "l2")
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), "l2")
    parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])
    assert st["fallback_queries"] == 0


def test_all_identical_points_use_exact_fallback(knn):
    R = np.full((2000, 5), 0.125, dtype=np.float32)
    Q = np.array([[0.125] * 5, [0.5] * 5], dtype=np.float32)
    g_dist, g_idx, st = run_case(knn, R, Q, 40, "l2")
    assert g_idx.tolist() == [list(range(40))] * 2
    assert st["fallback_queries"] == 2
    np.testing.assert_allclose(g_dist[1], np.full(40, np.sqrt(5 * 0.375 ** 2)), rtol=1e-7)


def test_identical_points_beyond_the_fallback_candidate_buffer(knn):
    """More equal-distance references (5000) than the fallback's shared-memory
    candidate buffer holds: the float64 selection over all m decides."""
    R = np.full((5000, 3), 0.25, dtype=np.float32)
    Q = np.array([[0.25] * 3, [0.75] * 3], dtype=np.float32)
    for k in (10, 1000):
        g_dist, g_idx, st = run_case(knn, R, Q, k, "l2")
        assert g_idx.tolist() == [list(range(k))] * 2
        assert st["fallback_queries"] == 2
        np.testing.assert_allclose(g_dist[1], np.full(k, np.sqrt(3 * 0.5 ** 2)), rtol=1e-7)


def test_duplicates_across_splits(knn):
    base = inputs.uniform(300, 8, seed=77)
    R = np.concatenate([base] * 20)      # every point 20 times, spread over the range
    Q = base[:40].copy()
    for metric in ("l2", "l1", "linf"):
        rows, exact, st = check(knn, R, Q, 30, metric)
        g_dist, g_idx, _ = run_case(knn, R, Q, 30, metric)
        o_dist, o_idx = oracle.knn(R, Q, 30, metric)
        np.testing.assert_array_equal(g_idx, o_idx)


def test_prefix_property(knn):
    R = inputs.uniform(6000, 20, seed=88)
    Q = inputs.uniform(200, 20, seed=89)
    d_big, i_big, _ = run_case(knn, R, Q, 50, "l2")
    for k in (1, 10, 49):
        d_k, i_k, _ = run_case(knn, R, Q, k, "l2")
        np.testing.assert_array_equal(i_k, i_big[:, :k])
        np.testing.assert_array_equal(d_k, d_big[:, :k])


def test_invalid_arguments(knn):
    import torch
    ix = knn.Index(0, "fp32")
    Q = torch.zeros((4, 3), device="cuda")
    with pytest.raises(knn.KnnError) as e:
        ix.search(Q, 1)
    assert e.value.status == 5            # KNN_ERR_NOREF
    ix.set_reference(torch.rand((10, 3), device="cuda"))
    for bad_k in (0, 11):
        with pytest.raises(knn.KnnError) as e:
            ix.search(Q, bad_k)
        assert e.value.status == 1
    with pytest.raises(knn.KnnError) as e:
        ix.search(torch.zeros((4, 5), device="cuda"), 1)
    assert e.value.status == 1
    d, i = ix.search(torch.zeros((0, 3), device="cuda"), 3)
    assert d.shape == (0, 3)
    ix.close()


def test_workspace_limit_reports_oom(knn):
    import torch
    ix = knn.Index(0, "fp32", workspace_limit=1024)
    ix.set_reference(torch.rand((5000, 16), device="cuda"))
    with pytest.raises(knn.KnnError) as e:
        ix.search(torch.rand((1000, 16), device="cuda"), 10)
    assert e.value.status == 2
    ix.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_many_queries_in_the_fallback_at_once(knn, precision):
    """40000 references at one point and 100 queries: every query goes to
    the exact fallback.  The first half of the scratch slots take their
    queries spread over several CTAs (three key chunks each, the last CTA to
    finish selects); the queries beyond take one CTA each."""
    import torch
    R = np.full((40000, 8), 0.5, dtype=np.float32)
    g = np.random.Generator(np.random.Philox(77))
    Q = g.uniform(0.0, 1.0, size=(100, 8)).astype(np.float32)
    ix = knn.Index(0, precision)
    ix.set_reference(torch.from_numpy(R).cuda())
    dist, idx = ix.search(torch.from_numpy(Q).cuda(), 12, "l2")
    ix.sync()
    st = ix.stats()
    ix.close()
    assert st["fallback_queries"] == 100
    assert idx.cpu().numpy().tolist() == [list(range(12))] * 100
    want = np.sqrt(((Q.astype(np.float64) - 0.5) ** 2).sum(1))
    np.testing.assert_allclose(dist.cpu().numpy(), np.repeat(want[:, None], 12, 1), rtol=1e-6)
