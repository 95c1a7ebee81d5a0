"""Tensor-core form (bf16 / tf32 tcgen05 contraction, float32 re-rank of
rerank_factor*k candidates, float64 near-tie re-check) against the oracle.

The candidates are ranked with low-precision products, so a true neighbour
could in principle fall outside them.  On these workloads it does not: every
case asserts recall@k = 1.0 against the float64 oracle, applies the parity
rule of tests/parity.py to every row, and checks that every returned distance
is the exact distance of the returned reference (float32 re-rank).  The
full-size workloads are in tests/test_gpu_fullsize.py.
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


def run(knn, R, Q, k, precision, rerank=4):
    import torch
    ix = knn.Index(0, precision, rerank_factor=rerank)
    ix.set_reference(torch.from_numpy(R).cuda())
    dist, idx = ix.search(torch.from_numpy(Q).cuda(), k, "l2")
    ix.sync()
    out = dist.cpu().numpy(), idx.cpu().numpy()
    ix.close()
    return out


def check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k, name=None):
    """Recall@k must be 1.0, every row must match the oracle under the parity
    rule, and every returned distance must be that reference's exact distance
    within 1e-5 relative."""
    m = R.shape[0]
    rec = parity.recall(g_idx, o_idx, k)
    if name:
        parity.record(name, g_dist, g_idx, o_dist, o_idx, k)
    assert rec == 1.0, f"recall@{k} = {rec}"
    parity.compare(g_dist, g_idx, o_dist, o_idx, k, m)
    qi = np.repeat(np.arange(Q.shape[0]), k)
    keys = oracle.key_pairs(R, Q, qi, g_idx.reshape(-1), "l2")
    exact = np.sqrt(keys).reshape(g_dist.shape)
    np.testing.assert_allclose(g_dist, exact, rtol=1e-5, atol=0)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("n,m,d,k", [
    (1, 1, 1, 1),
    (7, 300, 3, 5),           # less than one tile of queries and references
    (130, 1000, 33, 20),      # ragged: queries, references and coordinates
    (300, 4099, 96, 10),      # references one past a multiple of 128... plus 3
    (256, 2048, 128, 16),
    (129, 5000, 8, 20),
])
def test_uniform_shapes(knn, precision, n, m, d, k):
    R = inputs.uniform(m, d, seed=3000 + m)
    Q = inputs.uniform(n, d, seed=4000 + n)
    g_dist, g_idx = run(knn, R, Q, k, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, m), "l2")
    check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("n,m,d,k,gsize", [
    (12000, 1000, 40, 10, 16),   # every tile sampled, groups of 16; last tile 232 rows
    (12000, 777, 40, 20, 8),     # groups of 8; last tile 9 rows (a slice of 9 elements)
    (6000, 2400, 96, 20, 16),    # two reference splits, the second short
])
def test_pilot_small_groups(knn, precision, n, m, d, k, gsize):
    """Reference sets too small for pilot groups of 32: every tile is sampled,
    c' = c, and the groups shrink to 16 or 8 references."""
    p = knn.explain_plan(n, m, d, k, precision=precision)
    assert p["tensor_cores"] == 1 and p["pilot"] == 1 and p["pilot_stride"] == 1
    assert p["pilot_group_size"] == gsize and p["threshold_rank"] == p["candidates"]
    R = inputs.uniform(m, d, seed=3100 + m)
    Q = inputs.uniform(n, d, seed=4100 + n)
    g_dist, g_idx = run(knn, R, Q, k, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, m), "l2")
    check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_uniform_n1200_d8_k20(knn, precision):
    R, Q, k = inputs.workload("uniform_n1200_d8_k20")
    g_dist, g_idx = run(knn, R, Q, k, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), "l2")
    check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k,
                   name=f"uniform_n1200_d8_k20 {precision}")


def test_self_neighbours(knn):
    R = inputs.uniform(4000, 40, seed=99)
    Q = R[::13].copy()
    for precision in ("bf16", "tf32"):
        g_dist, g_idx = run(knn, R, Q, 5, precision)
        np.testing.assert_array_equal(g_idx[:, 0], np.arange(0, 4000, 13))
        assert np.all(g_dist[:, 0] == 0.0)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_near_tie_ladder(knn, precision):
    """Shells of references 3e-6 apart in squared distance around every query:
    all of them survive the low-precision filter, and the float32 re-rank plus
    the float-float re-check must reproduce the oracle's order exactly."""
    from tests.test_gpu_fp32 import near_tie_ladder
    R, Q = near_tie_ladder(96, "l2")
    k = 30
    g_dist, g_idx = run(knn, R, Q, k, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), "l2")
    assert parity.recall(g_idx, o_idx, k) == 1.0
    parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])


# ------------------------------------------------------------- edge cases

def run_stats(knn, R, Q, k, precision):
    import torch
    ix = knn.Index(0, precision)
    ix.set_reference(torch.from_numpy(R).cuda())
    dist, idx = ix.search(torch.from_numpy(Q).cuda(), k, "l2")
    ix.sync()
    st = ix.stats()
    ix.close()
    return dist.cpu().numpy(), idx.cpu().numpy(), st


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_all_identical_points(knn, precision):
    """Every reference at the same place: every one passes the filter, the
    lists overflow or the cut cannot choose, and the exact fallback orders
    them by index."""
    R = np.full((3000, 16), 0.5, dtype=np.float32)
    Q = np.array([[0.5] * 16, [0.25] * 16], dtype=np.float32)
    g_dist, g_idx, st = run_stats(knn, R, Q, 10, precision)
    assert g_idx.tolist() == [list(range(10))] * 2
    np.testing.assert_allclose(g_dist[0], 0.0, atol=0)
    np.testing.assert_allclose(g_dist[1], np.sqrt(16 * 0.25 ** 2), rtol=1e-6)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_k_equals_m(knn, precision):
    """k = m: the whole reference set, sorted, for every query."""
    R = inputs.uniform(200, 12, seed=3301)
    Q = inputs.uniform(33, 12, seed=3302)
    g_dist, g_idx, _ = run_stats(knn, R, Q, 200, precision)
    o_dist, o_idx = oracle.knn(R, Q, 200, "l2")
    parity.compare(g_dist, g_idx, o_dist, o_idx, 200, 200)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("m", [1500, 9000])
def test_long_rows(knn, precision, m):
    """d = 300: operand rows of several 128-byte K blocks, one K block per
    stage and the 16-bit-code staging; m = 1500 runs without a pilot (every
    reference appended), m = 9000 with one."""
    R = inputs.uniform(m, 300, seed=3400 + m)
    Q = inputs.uniform(150, 300, seed=3401 + m)
    k = 15
    g_dist, g_idx, st = run_stats(knn, R, Q, k, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, m), "l2")
    check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_one_partial_reference_tile(knn, precision):
    """m = 37 (one tile, mostly empty columns) and n = 1000 (several query
    tiles, ragged)."""
    R = inputs.uniform(37, 20, seed=3501)
    Q = inputs.uniform(1000, 20, seed=3502)
    g_dist, g_idx, _ = run_stats(knn, R, Q, 7, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(7, 37), "l2")
    parity.compare(g_dist, g_idx, o_dist, o_idx, 7, 37)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_duplicated_references(knn, precision):
    """Every reference three times (indices i, i + m0, i + 2 m0): equal
    distances ordered by index, and the three copies of the nearest point come
    first."""
    base = inputs.uniform(3000, 24, seed=3601)
    R = np.concatenate([base, base, base])
    Q = inputs.uniform(64, 24, seed=3602)
    g_dist, g_idx, _ = run_stats(knn, R, Q, 9, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(9, R.shape[0]), "l2")
    assert parity.recall(g_idx, o_idx, 9) == 1.0
    parity.compare(g_dist, g_idx, o_dist, o_idx, 9, R.shape[0])
    assert np.all(g_idx[:, 1] == g_idx[:, 0] + 3000) and np.all(g_idx[:, 2] == g_idx[:, 0] + 6000)


@pytest.mark.parametrize("precision", ["bf16", "tf32", "fp32"])
def test_pinned_host_buffers_equal_device_buffers(knn, precision):
    """Pinned host buffers are read and written by the kernels in place
    (tensor-core forms: the query preparation reads Q over the CPU-GPU link,
    the finalize writes the outputs there); pageable ones are copied.  All
    give the device-buffer result bit for bit."""
    import torch
    R = inputs.uniform(20000, 64, seed=3701)
    Q = inputs.uniform(3000, 64, seed=3702)
    k = 16
    ix = knn.Index(0, precision)
    ix.set_reference(torch.from_numpy(R).cuda())
    d_dev, i_dev = ix.search(torch.from_numpy(Q).cuda(), k, "l2")
    ix.sync()
    Qh = torch.from_numpy(Q).pin_memory()
    dh = torch.empty((3000, k), dtype=torch.float32).pin_memory()
    ih = torch.empty((3000, k), dtype=torch.int32).pin_memory()
    ix.search_into(Qh, k, dh, ih, "l2")            # synchronous for host buffers
    assert torch.equal(dh, d_dev.cpu()) and torch.equal(ih, i_dev.cpu())
    d_pg, i_pg = ix.search(Q, k, "l2")             # pageable numpy arrays: copies
    np.testing.assert_array_equal(d_pg, d_dev.cpu().numpy())
    np.testing.assert_array_equal(i_pg, i_dev.cpu().numpy())
    ix.close()


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("n", [12_001, 20_001])   # ragged second halves
def test_pinned_host_search_in_parts(knn, precision, n):
    """From 8192 queries on, a search whose queries and outputs are in pinned
    host memory runs in two parts, each on its own stream, the second part's
    queries crossing the link while the first part computes.  Its result is the device-buffer search's, bit for bit,
    and the oracle's under the parity rule."""
    import torch
    m, d, k = 5_000, 64, 16
    R = inputs.uniform(m, d, seed=3711)
    Q = inputs.uniform(n, d, seed=3712)
    ix = knn.Index(0, precision)
    ix.set_reference(torch.from_numpy(R).cuda())
    d_dev, i_dev = ix.search(torch.from_numpy(Q).cuda(), k, "l2")
    ix.sync()
    Qh = torch.from_numpy(Q).pin_memory()
    dh = torch.empty((n, k), dtype=torch.float32).pin_memory()
    ih = torch.empty((n, k), dtype=torch.int32).pin_memory()
    for _ in range(2):   # the second call reuses the side stream and the workspace
        dh.fill_(-1.0)
        ih.fill_(-1)
        ix.search_into(Qh, k, dh, ih, "l2")
        assert torch.equal(dh, d_dev.cpu()) and torch.equal(ih, i_dev.cpu())
    ix.close()
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, m), "l2")
    check_all_rows(R, Q, dh.numpy(), ih.numpy(), o_dist, o_idx, k)


# ------------------------------------------------- serving k range, large pools

@pytest.fixture(scope="module")
def serving_range():
    """A reference set of 262,144 points in d = 96 (the serving workload's
    dimension) and 300 queries (two full query tiles and a ragged third), with
    the oracle's first 256 + 32 neighbours of every query."""
    m, d, n = 262_144, 96, 300
    R = inputs.uniform(m, d, seed=5101)
    Q = inputs.uniform(n, d, seed=5102)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(256, m), "l2")
    return R, Q, o_dist, o_idx


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("k", [128, 256])
def test_serving_k_range(knn, serving_range, precision, k):
    """k up to 256, as the serving workload draws it (4k = 512 and 1024
    re-rank candidates): recall 1.0 and the parity rule on every row."""
    R, Q, o_dist, o_idx = serving_range
    g_dist, g_idx = run(knn, R, Q, k, precision)
    check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k,
                   name=f"uniform_m262144_n300_d96_k{k} {precision}")


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_k500_large_candidate_pool(knn, precision):
    """k = 500: 2000 re-rank candidates per query, a pool above the 1536 keys
    the per-lane sorted stripes hold, so the prefix selection rescans shared
    memory for every output position."""
    m, d, n, k = 20_000, 32, 130, 500
    R = inputs.uniform(m, d, seed=5201)
    Q = inputs.uniform(n, d, seed=5202)
    g_dist, g_idx = run(knn, R, Q, k, precision)
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, m), "l2")
    check_all_rows(R, Q, g_dist, g_idx, o_dist, o_idx, k,
                   name=f"uniform_m20000_n130_d32_k500 {precision}")


def test_injected_allocation_failure_reports_oom(knn, monkeypatch):
    """KNN_FAULT_INJECT_OOM=1 makes the workspace allocator refuse: the search
    returns KNN_ERR_OOM, writes nothing, and the same handle searches normally
    once the variable is cleared."""
    import torch
    R = inputs.uniform(3000, 16, seed=5301)
    Q = inputs.uniform(200, 16, seed=5302)
    ix = knn.Index(0, "bf16")
    ix.set_reference(torch.from_numpy(R).cuda())
    monkeypatch.setenv("KNN_FAULT_INJECT_OOM", "1")
    dist = torch.full((200, 8), -1.0, device="cuda")
    idx = torch.full((200, 8), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(knn.KnnError) as e:
        ix.search_into(torch.from_numpy(Q).cuda(), 8, dist, idx, "l2")
    assert e.value.status == 2            # KNN_ERR_OOM
    assert "KNN_FAULT_INJECT_OOM" in str(e.value)
    torch.cuda.synchronize()
    assert torch.all(dist == -1.0) and torch.all(idx == -1)
    monkeypatch.delenv("KNN_FAULT_INJECT_OOM")
    g_dist, g_idx = ix.search(torch.from_numpy(Q).cuda(), 8, "l2")
    ix.sync()
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(8, 3000), "l2")
    check_all_rows(R, Q, g_dist.cpu().numpy(), g_idx.cpu().numpy(), o_dist, o_idx, 8)
    ix.close()
