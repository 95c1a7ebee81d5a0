"""Search planning on the host (knn_explain_plan; no GPU): the plan of the
bench shape, the pilot's invariants over the Table 1 grid and the serving
shape, which searches run on tensor cores, the reference splits of the
float32 form, and argument checks."""
import math

import pytest

from paper_0804_1448_gb300 import knn

SMS = 152   # GB300


def plan(n, m, d, k, **kw):
    kw.setdefault("num_sms", SMS)
    return knn.explain_plan(n, m, d, k, **kw)


def test_bench_shape():
    p = plan(38400, 38400, 96, 20)
    assert p["tensor_cores"] == 1 and p["candidates"] == 80
    assert p["splits"] == 1 and p["chunk"] == 38400          # 300 query tiles fill two waves
    assert p["k_blocks"] == 2 and p["whole_tile_stages"] == 1 and p["stages"] == 2
    assert p["raw_staging"] == 1
    assert p["pilot"] == 1 and p["pilot_stride"] == 16
    assert p["pilot_groups"] == 80                             # 10 sampled tiles x 8 groups
    assert p["threshold_rank"] == 19                           # lambda = 80 * 10/150
    assert p["list_capacity"] == 256


@pytest.mark.parametrize("N", [1200, 2400, 4800, 9600, 19200, 38400])
@pytest.mark.parametrize("D", [8, 16, 32, 64, 80, 96])
def test_table1_grid_invariants(N, D):
    p = plan(N, N, D, 20)
    # an SM's share of the small-set select's distance products (CTAs of 8 queries)
    share = math.ceil(N / 8) * N * D / SMS
    if N < 4800 and share < 2.2e5:
        # the exact float32 small-set select (all N distances of a query in
        # shared memory) is faster than the tensor-core passes here
        assert p["tensor_cores"] == 0 and p["small_select"] == 1
        assert p["splits"] == 1 and p["chunk"] == N and p["candidates"] == 28 + 16
        return
    assert p["tensor_cores"] == 1 and p["small_select"] == 0
    assert p["chunk"] % 256 == 0 and p["splits"] * p["chunk"] >= N
    assert (p["splits"] - 1) * p["chunk"] < N                 # no empty split
    assert 1 <= p["splits"] <= 256
    assert p["list_capacity"] % 32 == 0
    assert p["pilot"] == 1
    assert p["pilot_groups"] <= 2048
    # the c'-th largest of the group maxima needs groups to spare
    assert p["pilot_groups"] >= p["threshold_rank"] + 8
    if N == 2400:
        # every tile sampled: c' = c, and groups of 16 (75 groups of 32 are too few)
        assert p["pilot_stride"] == 1 and p["threshold_rank"] == p["candidates"]
        assert p["pilot_group_size"] == 16 and p["pilot_groups"] == 2 * 5 * 16
    else:
        assert p["pilot_group_size"] == 32


def test_pilot_groups_shrink_when_every_tile_is_sampled():
    # m = 777: 25 groups of 32 or 49 of 16 are too few for c' = c = 80 (+8)
    p = plan(12000, 777, 40, 20)
    assert p["tensor_cores"] == 1 and p["pilot_stride"] == 1
    assert p["pilot_group_size"] == 8 and p["threshold_rank"] == 80
    assert p["pilot_groups"] == 4 * 32                         # 4 tiles x 8 slices x 4 groups
    # m = 600: 75 groups of 8 are too few; no pilot, so the small-set select
    p = plan(12000, 600, 40, 20)
    assert p["tensor_cores"] == 0 and p["small_select"] == 1
    # sampled pilots keep groups of 32 and the Poisson margin
    p = plan(38400, 38400, 96, 20)
    assert p["pilot_group_size"] == 32 and p["threshold_rank"] > p["candidates"] * 10 / 150


@pytest.mark.parametrize("n", [1, 64, 256])
def test_small_batches_spread_over_every_sm(n):
    p = plan(n, 4194304, 96, 20)
    ctas = math.ceil(n / 128) * p["splits"]                    # query tiles x reference splits
    assert ctas >= math.ceil(0.85 * SMS)                       # most SMs busy
    assert p["pilot"] == 1 and p["pilot_groups"] <= 2048


def test_which_searches_use_tensor_cores():
    assert plan(1000, 5000, 32, 10, precision="fp32")["tensor_cores"] == 0
    assert plan(1000, 5000, 32, 10, metric="l1")["tensor_cores"] == 0
    assert plan(1000, 5000, 32, 10, metric="linf")["tensor_cores"] == 0
    assert plan(1000, 5000, 32, 10, metric="mahalanobis")["tensor_cores"] == 1
    # rows longer than the tensor-core tile holds run in float32
    assert plan(100, 5000, 444, 10)["tensor_cores"] == 1
    assert plan(100, 5000, 445, 10)["tensor_cores"] == 0
    assert plan(100, 5000, 220, 10, precision="tf32")["tensor_cores"] == 1
    assert plan(100, 5000, 221, 10, precision="tf32")["tensor_cores"] == 0


def test_rerank_factor_sets_the_candidates():
    assert plan(5000, 50000, 64, 10, rerank_factor=4)["candidates"] == 40
    assert plan(5000, 50000, 64, 10, rerank_factor=8)["candidates"] == 80


def test_bad_arguments_are_refused():
    with pytest.raises(knn.KnnError) as e:
        plan(10, 100, 8, 101)                                  # k > m
    assert e.value.status == 1
    for bad in (dict(n=0), dict(d=0), dict(num_sms=0), dict(rerank_factor=0)):
        args = dict(n=10, m=100, d=8, k=5)
        args.update(bad)
        with pytest.raises(knn.KnnError):
            knn.explain_plan(args.pop("n"), args.pop("m"), args.pop("d"), args.pop("k"), **args)
    with pytest.raises(knn.KnnError) as e:
        plan(10, 5000, 8, 2000)                                # k above KNN_K_MAX
    assert e.value.status == 7


# ---------------------------------------------------------------------------
# float32 CUDA-core form: reference splits
# ---------------------------------------------------------------------------
def fp32(n, m, d, k, **kw):
    return plan(n, m, d, k, precision="fp32", **kw)


def test_fp32_bench_shape_keeps_one_split():
    # 300 tiles of 128 queries, two CTAs per SM: one wave of 300 CTAs on the
    # 304 slots, which splitting the references cannot shorten
    p = fp32(38400, 38400, 96, 20)
    assert p["tensor_cores"] == 0 and p["candidates"] == 28    # k + max(8, k/4)
    assert p["splits"] == 1 and p["chunk"] == 38400


def test_fp32_long_reference_set_is_split():
    # 256 query tiles, k = 100: two CTAs per SM; one split per query tile
    # would leave a last wave of 208 CTAs holding two on most SMs
    p = fp32(16384, 1 << 20, 128, 100)
    assert p["candidates"] == 125 and p["splits"] == 7


@pytest.mark.parametrize("N,S", [(4800, 6), (9600, 6), (19200, 3), (38400, 1)])
def test_fp32_table1_splits(N, S):
    # at least two CTAs per SM where the query tiles alone give fewer (with
    # 5% slack); query tiles of 64 rows below 8192 queries, of 128 above
    p = fp32(N, N, 96, 20)
    assert p["splits"] == S
    tiles = math.ceil(N / (128 if N >= 8192 else 64))
    if tiles * 100 < 95 * 2 * SMS:
        # splits no longer than those of the smallest count giving two CTAs
        # per SM (or of the most splits 8c-long references allow)
        s_min = min(math.ceil(2 * SMS / tiles), N // (8 * 28))
        assert p["chunk"] <= math.ceil(math.ceil(N / s_min) / 128) * 128


@pytest.mark.parametrize("n,m,k", [(1, 1000, 5), (64, 4194304, 20), (700, 5000, 16), (4096, 4194304, 20),
                                   (38400, 38400, 1000), (100000, 1000, 5), (333, 123457, 64)])
def test_fp32_split_invariants(n, m, k):
    p = fp32(n, m, 24, k)
    S, chunk, c = p["splits"], p["chunk"], p["candidates"]
    if p["small_select"]:                                               # one split of the whole set
        assert S == 1 and chunk == m and c <= m
        return
    assert chunk % 128 == 0 and S * chunk >= m and (S - 1) * chunk < m   # no empty split
    assert S * c <= 4096                                                 # one finalize pool
    if S > 1:
        assert chunk >= 8 * c - 127                                     # splits much longer than c


@pytest.mark.parametrize("m,d,small", [(1200, 8, 1), (4096, 96, 1), (4097, 96, 0), (4096, 256, 1),
                                       (4096, 444, 1), (4096, 3000, 0), (2000, 200, 1)])
def test_small_reference_sets_use_the_small_select(m, d, small):
    """Reference sets of at most 4096 points whose distances, eight query rows
    of them, fit one CTA's shared memory take the small-set select (one split
    of k + max(8, k/4) keys per query and 16 spare slots); larger ones the
    tiled select."""
    p = fp32(300, m, d, 20)
    assert p["small_select"] == small and p["tensor_cores"] == 0
    if small:
        assert p["splits"] == 1 and p["chunk"] == m and p["candidates"] == 28 + 16
