"""Batched search (knn_search_batch) on the GPU (needs a GB300).

Mixed batches (some Manhattan instances) and float32 batches run as a graph of
the instances' own launches: every instance gives exactly what a lone
knn_search gives, the float32 form matches the oracle under the parity rule,
graph replays, the no-graph form and the autotuned form agree, and bad
instances are refused.  Euclidean batches in bf16 / tf32 run as ONE persistent
kernel launch popping work items from a device queue: every instance matches
the oracle (recall 1.0 and the parity rule on every row), the launch count is
one, replays and the autotuned split lengths give the same results."""
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


def make_batch(count, seed, m_rng=(1000, 20000), n_rng=(16, 512), l1_every=5):
    """Instances with m, n uniform in the ranges, d in {32, 64, 128}, k in
    {1, 10, 50} (k <= m), float32 uniform data (the batching workload's
    distribution at test sizes); every l1_every-th instance Manhattan (0:
    none)."""
    import torch
    g = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(g.integers(m_rng[0], m_rng[1] + 1))
        n = int(g.integers(n_rng[0], n_rng[1] + 1))
        d = int(g.choice([32, 64, 128]))
        k = int(g.choice([1, 10, 50]))
        R = inputs.uniform(m, d, seed=10000 + 2 * (seed * 1000 + i))
        Q = inputs.uniform(n, d, seed=10001 + 2 * (seed * 1000 + i))
        out.append(dict(R=torch.from_numpy(R).cuda(), Q=torch.from_numpy(Q).cuda(), k=k,
                        dist=torch.empty((n, k), device="cuda"),
                        idx=torch.empty((n, k), dtype=torch.int32, device="cuda"),
                        R_host=R, Q_host=Q,
                        metric="l1" if l1_every and i % l1_every == 0 else "l2"))
    return out


def lone(knn, precision, x):
    ix = knn.Index(0, precision)
    ix.set_reference(x["R"])
    d, i = ix.search(x["Q"], x["k"], x["metric"])
    ix.sync()
    ix.close()
    return d.cpu(), i.cpu()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_equals_lone_searches(knn, precision):
    import torch
    batch = make_batch(24, seed=1)
    ix = knn.Index(0, precision)
    ix.search_batch(batch)
    ix.sync()
    info = ix.batch_info()
    assert info["graph_nodes"] > 0 and info["branches"] > 1
    for j, x in enumerate(batch):
        d1, i1 = lone(knn, precision, x)
        assert torch.equal(x["idx"].cpu(), i1), f"instance {j}: indices differ from a lone search"
        if precision == "fp32":
            assert torch.equal(x["dist"].cpu(), d1), f"instance {j}: distances differ"
        else:
            # a batch instance is planned for a share of the SMs, so its pilot
            # samples other tiles and its candidate set can differ; an entry
            # re-checked in float-float in one plan and not in the other then
            # differs in the last bits of its distance
            np.testing.assert_allclose(x["dist"].cpu().numpy(), d1.numpy(), rtol=1e-6, atol=0)
    ix.close()


def test_batch_fp32_matches_the_oracle(knn):
    batch = make_batch(12, seed=2)
    ix = knn.Index(0, "fp32")
    ix.search_batch(batch)
    ix.sync()
    rng = np.random.default_rng(3)
    for x in batch:
        R, Q, k = x["R_host"], x["Q_host"], x["k"]
        sel = rng.choice(Q.shape[0], min(16, Q.shape[0]), replace=False)
        o_dist, o_idx = oracle.knn_subset(R, Q, sel, parity.oracle_k(k, R.shape[0]), x["metric"])
        parity.compare(x["dist"].cpu().numpy()[sel], x["idx"].cpu().numpy()[sel], o_dist, o_idx,
                       k, R.shape[0])
    ix.close()


def test_replay_no_graph_and_autotune_agree(knn):
    import torch
    batch = make_batch(16, seed=4)
    ix = knn.Index(0, "bf16")
    ix.search_batch(batch)
    ix.sync()
    ref = [(x["dist"].cpu().clone(), x["idx"].cpu().clone()) for x in batch]
    for x in batch:
        x["dist"].fill_(-1.0)
        x["idx"].fill_(-1)
    ix.search_batch(batch)                       # cached graph: one launch
    ix.sync()
    assert ix.batch_info()["tuned"] == 0
    for x, (d, i) in zip(batch, ref):
        assert torch.equal(x["dist"].cpu(), d) and torch.equal(x["idx"].cpu(), i)
    for x in batch:
        x["idx"].fill_(-1)
    ix.search_batch(batch, flags=knn.KNN_BATCH_NO_GRAPH)
    ix.sync()
    assert ix.batch_info()["graph_nodes"] == 0
    for x, (d, i) in zip(batch, ref):
        assert torch.equal(x["idx"].cpu(), i)
    ix.close()
    ix = knn.Index(0, "bf16")
    ix.search_batch(batch, flags=knn.KNN_BATCH_AUTOTUNE)
    ix.sync()
    first = ix.batch_info()
    assert first["tuned"] == 1 and first["tune_ms"] > 0
    ix.search_batch(batch, flags=knn.KNN_BATCH_AUTOTUNE)
    ix.sync()
    second = ix.batch_info()
    assert second["tuned"] == 0 and second["branches"] == first["branches"]
    for x, (d, i) in zip(batch, ref):
        assert torch.equal(x["idx"].cpu(), i)
    ix.close()


def test_bad_instances_are_refused(knn):
    import torch
    batch = make_batch(3, seed=5)
    ix = knn.Index(0, "fp32")
    bad = dict(batch[1])
    bad["k"] = bad["R"].shape[0] + 1
    with pytest.raises(knn.KnnError) as e:
        ix.search_batch([batch[0], bad, batch[2]])
    assert e.value.status == 1
    ix.search_batch([])                          # an empty batch is a no-op
    ix.close()


# ------------------------------------------------------------- persistent form

def check_instances(batch):
    """Every row of every instance against the oracle: recall@k 1.0 and the
    parity rule."""
    for j, x in enumerate(batch):
        R, Q, k = x["R_host"], x["Q_host"], x["k"]
        o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), x["metric"])
        g_dist, g_idx = x["dist"].cpu().numpy(), x["idx"].cpu().numpy()
        assert parity.recall(g_idx, o_idx, k) == 1.0, f"instance {j}"
        parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_persistent_batch_matches_the_oracle(knn, precision):
    """24 Euclidean instances (m from 1000, below the size the pilot needs, to
    20000; n from 16 to 512; d in {32, 64, 128}; k in {1, 10, 50}) in one
    kernel launch."""
    batch = make_batch(24, seed=11, l1_every=0)
    ix = knn.Index(0, precision)
    ix.search_batch(batch)
    ix.sync()
    info = ix.batch_info()
    assert info["persistent"] == 1 and info["launches"] == 1 and info["items"] > 24
    check_instances(batch)
    st = ix.stats()
    assert st["searches"] == 24
    # where the launch spent its time: every item counted once, per stage
    times = ix.batch_stage_times()
    assert sum(v["items"] for v in times.values()) == info["items"]
    assert times["filter"]["items"] > 0 and times["filter"]["work_ms"] > 0
    assert times["finalize"]["items"] > 0 and all(v["wait_ms"] >= 0 for v in times.values())
    # a later search clears them
    ix.set_reference(batch[0]["R"])
    ix.search(batch[0]["Q"], 1, "l2")
    with pytest.raises(knn.KnnError) as e:
        ix.batch_stage_times()
    assert e.value.status == 7   # KNN_ERR_UNSUPPORTED
    ix.close()


def test_persistent_replay_and_autotune(knn):
    import torch
    batch = make_batch(16, seed=12, l1_every=0)
    ix = knn.Index(0, "bf16")
    ix.search_batch(batch)
    ix.sync()
    ref = [(x["dist"].cpu().clone(), x["idx"].cpu().clone()) for x in batch]
    for x in batch:
        x["dist"].fill_(-1.0)
        x["idx"].fill_(-1)
    ix.search_batch(batch)                       # cached graph: the same launch again
    ix.sync()
    info = ix.batch_info()
    assert info["persistent"] == 1 and info["tuned"] == 0
    for x, (d, i) in zip(batch, ref):
        assert torch.equal(x["dist"].cpu(), d) and torch.equal(x["idx"].cpu(), i)
    ix.close()
    ix = knn.Index(0, "bf16")
    ix.search_batch(batch, flags=knn.KNN_BATCH_AUTOTUNE)
    ix.sync()
    first = ix.batch_info()
    assert first["persistent"] == 1 and first["tuned"] == 1 and first["tune_ms"] > 0
    check_instances(batch)
    ix.search_batch(batch, flags=knn.KNN_BATCH_AUTOTUNE)   # tuned shape: no new tuning
    ix.sync()
    assert ix.batch_info()["tuned"] == 0
    check_instances(batch)
    # the graph of per-instance launches, asked for explicitly, agrees
    for x in batch:
        x["idx"].fill_(-1)
    ix.search_batch(batch, flags=knn.KNN_BATCH_BRANCHES)
    ix.sync()
    assert ix.batch_info()["persistent"] == 0
    check_instances(batch)
    ix.close()


def test_persistent_edge_instances(knn):
    """Instances at the edges: one query, n = 129 (a ragged second query
    tile), k = m, m below one reference tile, duplicated references (exact
    fallback), a reference set with every point equal."""
    import torch
    rng_seed = 13
    specs = [(1, 5000, 32, 10), (129, 3000, 64, 50), (40, 50, 32, 50), (77, 200, 128, 1)]
    batch = []
    for j, (n, m, d, k) in enumerate(specs):
        R = inputs.uniform(m, d, seed=20000 + 2 * j)
        Q = inputs.uniform(n, d, seed=20001 + 2 * j)
        batch.append(dict(R_host=R, Q_host=Q, k=k, metric="l2"))
    base = inputs.uniform(800, 32, seed=20100)
    batch.append(dict(R_host=np.concatenate([base, base, base]), Q_host=base[:60].copy(), k=9,
                      metric="l2"))
    batch.append(dict(R_host=np.full((3000, 32), 0.5, dtype=np.float32),
                      Q_host=inputs.uniform(20, 32, seed=20101), k=10, metric="l2"))
    for x in batch:
        n, k = x["Q_host"].shape[0], x["k"]
        x.update(R=torch.from_numpy(x["R_host"]).cuda(), Q=torch.from_numpy(x["Q_host"]).cuda(),
                 dist=torch.empty((n, k), device="cuda"),
                 idx=torch.empty((n, k), dtype=torch.int32, device="cuda"))
    ix = knn.Index(0, "bf16")
    ix.search_batch(batch)
    ix.sync()
    assert ix.batch_info()["persistent"] == 1
    check_instances(batch)
    assert ix.stats()["fallback_queries"] >= 20   # the equal-points instance
    ix.close()
