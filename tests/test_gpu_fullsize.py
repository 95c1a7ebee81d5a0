"""The bench workload at full size, every row against the oracle (needs a GB300).

n = m = 38400, d = 96, k = 20, uniform [0,1) (Table 1's largest cell): one
search of all 38400 queries in each form, and the oracle's first k + 32
neighbours of every query (computed once per distance, module fixtures).

* float32 CUDA-core form, Euclidean, Manhattan and Chebyshev: the parity rule
  of tests/parity.py on all 38400 rows.
* bf16 and tf32 tensor-core forms (low-precision filter, float32 re-rank of
  4k = 80 candidates, float-float / float64 re-check of near ties): recall@k
  must be 1.0 over all rows, the parity rule must hold on all rows, and every
  returned distance must be the exact distance of the returned reference.
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


@pytest.fixture(scope="module")
def bench_shape(knn):
    import torch
    R, Q, k = inputs.workload("uniform_n38400_d96_k20")
    return dict(R=R, Q=Q, k=k, Rd=torch.from_numpy(R).cuda(), Qd=torch.from_numpy(Q).cuda(),
                oracle={})


def oracle_rows(shape, metric):
    """The oracle's first k + 32 neighbours of all 38400 queries (cached)."""
    if metric not in shape["oracle"]:
        R, Q, k = shape["R"], shape["Q"], shape["k"]
        shape["oracle"][metric] = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), metric)
    return shape["oracle"][metric]


def search(knn, shape, precision, metric):
    import torch
    ix = knn.Index(0, precision, rerank_factor=4)
    ix.set_reference(shape["Rd"])
    dist, idx = ix.search(shape["Qd"], shape["k"], metric)
    ix.sync()
    st = ix.stats()
    ix.close()
    torch.cuda.synchronize()
    return dist.cpu().numpy(), idx.cpu().numpy(), st


@pytest.mark.parametrize("metric", ["l2", "l1", "linf"])
def test_fp32_every_row(knn, bench_shape, metric):
    g_dist, g_idx, _ = search(knn, bench_shape, "fp32", metric)
    o_dist, o_idx = oracle_rows(bench_shape, metric)
    k, m = bench_shape["k"], bench_shape["R"].shape[0]
    parity.record(f"uniform_n38400_d96_k20 fp32 {metric}", g_dist, g_idx, o_dist, o_idx, k)
    rows, _ = parity.compare(g_dist, g_idx, o_dist, o_idx, k, m)
    assert rows == 38400


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_tensor_core_every_row(knn, bench_shape, precision):
    g_dist, g_idx, st = search(knn, bench_shape, precision, "l2")
    o_dist, o_idx = oracle_rows(bench_shape, "l2")
    R, Q, k = bench_shape["R"], bench_shape["Q"], bench_shape["k"]
    rec, err = parity.record(f"uniform_n38400_d96_k20 {precision}", g_dist, g_idx, o_dist, o_idx,
                             k)
    print(f"{precision}: recall@{k} = {rec} over {len(Q)} rows, max rel dist err {err:.2e}, "
          f"stats {st}")
    assert rec == 1.0
    rows, _ = parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])
    assert rows == 38400
    qi = np.repeat(np.arange(Q.shape[0]), k)
    keys = oracle.key_pairs(R, Q, qi, g_idx.reshape(-1), "l2")
    np.testing.assert_allclose(g_dist, np.sqrt(keys).reshape(g_dist.shape), rtol=1e-5, atol=0)
