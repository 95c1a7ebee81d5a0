"""Precision workload at full size: m = 1,048,576 references, n = 16,384 queries,
d = 128, k = 100, Gaussian mixture of 1024 centres (sigma = 0.05), searched in
one launch per form; 1024 sampled query rows (the first, the last and 1022
drawn with a fixed seed) are checked against the float64 oracle (needs a
GB300).

* float32 (CUDA-core select + exact re-check): parity rule of tests/parity.py
  on every sampled row.
* bf16 / tf32 (tensor-core filter, float32 re-rank of 400 candidates,
  float-float / float64 boundary re-check): recall@k = 1.0 over the sampled
  rows, the parity rule on every sampled row, and exact float32 distances for
  every returned reference.
"""
import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

N_SAMPLE = 1024


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_1448_gb300 import knn as mod
    return mod


@pytest.fixture(scope="module")
def mixture(knn):
    import torch
    R, Q, k = inputs.workload("mixture_m1048576_n16384_d128_k100")
    sel = np.random.default_rng(11).choice(Q.shape[0], N_SAMPLE, replace=False)
    sel[0], sel[1] = 0, Q.shape[0] - 1
    o_dist, o_idx = oracle.knn_subset(R, Q, sel, parity.oracle_k(k, R.shape[0]), "l2")
    return dict(R=R, Q=Q, k=k, sel=sel, o_dist=o_dist, o_idx=o_idx,
                Rd=torch.from_numpy(R).cuda(), Qd=torch.from_numpy(Q).cuda())


def search(knn, mix, precision):
    import torch
    ix = knn.Index(0, precision, rerank_factor=4)
    ix.set_reference(mix["Rd"])
    dist, idx = ix.search(mix["Qd"], mix["k"], "l2")
    torch.cuda.synchronize()
    st = ix.stats()
    ix.close()
    return dist.cpu().numpy(), idx.cpu().numpy(), st


def test_mixture_fp32_parity(knn, mixture):
    g_dist, g_idx, _ = search(knn, mixture, "fp32")
    sel, k, m = mixture["sel"], mixture["k"], mixture["R"].shape[0]
    parity.record("mixture_m1048576_n16384_d128_k100 fp32", g_dist[sel], g_idx[sel],
                  mixture["o_dist"], mixture["o_idx"], k)
    parity.compare(g_dist[sel], g_idx[sel], mixture["o_dist"], mixture["o_idx"], k, m)
    assert np.all(np.diff(g_dist, axis=1) >= 0)
    assert np.all((g_idx >= 0) & (g_idx < m))


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_mixture_tensor_core_recall(knn, mixture, precision):
    g_dist, g_idx, st = search(knn, mixture, precision)
    sel, k, R, Q = mixture["sel"], mixture["k"], mixture["R"], mixture["Q"]
    o_dist, o_idx = mixture["o_dist"], mixture["o_idx"]
    rec, err = parity.record(f"mixture_m1048576_n16384_d128_k100 {precision}", g_dist[sel],
                             g_idx[sel], o_dist, o_idx, k)
    print(f"{precision}: recall@{k} = {rec:.6f} on {len(sel)} sampled rows, "
          f"max rel dist err {err:.2e}, stats {st}")
    assert rec == 1.0
    parity.compare(g_dist[sel], g_idx[sel], o_dist, o_idx, k, R.shape[0])
    # every returned distance is that reference's exact distance
    qi = np.repeat(sel, k)
    keys = oracle.key_pairs(R, Q, qi, g_idx[sel].reshape(-1), "l2")
    np.testing.assert_allclose(g_dist[sel], np.sqrt(keys).reshape(len(sel), k), rtol=1e-5, atol=0)
    assert np.all(np.diff(g_dist, axis=1) >= 0)
