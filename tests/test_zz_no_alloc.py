"""knn_search_static: the allocation-free entry point (needs a GB300).

Callers that cannot allocate device memory when they search (a framework that
hands out all device memory from its own pool, a latency-critical path that
cannot take the device-wide synchronisation of cudaMalloc/cudaFree) use
knn_search_static, which keeps its intermediates in a fixed 32 MiB __device__
array of the library instead of a handle's workspace.  This file checks,
through the C ABI, that two calls in a row give the oracle's result under the
parity rule the other tests use and the same result as the handle-based
knn_search, and that a problem too large for the array is refused.  It is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_1448_gb300 import knn
    return torch, knn


def static_search(torch, knn, Rd, Qd, k, metric):
    n, d = Qd.shape
    dist = torch.full((n, k), -1.0, dtype=torch.float32, device="cuda")
    idx = torch.full((n, k), -2, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream or 1
    st = knn.knn_search_static(Rd.data_ptr(), Rd.shape[0], Qd.data_ptr(), n, d, k,
                               knn.METRICS[metric], dist.data_ptr(), idx.data_ptr(), stream)
    assert st == 0, knn.STATUS.get(st, st)
    torch.cuda.synchronize()
    return dist.cpu().numpy(), idx.cpu().numpy()


@pytest.mark.parametrize("metric", ["l2", "l1", "linf"])
def test_two_calls_match_knn_search(env, metric):
    torch, knn = env
    R = inputs.uniform(5000, 24, seed=401)
    Rd = torch.from_numpy(R).cuda()
    ix = knn.Index(0, "fp32")
    ix.set_reference(Rd)
    for call, (n, seed) in enumerate(((700, 402), (333, 403))):
        Q = inputs.uniform(n, 24, seed=seed)
        Qd = torch.from_numpy(Q).cuda()
        k = 16
        s_dist, s_idx = static_search(torch, knn, Rd, Qd, k, metric)
        o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(k, R.shape[0]), metric)
        parity.compare(s_dist, s_idx, o_dist, o_idx, k, R.shape[0])
        h_dist, h_idx = ix.search(Qd, k, metric)
        torch.cuda.synchronize()
        h_dist, h_idx = h_dist.cpu().numpy(), h_idx.cpu().numpy()
        # and the result of the existing entry point, under the same rule
        parity.compare(s_dist, s_idx, h_dist.astype(np.float64), h_idx, k, R.shape[0])
    ix.close()


def test_duplicates_go_through_the_exact_fallback(env):
    torch, knn = env
    R = np.full((900, 6), 0.25, dtype=np.float32)
    Rd = torch.from_numpy(R).cuda()
    Qd = torch.from_numpy(np.array([[0.25] * 6, [0.75] * 6], dtype=np.float32)).cuda()
    for _ in range(2):
        dist, idx = static_search(torch, knn, Rd, Qd, 12, "l2")
        assert idx.tolist() == [list(range(12))] * 2
        np.testing.assert_allclose(dist[1], np.full(12, np.sqrt(6 * 0.25)), rtol=1e-7)


def test_problem_too_large_for_the_static_scratch_is_refused(env):
    torch, knn = env
    n, m, d, k = 2_000_000, 1000, 8, 16          # candidates alone would need ~0.4 GB
    Rd = torch.rand((m, d), device="cuda")
    Qd = torch.rand((n, d), device="cuda")
    dist = torch.empty((n, k), dtype=torch.float32, device="cuda")
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    st = knn.knn_search_static(Rd.data_ptr(), m, Qd.data_ptr(), n, d, k, knn.KNN_L2,
                               dist.data_ptr(), idx.data_ptr(), None)
    assert st == 7   # KNN_ERR_UNSUPPORTED
