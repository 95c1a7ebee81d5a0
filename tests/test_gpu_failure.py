"""Failure detection of the bounded device-side waits, on the GPU (needs a
GB300), without a fault: a wait that nothing completes gives up after its
short limit, raises the handle's error flag, and the host reports
KNN_ERR_TIMEOUT; the handle and the context stay usable."""
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


def test_a_wait_that_runs_out_is_reported_and_the_handle_recovers(knn):
    import torch
    ix = knn.Index(0, "bf16")
    status = knn.knn_selftest_bounded_wait(ix.h, 20)        # 20 ms limit
    assert status == 4                                      # KNN_ERR_TIMEOUT
    assert knn.knn_sync(ix.h) == 0                          # the flag was cleared
    R = inputs.uniform(3000, 16, seed=8801)
    Q = inputs.uniform(50, 16, seed=8802)
    ix.set_reference(torch.from_numpy(R).cuda())
    dist, idx = ix.search(torch.from_numpy(Q).cuda(), 8, "l2")
    ix.sync()
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(8, 3000), "l2")
    parity.compare(dist.cpu().numpy(), idx.cpu().numpy(), o_dist, o_idx, 8, 3000)
    ix.close()


def test_limits_are_checked(knn):
    ix = knn.Index(0, "fp32")
    assert knn.knn_selftest_bounded_wait(ix.h, 0) == 1      # KNN_ERR_INVALID
    assert knn.knn_selftest_bounded_wait(ix.h, 5000) == 1
    ix.close()


def test_persistent_batch_queue_wait_runs_out(knn):
    """The persistent batch kernel with its ready word withheld: every CTA's
    first wait gives up after 20 ms, raises the error flag and leaves; the
    host reports KNN_ERR_TIMEOUT, and the same handle then runs a batch."""
    import torch
    ix = knn.Index(0, "bf16")
    assert knn.knn_selftest_batch_queue(ix.h, 20) == 4      # KNN_ERR_TIMEOUT
    assert knn.knn_sync(ix.h) == 0
    assert knn.knn_selftest_batch_queue(ix.h, 0) == 1       # KNN_ERR_INVALID
    R = inputs.uniform(4000, 32, seed=8811)
    Q = inputs.uniform(70, 32, seed=8812)
    x = dict(R=torch.from_numpy(R).cuda(), Q=torch.from_numpy(Q).cuda(), k=6,
             dist=torch.empty((70, 6), device="cuda"),
             idx=torch.empty((70, 6), dtype=torch.int32, device="cuda"))
    ix.search_batch([x])
    ix.sync()
    assert ix.batch_info()["persistent"] == 1
    o_dist, o_idx = oracle.knn(R, Q, parity.oracle_k(6, 4000), "l2")
    parity.compare(x["dist"].cpu().numpy(), x["idx"].cpu().numpy(), o_dist, o_idx, 6, 4000)
    ix.close()
