"""Mahalanobis distance (Sec. 2.1) on the GPU (needs a GB300): a Euclidean
search of whitened points x' = L^T x, S^-1 = L L^T, in every precision,
against the oracle's quadratic form in float64 (oracle.knn_mahalanobis), under
the parity rule of tests/parity.py; the identity matrix reproduces the
Euclidean search bit for bit; host buffers; a new reference set is
re-whitened; bad matrices and unsupported entry points are refused."""
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


def spd(d, seed, cond=30.0):
    """Inverse covariance with eigenvalues spread over [1, cond] (seeded)."""
    g = np.random.Generator(np.random.Philox(seed))
    Qm, _ = np.linalg.qr(g.standard_normal((d, d)))
    ev = np.geomspace(1.0, cond, d)
    M = (Qm * ev) @ Qm.T
    return 0.5 * (M + M.T)


def search(knn, R, Q, k, precision, M, device_io=True):
    import torch
    ix = knn.Index(0, precision)
    ix.set_mahalanobis(M)
    if device_io:
        ix.set_reference(torch.from_numpy(R).cuda())
        dist, idx = ix.search(torch.from_numpy(Q).cuda(), k, "mahalanobis")
        ix.sync()
        out = dist.cpu().numpy(), idx.cpu().numpy()
    else:
        ix.set_reference(R)
        out = ix.search(Q, k, "mahalanobis")
    st = ix.stats()
    ix.close()
    return out[0], out[1], st


@pytest.mark.parametrize("precision", ["fp32", "bf16", "tf32"])
@pytest.mark.parametrize("n,m,d,k", [(300, 4099, 24, 10), (130, 2000, 96, 20), (7, 300, 3, 5)])
def test_matches_the_oracle(knn, precision, n, m, d, k):
    R = inputs.uniform(m, d, seed=7000 + d)
    Q = inputs.uniform(n, d, seed=7100 + d)
    M = spd(d, 7200 + d)
    g_dist, g_idx, st = search(knn, R, Q, k, precision, M)
    o_dist, o_idx = oracle.knn_mahalanobis(R, Q, M, parity.oracle_k(k, m))
    if precision != "fp32":
        assert parity.recall(g_idx, o_idx, k) == 1.0
    parity.compare(g_dist, g_idx, o_dist, o_idx, k, m)


def test_identity_matrix_is_the_euclidean_search(knn):
    import torch
    R = inputs.uniform(3000, 32, seed=7301)
    Q = inputs.uniform(200, 32, seed=7302)
    ix = knn.Index(0, "fp32")
    ix.set_reference(torch.from_numpy(R).cuda())
    ix.set_mahalanobis(np.eye(32))
    d1, i1 = ix.search(torch.from_numpy(Q).cuda(), 16, "l2")
    d2, i2 = ix.search(torch.from_numpy(Q).cuda(), 16, "mahalanobis")
    ix.sync()
    assert torch.equal(i1, i2) and torch.equal(d1, d2)
    ix.close()


def test_host_buffers_and_a_new_reference_set(knn):
    d, k = 16, 12
    M = spd(d, 7401)
    Q = inputs.uniform(64, d, seed=7402)
    ix = knn.Index(0, "bf16")
    ix.set_mahalanobis(M)
    for seed in (7403, 7404):                  # the second set must be re-whitened
        R = inputs.uniform(2500, d, seed=seed)
        ix.set_reference(R)
        g_dist, g_idx = ix.search(Q, k, "mahalanobis")
        o_dist, o_idx = oracle.knn_mahalanobis(R, Q, M, parity.oracle_k(k, R.shape[0]))
        assert parity.recall(g_idx, o_idx, k) == 1.0
        parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])
    ix.close()


def test_refusals(knn):
    import torch
    R = torch.from_numpy(inputs.uniform(500, 8, seed=7501)).cuda()
    Q = torch.from_numpy(inputs.uniform(10, 8, seed=7502)).cuda()
    ix = knn.Index(0, "fp32")
    ix.set_reference(R)
    with pytest.raises(knn.KnnError) as e:          # no matrix yet
        ix.search(Q, 5, "mahalanobis")
    assert e.value.status == 1
    bad = np.eye(8)
    bad[3, 3] = -1.0                                 # not positive definite
    with pytest.raises(knn.KnnError) as e:
        ix.set_mahalanobis(bad)
    assert e.value.status == 1
    ix.set_mahalanobis(np.eye(6))                    # wrong dimension for this set
    with pytest.raises(knn.KnnError) as e:
        ix.search(Q, 5, "mahalanobis")
    assert e.value.status == 1
    ix.set_mahalanobis(np.eye(8))
    with pytest.raises(knn.KnnError) as e:          # self-join: not offered
        ix.search_self(3, "mahalanobis")
    assert e.value.status == 7                       # KNN_ERR_UNSUPPORTED
    ix.set_mahalanobis(None)
    with pytest.raises(knn.KnnError):
        ix.search(Q, 5, "mahalanobis")
    ix.close()
