"""Self-join with self-exclusion (knn_search_self) and the Sec. 2.2
applications on the GPU (needs a GB300), against the oracle."""
import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import apps, inputs
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_1448_gb300 import knn as mod
    return mod


def oracle_self(R, K):
    """The oracle's first K neighbours of every point among the others."""
    dist, idx = oracle.knn(R, R, min(R.shape[0], K + 1), "l2")
    D = np.empty((R.shape[0], K))
    I = np.empty((R.shape[0], K), dtype=np.int64)
    for i in range(R.shape[0]):
        keep = [s for s in range(idx.shape[1]) if idx[i, s] != i][:K]
        D[i], I[i] = dist[i, keep], idx[i, keep]
    return D, I


def self_data():
    R = inputs.uniform(4000, 16, seed=601)
    R[3000:3050] = R[100:150]            # duplicates: other points at distance 0 stay
    return R


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_self_join_matches_the_oracle(knn, precision):
    import torch
    R = self_data()
    k = 10
    ix = knn.Index(0, precision)
    ix.set_reference(torch.from_numpy(R).cuda())
    dist, idx = ix.search_self(k)
    ix.sync()
    g_dist, g_idx = dist.cpu().numpy(), idx.cpu().numpy()
    ix.close()
    assert np.all(g_idx != np.arange(R.shape[0])[:, None]), "a point is its own neighbour"
    o_dist, o_idx = oracle_self(R, k + 32)
    if precision == "fp32":
        parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])
    else:
        assert parity.recall(g_idx, o_idx, k) == 1.0
        parity.compare(g_dist, g_idx, o_dist, o_idx, k, R.shape[0])
    # duplicated rows find their twin at distance 0
    assert np.all(g_dist[3000:3050, 0] == 0.0)
    np.testing.assert_array_equal(g_idx[3000:3050, 0], np.arange(100, 150))


def test_entropy_matches_the_oracle_distances(knn):
    import torch
    R = inputs.uniform(20000, 3, seed=602)
    ix = knn.Index(0, "fp32")
    ix.set_reference(torch.from_numpy(R).cuda())
    H = apps.entropy(ix, 4)
    ix.close()
    o_dist, _ = oracle_self(R, 4)
    H_o = apps.entropy_from_rho(o_dist[:, 3], 3, 4)
    assert H == pytest.approx(H_o, abs=1e-5)
    assert abs(H) < 0.08                 # uniform in the unit cube: true entropy 0 (edge bias)


def test_classification_matches_the_oracle_vote(knn):
    import torch
    centres = np.array([[0.2] * 8, [0.8] * 8, [0.2] * 4 + [0.8] * 4], dtype=np.float32)
    g = np.random.Generator(np.random.Philox(603))
    lab = g.integers(0, 3, size=3000)
    R = (centres[lab] + 0.12 * g.standard_normal((3000, 8))).astype(np.float32)
    ql = g.integers(0, 3, size=500)
    Q = (centres[ql] + 0.12 * g.standard_normal((500, 8))).astype(np.float32)
    ix = knn.Index(0, "fp32")
    ix.set_reference(torch.from_numpy(R).cuda())
    pred = apps.classify(ix, lab, torch.from_numpy(Q).cuda(), 7)
    ix.close()
    _, o_idx = oracle.knn(R, Q, 7, "l2")
    np.testing.assert_array_equal(pred, apps.majority_vote(lab[o_idx]))
    assert np.mean(pred == ql) > 0.95
