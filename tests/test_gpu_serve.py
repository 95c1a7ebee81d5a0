"""Serving loop on the GPU (needs a GB300): requests overlapping on shared
reference slots give the same results as each alone, match the oracle, and
respect the memory budget."""
import numpy as np
import pytest

import oracle
from paper_0804_1448_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

M, D = 262144, 96


@pytest.fixture(scope="module")
def server():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_1448_gb300 import serve
    R = inputs.uniform(M, D, seed=41)
    srv = serve.Server(torch.from_numpy(R).cuda(), "bf16", slots=4, n_max=2048, k_max=64)
    yield srv, R
    srv.close()


def make_requests(count, seed, rate=None):
    import torch
    from paper_0804_1448_gb300 import serve
    reqs = serve.workload(count, seed, rate, n_max=2048, k_max=64)
    for r in reqs:
        Q = inputs.uniform(r.n, D, seed=100000 + 1000 * seed + r.rid)
        r.queries = torch.from_numpy(Q).cuda()
        r.host_q = Q
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix(server):
    import torch
    srv, R = server
    reqs = make_requests(24, 31)          # all arrive at once: the most overlap
    done, sched, out = srv.serve(reqs)
    assert sched.peak_running > 1, "no two requests were on the GPU together"
    mixed = {rid: (d.cpu(), i.cpu()) for rid, (d, i) in out.items()}
    for r in reqs:
        d1, i1 = srv.alone(r)
        assert torch.equal(i1.cpu(), mixed[r.rid][1]), f"request {r.rid}: indices differ"
        assert torch.equal(d1.cpu(), mixed[r.rid][0]), f"request {r.rid}: distances differ"


def test_mixed_results_match_the_oracle(server):
    srv, R = server
    reqs = make_requests(12, 32, rate=400.0)
    done, sched, out = srv.serve(reqs)
    rng = np.random.default_rng(5)
    for r in reqs[:6]:
        dist, idx = (t.cpu().numpy() for t in out[r.rid])
        sel = rng.choice(r.n, min(r.n, 8), replace=False)
        o_dist, o_idx = oracle.knn_subset(R, r.host_q, sel, parity.oracle_k(r.k, M), "l2")
        assert parity.recall(idx[sel], o_idx, r.k) == 1.0
        parity.compare(dist[sel], idx[sel], o_dist, o_idx, r.k, M)
    for r in done:
        assert r.done >= r.arrival


def test_memory_budget_bounds_what_runs_together(server):
    srv, R = server
    reqs = make_requests(16, 33)
    srv.sized(reqs)
    budget = 2 * max(r.ws_bytes for r in reqs)
    saved = srv.mem_budget
    srv.mem_budget = budget
    try:
        done, sched, out = srv.serve(reqs)
    finally:
        srv.mem_budget = saved
    assert sched.peak_mem <= budget
    assert sorted(r.rid for r in done) == list(range(16))
