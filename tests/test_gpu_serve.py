"""The continuous-batching server on the GPU: requests of different N, s and
perplexity arrive while others run, are admitted under an HBM budget that
forces queueing, overlap on the device, and each result equals the same job
run alone (bitwise: the kernels never mix jobs and reduce in a fixed order).
"""
import numpy as np
import pytest
import torch

import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs
from paper_1712_09005_gb300.serve import Request, Server, poisson_arrivals, run_alone

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def requests(n, seed=5):
    rng = np.random.default_rng(seed)
    sizes = inputs.log_uniform_sizes(n, 400, 4000, seed=seed)
    arr = poisson_arrivals(n, 400.0, seed=seed)  # all arrive within ~25 ms
    out = []
    for i in range(n):
        N = int(sizes[i])
        s = int(rng.integers(1, 3))
        perp = float(rng.choice([10.0, 30.0]))
        args = inputs.mixture_args(5, job=i, N=N)
        P = inputs.affinities(inputs.mixture(**args), perp, device="cuda")
        Y0 = inputs.initial_embedding(N, s, seed=args["seed"])
        out.append(Request(i, float(arr[i]), s, P.row_ptr, P.col, P.val, Y0,
                           pkg.Schedule(n_iter=80, early_iters=30)))
    return out


def test_served_results_equal_alone_and_budget_holds():
    reqs = requests(10)
    probe = pkg.Batch(2, max_jobs=1)
    per_job = max(probe.job_bytes(r.N) + r.p_bytes for r in reqs)
    probe.close()
    budget = 3 * per_job  # at most about three resident jobs: requests queue
    srv = Server(budget_bytes=budget, max_jobs=4, iters_per_round=10)
    try:
        out = srv.serve(reqs)
    finally:
        srv.close()
    res = {r.rid: r for r in out["results"]}
    assert sorted(res) == list(range(len(reqs)))
    assert all(r.status == 0 for r in res.values())
    assert srv.peak_used <= budget
    assert any(r.admitted > r.arrival + 5e-3 for r in res.values())  # some waited for memory
    assert out["p99_s"] >= out["p50_s"] > 0
    for req in reqs:
        alone = run_alone(req)
        assert np.array_equal(res[req.rid].Y, alone), req.rid
