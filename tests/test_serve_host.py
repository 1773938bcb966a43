"""Host-side scheduling of the serving loop (no GPU): admission under the HBM
budget in arrival order, continuous batching, retirement. The device batch
is replaced by a stand-in that counts iterations; the kernels are covered by
the GPU tests (test_gpu_serve.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _Y:
    def __init__(self, n):
        self.n = n

    def cpu(self):
        return self

    def numpy(self):
        return np.zeros(self.n, np.float32)


class FakeBatch:
    """Stand-in for paper_1712_09005_gb300.Batch: jobs advance one iteration
    per iterate() step until their schedule ends."""

    def __init__(self, s, max_jobs=3, bytes_per_point=100):
        self.s, self.max_jobs, self.bpp = s, max_jobs, bytes_per_point
        self.jobs = {}

    def job_bytes(self, N):
        return self.bpp * N

    def upload(self, req):
        return None, None

    def add(self, P, Y0, sched, n_int):
        j = next(i for i in range(self.max_jobs) if i not in self.jobs)
        self.jobs[j] = [0, sched.n_iter]
        return j

    def iterate(self, k):
        for v in self.jobs.values():
            v[0] = min(v[1], v[0] + k)

    def poll(self):
        it = [self.jobs[i][0] if i in self.jobs else -1 for i in range(self.max_jobs)]
        return it, [0] * self.max_jobs

    def get_y(self, j):
        return _Y(4)

    def remove(self, j):
        del self.jobs[j]

    def set_tuning(self, t):
        pass

    def close(self):
        pass


def make_requests(sizes, arrivals, s_list, n_iter):
    from paper_1712_09005_gb300 import Schedule
    from paper_1712_09005_gb300.serve import Request
    out = []
    for i, (N, a, s) in enumerate(zip(sizes, arrivals, s_list)):
        rp = np.zeros(N + 1, np.int32)
        out.append(Request(i, float(a), s, rp, np.zeros(0, np.int32), np.zeros(0, np.float32),
                           np.zeros((N, s), np.float32), Schedule(n_iter=n_iter)))
    return out


def test_admission_respects_budget_and_arrival_order():
    from paper_1712_09005_gb300.serve import Server
    sizes = [1000, 5000, 800, 3000, 4000, 600, 2000]
    reqs = make_requests(sizes, np.arange(len(sizes)) * 0.001, [2, 2, 1, 2, 1, 2, 2], 50)
    peak = []
    srv = Server(budget_bytes=700_000, iters_per_round=10,
                 batch_factory=lambda s: FakeBatch(s, max_jobs=2))
    orig = srv.admit

    def admit(req, now):
        orig(req, now)
        peak.append(srv.used)
        assert srv.used <= srv.budget

    srv.admit = admit
    out = srv.serve(reqs, time_scale=1.0)
    assert sorted(r.rid for r in out["results"]) == list(range(len(sizes)))
    # admitted in arrival order (no request overtakes the head of the queue)
    assert srv.admission_order == list(range(len(sizes)))
    assert max(peak) <= 700_000 and srv.used == 0
    assert out["p50_s"] >= 0 and out["p99_s"] >= out["p50_s"]
    assert out["embeddings_per_s"] > 0


def test_slots_limit_resident_jobs():
    from paper_1712_09005_gb300.serve import Server
    reqs = make_requests([10] * 6, [0.0] * 6, [2] * 6, 30)
    srv = Server(budget_bytes=10 ** 9, iters_per_round=10,
                 batch_factory=lambda s: FakeBatch(s, max_jobs=2))
    seen = []
    orig = srv.step

    def step():
        seen.append(sum(1 for (s, _) in srv.resident if s == 2))
        orig()

    srv.step = step
    out = srv.serve(reqs)
    assert len(out["results"]) == 6
    assert max(seen) == 2


def test_oversized_request_is_rejected():
    from paper_1712_09005_gb300.serve import Server
    reqs = make_requests([10_000], [0.0], [2], 10)
    srv = Server(budget_bytes=1000, batch_factory=lambda s: FakeBatch(s))
    with pytest.raises(ValueError):
        srv.serve(reqs)


def test_poisson_arrivals_rate():
    from paper_1712_09005_gb300.serve import poisson_arrivals
    t = poisson_arrivals(4000, 4.0, seed=5)
    assert np.all(np.diff(t) > 0)
    assert abs(4000 / t[-1] - 4.0) < 0.3
