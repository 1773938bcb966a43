"""Batched iterations of many jobs (one launch per phase for every job, one
CUDA graph per iteration) against the single-job path and the FP64 oracle.

A job's arithmetic does not depend on the other jobs of its table (no kernel
mixes values of different jobs, every reduction has a fixed order), so the
batch must reproduce a plan run of the same job BITWISE at the same tuning
(the plan without locality relabelling). The single-job path itself is held
to the oracle by test_gpu_parity.py; the first step of every batched job is
also checked against the oracle's step here (dY tolerance 1e-5).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


_CACHE = {}


def job(N, seed, s):
    key = (N, seed, s)
    if key not in _CACHE:
        X = inputs.mixture(N=N, n_clusters=5, seed=seed)
        P = inputs.affinities(X, 20.0, device="cpu")
        Y0 = inputs.initial_embedding(N, s, seed=seed)
        _CACHE[key] = (P, Y0)
    return _CACHE[key]


def plan_run(P, Y0, s, sched, n_intervals=0):
    with pkg.Plan(P.N, s, n_intervals=n_intervals, relabel_first=-1) as plan:
        Y = torch.as_tensor(Y0.copy(), device="cuda")
        plan.run(pkg.DeviceCSR.from_host(*P.as_tuple()), Y, sched, want_kl=False)
        torch.cuda.synchronize()
        assert plan.status() == 0
        return Y.cpu().numpy()


SIZES = [(1100, 1), (2503, 2), (700, 3), (4001, 4), (1537, 5)]


@pytest.mark.parametrize("s", [1, 2])
def test_batch_equals_plan_bitwise(s):
    sched = pkg.Schedule(n_iter=40, early_iters=20)
    with pkg.Batch(s, max_jobs=8) as b:
        ids = {}
        for N, seed in SIZES:
            P, Y0 = job(N, seed, s)
            ids[(N, seed)] = b.add(pkg.DeviceCSR.from_host(*P.as_tuple()),
                                   torch.as_tensor(Y0, device="cuda"), sched)
        b.iterate(40)
        it, st = b.poll()
        for (N, seed), jid in ids.items():
            assert it[jid] == 40 and st[jid] == 0
            got = b.get_y(jid).cpu().numpy()
            P, Y0 = job(N, seed, s)
            want = plan_run(P, Y0, s, sched)
            assert np.array_equal(got, want), (N, seed)


def test_first_step_matches_oracle():
    s = 2
    sched = pkg.Schedule(n_iter=10)
    with pkg.Batch(s, max_jobs=4) as b:
        ids = []
        for N, seed in SIZES[:3]:
            P, Y0 = job(N, seed, s)
            # a spread-out start so the step is a real gradient step
            Ys = (Y0 * 1000.0).astype(np.float32)
            ids.append((b.add(pkg.DeviceCSR.from_host(*P.as_tuple()), torch.as_tensor(Ys, device="cuda"),
                              sched), P, Ys))
        b.iterate(1)
        for jid, P, Ys in ids:
            got = b.get_y(jid).cpu().numpy().astype(np.float64)
            ref = oracle.interp_gradient(Ys.astype(np.float64), P.as_tuple(), alpha=12.0,
                                         opts=oracle.InterpOptions(p=3, n_min=50, n_int_max=400))
            Yo = Ys.astype(np.float64).copy()
            uo = np.zeros_like(Yo)
            go = np.ones_like(Yo)
            oracle.step(Yo, uo, go, ref["dY"], oracle.Schedule(n_iter=10), 0)
            # one step moves Y by lr * gain * dY; the gradient tolerance bounds the difference
            step = np.linalg.norm(200.0 * go * ref["dY"])
            assert np.linalg.norm(got - Yo) <= 2e-5 * step + 1e-6 * np.linalg.norm(Yo)


def test_jobs_join_and_finish_at_different_times():
    """Continuous batching: a job added while others are mid-run, jobs with
    different lengths; each result equals its run alone."""
    s = 2
    sched_a = pkg.Schedule(n_iter=30, early_iters=10)
    sched_b = pkg.Schedule(n_iter=12, early_iters=5)
    with pkg.Batch(s, max_jobs=4) as b:
        Pa, Ya = job(2503, 2, s)
        Pb, Yb = job(1100, 1, s)
        Pc, Yc = job(700, 3, s)
        ja = b.add(pkg.DeviceCSR.from_host(*Pa.as_tuple()), torch.as_tensor(Ya, device="cuda"), sched_a)
        b.iterate(7)
        jb = b.add(pkg.DeviceCSR.from_host(*Pb.as_tuple()), torch.as_tensor(Yb, device="cuda"), sched_b)
        b.iterate(5)
        jc = b.add(pkg.DeviceCSR.from_host(*Pc.as_tuple()), torch.as_tensor(Yc, device="cuda"), sched_a)
        b.iterate(40)  # more than anyone needs: finished jobs stop
        it, st = b.poll()
        assert (it[ja], it[jb], it[jc]) == (30, 12, 30)
        ya, yb, yc = (b.get_y(j).cpu().numpy() for j in (ja, jb, jc))
        b.remove(jb)
        assert b.poll()[0][jb] == -1
    assert np.array_equal(ya, plan_run(Pa, Ya, s, sched_a))
    assert np.array_equal(yb, plan_run(Pb, Yb, s, sched_b))
    assert np.array_equal(yc, plan_run(Pc, Yc, s, sched_a))


def test_graph_and_plain_launches_agree():
    s = 2
    sched = pkg.Schedule(n_iter=15)
    out = []
    for use_graph in (True, False):
        with pkg.Batch(s, max_jobs=4, use_graph=use_graph) as b:
            js = []
            for N, seed in SIZES[:3]:
                P, Y0 = job(N, seed, s)
                js.append(b.add(pkg.DeviceCSR.from_host(*P.as_tuple()), torch.as_tensor(Y0, device="cuda"), sched))
            b.iterate(15)
            out.append([b.get_y(j).cpu().numpy() for j in js])
            launches = b.launch_count()
            assert launches >= 15 * 10
    for a, c in zip(*out):
        assert np.array_equal(a, c)


def test_autotune_restores_state_and_tuning_is_applied():
    s = 2
    sched = pkg.Schedule(n_iter=25)
    res = []
    tuned = None
    for mode in ("autotune", "set"):
        with pkg.Batch(s, max_jobs=4) as b:
            js = []
            for N, seed in SIZES[:4]:
                P, Y0 = job(N, seed, s)
                js.append(b.add(pkg.DeviceCSR.from_host(*P.as_tuple()), torch.as_tensor(Y0, device="cuda"), sched))
            b.iterate(3)
            if mode == "autotune":
                tuned = b.autotune(iters=2)
                assert tuned.chunk in (32, 64, 128, 256)
                assert tuned.fft_threads in (0, 256, 512, 1024)
                assert tuned.ms_per_iter > 0
                assert b.poll()[0][js[0]] == 3  # the trials left no trace
            else:
                b.set_tuning(pkg.Tuning(tuned.chunk, tuned.fft_threads, tuned.n_int_policy))
            b.iterate(22)
            res.append([b.get_y(j).cpu().numpy() for j in js])
    for a, c in zip(*res):
        assert np.array_equal(a, c)


def test_fill_policy_keeps_at_least_the_rule_and_matches_oracle():
    """TSNE_NINT_FILL takes more intervals at the same FFT length: the gradient
    still matches the oracle evaluated with that interval count."""
    s = 2
    N, seed = 2503, 2
    P, Y0 = job(N, seed, s)
    Ys = (Y0 * 3000.0).astype(np.float32)  # width ~ 150: rule gives 150 intervals
    sched = pkg.Schedule(n_iter=5, early_iters=0)
    with pkg.Batch(s, max_jobs=2) as b:
        b.set_tuning(pkg.Tuning(128, 0, pkg._abi.TSNE_NINT_FILL))
        j = b.add(pkg.DeviceCSR.from_host(*P.as_tuple()), torch.as_tensor(Ys, device="cuda"), sched)
        b.iterate(1)
        got = b.get_y(j).cpu().numpy().astype(np.float64)
    box = oracle.box(Ys.astype(np.float64), oracle.InterpOptions(p=3, n_min=50, n_int_max=400))
    rule = box.n_int
    # the FFT length of the rule's node count: the first even 5-smooth L >= 6 rule
    def smooth(x):
        for f in (2, 3, 5):
            while x % f == 0:
                x //= f
        return x == 1
    L = next(x for x in range(6 * rule, 10 * rule) if x % 2 == 0 and smooth(x))
    fill = min(400, L // 6)
    assert fill >= rule
    ref = oracle.interp_gradient(Ys.astype(np.float64), P.as_tuple(), alpha=1.0,
                                 opts=oracle.InterpOptions(p=3, n_int_fixed=fill))
    Yo = Ys.astype(np.float64).copy()
    uo, go = np.zeros_like(Yo), np.ones_like(Yo)
    oracle.step(Yo, uo, go, ref["dY"], oracle.Schedule(n_iter=5, early_iters=0), 0)
    step = np.linalg.norm(200.0 * go * ref["dY"])
    assert np.linalg.norm(got - Yo) <= 2e-5 * step + 1e-6 * np.linalg.norm(Yo)


def test_batch_kl_and_capacity():
    s = 2
    sched = pkg.Schedule(n_iter=20)
    P, Y0 = job(2503, 2, s)
    with pkg.Batch(s, max_jobs=2) as b:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        j0 = b.add(Pd, torch.as_tensor(Y0, device="cuda"), sched)
        j1 = b.add(Pd, torch.as_tensor(Y0, device="cuda"), sched)
        with pytest.raises(pkg.TsneError) as e:
            b.add(Pd, torch.as_tensor(Y0, device="cuda"), sched)
        assert e.value.code == pkg._abi.TSNE_ERR_CAPACITY
        assert b.bytes_in_use() == 2 * b.job_bytes(2503)
        b.iterate(20)
        y = b.get_y(j0)
        kl = b.kl(j0)
        with pkg.Plan(2503, s) as plan:
            want = plan.kl(Pd, y)
        assert kl == want
        b.remove(j1)
        assert b.bytes_in_use() == b.job_bytes(2503)
        j2 = b.add(Pd, torch.as_tensor(Y0, device="cuda"), sched)
        assert j2 == j1


def test_tuning_knobs_do_not_change_results():
    """The spread's integer sums, the FFT's per-element arithmetic and Z's
    fixed-order Parseval sum make a job's result independent of the spread
    work-item size and the FFT passes' CTA size (only the interval policy
    changes the approximation)."""
    s = 2
    sched = pkg.Schedule(n_iter=12)
    res = []
    for chunk, thr in ((128, 0), (32, 1024), (256, 256), (64, 512)):
        with pkg.Batch(s, max_jobs=4) as b:
            b.set_tuning(pkg.Tuning(chunk, thr, pkg._abi.TSNE_NINT_RULE))
            js = []
            for N, seed in SIZES[:3]:
                P, Y0 = job(N, seed, s)
                js.append(b.add(pkg.DeviceCSR.from_host(*P.as_tuple()), torch.as_tensor(Y0 * 500.0, device="cuda"), sched))
            b.iterate(12)
            res.append([b.get_y(j).cpu().numpy() for j in js])
    for other in res[1:]:
        for a, c in zip(res[0], other):
            assert np.array_equal(a, c)
