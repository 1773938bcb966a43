"""Benchmark of the GB300 FIt-SNE gradient step: point-iterations/s.

One "step" is one iteration of t-SNE gradient descent through the C ABI
(bounding box, counting sort, spread, FFT convolution, Z, attraction +
interpolation + gains/momentum update) on N points. By default the timed
region is the whole 1000-iteration job of the N = 1,000,000, s = 2 workload
(50-d Gaussian mixture with 100 clusters + 5% uniform background, perplexity
30, exact k = 90 kNN affinities), starting from Y0; warm-up iterations run
first on a scratch copy of the same job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload n1m_2d|n1m_1d|n100k_2d|n2k_2d|served|affinity|heatmap]

The same JSON line also carries two sub-measurements of the batched forms:
  "batched": 64 independent jobs (N log-uniform in [1k, 200k], s = 2, 1000
             iterations each), run as one batch (one launch per phase for
             all jobs, one CUDA graph per iteration, autotuned) and as a plain
             one-plan-at-a-time loop: embeddings/s of both and the largest
             relative difference of the jobs' final KL.
  "served":  a bounded sample (the first jobs) of the served stream: Poisson
             arrivals at 4/s, N log-uniform in [500, 500k], s in {1, 2},
             perplexity in {10, 30, 50}, 1000 iterations each, admitted
             under a 40 GB HBM budget; p50/p99 latency and embeddings/s.
             --workload served runs the whole 500-job stream instead.
--workload affinity times the GPU construction of P itself (exact kNN,
bandwidths, symmetrisation) for the N = 1M, D = 50 mixture.
--workload heatmap times the t-SNE heatmaps of Sec. 5 (bins of a 1-D
embedding, gene x bin sums, nearest genes) on a synthetic 50,000-cell x
25,000-gene count matrix.

Under torchrun each rank runs its own independent job (its own seed): the
method shards by job with no data-path exchange, so scaling is weak and
value = all ranks' point-iterations / the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores instead
(rank 0 only; a bounded number of iterations of the same job).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "point-iterations/s (FIt-SNE gradient, N=1M, 2D)"
UNIT = "point-iterations/s"

WORKLOADS = {
    # name: (workload number, N, s, fixed intervals, schedule overrides, description)
    "n1m_2d": (3, 1_000_000, 2, 0, dict(late_iters=250, late_alpha=4.0),
               "N=1,000,000 50-d Gaussian mixture (100 equal clusters + 5% uniform background), "
               "perplexity 30, exact kNN k=90, symmetrised CSR fp32 P; s=2, p=3, "
               "N_int=max(50, ceil(width)) capped at 400; 1000-iteration schedule: "
               "exaggeration 12 for 250, late exaggeration 4 over the final 250, lr 200"),
    "n1m_1d": (3, 1_000_000, 1, 0, dict(late_iters=250, late_alpha=4.0),
               "N=1,000,000 mixture as n1m_2d; s=1, p=3, N_int=max(50, ceil(width)) capped at 1000"),
    "n100k_2d": (2, 100_000, 2, 0, {},
                 "N=100,000 50-d Gaussian mixture, 30 clusters of Dirichlet(1) sizes, perplexity 30, "
                 "k=90; s=2, p=3, N_int=max(50, ceil(width)); 1000 iterations"),
    "n2k_2d": (1, 2000, 2, 50, {},
               "N=2,000 50-d Gaussian mixture, 10 clusters, perplexity 30, k=90; s=2, p=3, "
               "50 intervals; 1000 iterations"),
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(v: float) -> float:
    """The largest v over the ranks of the process group (v itself alone).
    The replicas exchange only this scalar (and barriers): no data path."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, N: int, K: int, seconds_max: float) -> float:
    """Point-iterations/s of the whole job: every rank runs its own N-point job
    for K iterations (weak scaling), timed by the slowest rank."""
    return world * N * K / seconds_max


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def force_traffic(s: int, N: int):
    """DRAM bytes per force-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "force_kernel_n1m.txt")
    src = os.path.join(ROOT, "paper_1712_09005_gb300", "csrc", "fitsne_kernels.cu")
    try:
        lines = open(path).read().splitlines()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    rec = {}
    for ln in lines:
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_source_sha1") != sha or rec.get(f"dram_bytes_per_launch_s{s}_N{N}") is None:
        return None
    return float(rec[f"dram_bytes_per_launch_s{s}_N{N}"])


def make_inputs(wl: str, job: int, device: str, N: int):
    from paper_1712_09005_gb300 import inputs
    num, _, s, fixed, over, desc = WORKLOADS[wl]
    args = inputs.mixture_args(num, job=job, N=N)
    X = inputs.mixture(**args)
    P = inputs.affinities(X, 30.0, device=device)
    Y0 = inputs.initial_embedding(N, s, seed=args["seed"])
    if device != "cpu":
        import torch
        torch.cuda.empty_cache()  # release the kNN scratch
    return P, Y0


def schedule(wl: str, n_iter: int):
    import paper_1712_09005_gb300 as pkg
    over = WORKLOADS[wl][4]
    return pkg.Schedule(n_iter=n_iter, **over)


def oracle_iterations(P, Y0, wl, sched_args, budget_s, max_iters):
    """Times the FP64 oracle (gradient + update) from Y0 for up to budget_s."""
    import oracle
    num, _, s, fixed, over, desc = WORKLOADS[wl]
    opts = oracle.InterpOptions(p=3, n_int_fixed=fixed, n_min=50,
                                n_int_max=400 if s == 2 else 1000, use_fft=True)
    sc = oracle.Schedule(**sched_args)
    Y = Y0.astype(np.float64).copy()
    uY = np.zeros_like(Y)
    g = np.ones_like(Y)
    Pt = P.as_tuple()
    it = 0
    t0 = time.perf_counter()
    while it < max_iters:
        out = oracle.interp_gradient(Y, Pt, alpha=oracle.alpha_at(sc, it), opts=opts)
        oracle.step(Y, uY, g, out["dY"], sc, it)
        it += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return it, dt, oracle.num_threads()


def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    num, N, s, fixed, over, desc = WORKLOADS[a.workload]
    if a.n:
        N = a.n
        desc = f"{desc} [N overridden to {N}]"
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    P, Y0 = make_inputs(a.workload, 0, dev, N)
    sched_args = dict(n_iter=max(1000, a.steps), **over)
    # W warm-up iterations, then a bounded number of timed iterations
    if a.warmup > 0:
        oracle_iterations(P, Y0, a.workload, sched_args, 1e9, a.warmup)
    iters, dt, cores = oracle_iterations(P, Y0, a.workload, sched_args, a.ref_budget, a.steps)
    value = N * iters / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": iters, "warmup": a.warmup, "ms_per_step": 1e3 * dt / iters,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "N": N, "nnz": int(P.nnz), "s": s,
                                        "iterations": [0, iters]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{iters} oracle iterations (interpolated gradient in FP64 "
                                   f"with its radix-2 FFT, plus the update) of this job from Y0"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_jobs(n_jobs: int, seed: int = 4000):
    """Workload 4: n_jobs mixtures (10-30 clusters, Dirichlet sizes), N
    log-uniform in [1k, 200k], perplexity 30, k = 90, Y0 ~ N(0, 1e-4)."""
    import torch
    from paper_1712_09005_gb300 import inputs
    sizes = inputs.log_uniform_sizes(n_jobs, 1000, 200_000, seed=seed)
    jobs = []
    for j, N in enumerate(sizes):
        args = inputs.mixture_args(4, job=j, N=int(N))
        P = inputs.affinities(inputs.mixture(**args), 30.0, device="cuda")
        jobs.append((P, inputs.initial_embedding(int(N), 2, seed=args["seed"])))
    torch.cuda.empty_cache()
    return jobs


def run_batched_compare(n_jobs: int, n_iter: int):
    """Embeddings/s of one batch vs a plain loop of plans, same jobs, same schedule."""
    import torch
    import paper_1712_09005_gb300 as pkg
    jobs = batched_jobs(n_jobs)
    sched = pkg.Schedule(n_iter=n_iter)
    Pds = [pkg.DeviceCSR.from_host(*P.as_tuple()) for P, _ in jobs]
    # a plain one-job-at-a-time loop: one plan per job (allocated before the clock)
    plans = [pkg.Plan(P.N, 2) for P, _ in jobs]
    Ys = [torch.as_tensor(Y0.copy(), device="cuda") for _, Y0 in jobs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for plan, Pd, Y in zip(plans, Pds, Ys):
        plan.run(Pd, Y, sched, want_kl=False)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    kl_seq = [plan.kl(Pd, Y) for plan, Pd, Y in zip(plans, Pds, Ys)]
    launches_seq = sum(pl.launch_count() for pl in plans)
    for pl in plans:
        pl.close()
    del plans, Ys
    torch.cuda.empty_cache()
    def batched_run(tuning):
        with pkg.Batch(2, max_jobs=max(64, n_jobs)) as b:
            ids = [b.add(Pd, torch.as_tensor(Y0, device="cuda"), sched) for Pd, (_, Y0) in zip(Pds, jobs)]
            if tuning is None:
                tuning = b.autotune(iters=3)  # restores every job's state afterwards
                picked = tuning
            else:
                b.set_tuning(tuning)
                picked = None
            b.poll()
            l0 = b.launch_count()
            t0 = time.perf_counter()
            b.iterate(n_iter)
            it, st = b.poll()
            dt = time.perf_counter() - t0
            launches = b.launch_count() - l0
            assert all(it[j] == n_iter and st[j] == 0 for j in ids)
            kls = [b.kl(j) for j in ids]
        return dt, kls, launches, picked

    # the autotuner's pick (chunk, FFT threads; the plans' interval rule):
    # the batch computes exactly what the loop of plans computes
    t_bat, kl_bat, launches_bat, tuning = batched_run(None)
    rel = [abs(x - y) / abs(y) for x, y in zip(kl_bat, kl_seq)]
    sumN = int(sum(P.N for P, _ in jobs))
    return {
        "jobs": n_jobs, "sum_N": sumN, "iterations": n_iter, "s": 2,
        "embeddings_per_s": n_jobs / t_bat,
        "sequential_embeddings_per_s": n_jobs / t_seq,
        "speedup": t_seq / t_bat,
        "point_iterations_per_s": sumN * n_iter / t_bat,
        "kl_max_rel_diff": max(rel), "kl_mean": float(np.mean(kl_bat)),
        "tuning": {"chunk": tuning.chunk, "fft_threads": tuning.fft_threads,
                   "n_int_policy": "rule", "ms_per_iter": tuning.ms_per_iter,
                   "note": "the autotuner's pick, timed after the tuning (its trials excluded)"},
        "gpu_launches_batched": launches_bat, "gpu_launches_sequential": launches_seq,
        "timing": "wall clock around the whole runs, device synchronised",
        "workload": "N log-uniform in [1k, 200k], 10-30-cluster Gaussian mixtures in 50-d, "
                    "perplexity 30, k=90; one batch (graph per iteration, autotuned chunk and FFT "
                    "threads, the plans' interval rule) vs a loop of plans",
    }


def served_requests(n_take: int, n_stream: int = 500, seed: int = 5000):
    """Workload 5: a Poisson stream (4/s) of n_stream jobs, N log-uniform in
    [500, 500k], s in {1, 2}, perplexity in {10, 30, 50}, 1000 iterations;
    the first n_take requests with their P built (P is ready on arrival)."""
    import paper_1712_09005_gb300 as pkg
    from paper_1712_09005_gb300 import inputs
    from paper_1712_09005_gb300.serve import Request, poisson_arrivals
    sizes = inputs.log_uniform_sizes(n_stream, 500, 500_000, seed=seed)
    arr = poisson_arrivals(n_stream, 4.0, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    s_of = rng.integers(1, 3, size=n_stream)
    perp_of = rng.choice([10.0, 30.0, 50.0], size=n_stream)
    out = []
    for i in range(n_take):
        N = int(sizes[i])
        args = inputs.mixture_args(5, job=i, N=N)
        P = inputs.affinities(inputs.mixture(**args), float(perp_of[i]), device="cuda")
        Y0 = inputs.initial_embedding(N, int(s_of[i]), seed=args["seed"])
        out.append(Request(i, float(arr[i]), int(s_of[i]), P.row_ptr, P.col, P.val, Y0,
                           pkg.Schedule(n_iter=1000)))
    import torch
    torch.cuda.empty_cache()
    return out


def run_served(n_take: int, n_stream: int = 500):
    from paper_1712_09005_gb300.serve import Server
    reqs = served_requests(n_take, n_stream)
    srv = Server(budget_bytes=40 * 10 ** 9, max_jobs=64, iters_per_round=25)
    try:
        out = srv.serve(reqs)
    finally:
        srv.close()
    res = out["results"]
    ok = sum(1 for r in res if r.status == 0)
    return {
        "jobs": len(res), "ok": ok, "p50_latency_s": out["p50_s"], "p99_latency_s": out["p99_s"],
        "embeddings_per_s": out["embeddings_per_s"], "makespan_s": out["makespan_s"],
        "peak_resident_bytes": out["peak_bytes"], "budget_bytes": 40 * 10 ** 9,
        "point_iterations": int(sum(r.N for r in res)) * 1000,
        "sample": (f"the first {n_take} of the {n_stream}-job stream" if n_take < n_stream
                   else f"the whole {n_stream}-job stream"),
        "workload": "Poisson arrivals 4/s, N log-uniform [500, 500k], s in {1,2}, perplexity "
                    "{10,30,50}, 1000 iterations, 40 GB budget; latency = arrival to "
                    "embedding in host memory",
    }


def run_served_saturated(n_take: int):
    """The served form against a plain one-job-at-a-time loop on the same
    requests, all present at t = 0 (the server is never idle waiting for
    arrivals): embeddings/s of both and the jobs' final KL agreement."""
    import dataclasses
    import torch
    import paper_1712_09005_gb300 as pkg
    from paper_1712_09005_gb300.serve import Server
    reqs = [dataclasses.replace(r, arrival=0.0) for r in served_requests(n_take)]
    srv = Server(budget_bytes=40 * 10 ** 9, max_jobs=64, iters_per_round=25)
    try:
        out = srv.serve(reqs)
    finally:
        srv.close()
    t_srv = out["makespan_s"]
    served_Y = {r.rid: r.Y for r in out["results"]}
    # one job at a time: upload P and Y0, create the job's plan, run it, read Y back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_Y = {}
    for r in reqs:
        Pd = pkg.DeviceCSR.from_host(r.row_ptr, r.col, r.val)
        Y = torch.as_tensor(r.Y0, device="cuda")
        with pkg.Plan(r.N, r.s) as plan:
            plan.run(Pd, Y, r.sched, want_kl=False)
            seq_Y[r.rid] = Y.cpu().numpy()
    t_seq = time.perf_counter() - t0
    # final KL of both results of every job (a plan evaluates both)
    rel = []
    for r in reqs:
        Pd = pkg.DeviceCSR.from_host(r.row_ptr, r.col, r.val)
        with pkg.Plan(r.N, r.s) as plan:
            k_srv = plan.kl(Pd, torch.as_tensor(served_Y[r.rid], device="cuda"))
            k_seq = plan.kl(Pd, torch.as_tensor(seq_Y[r.rid], device="cuda"))
        rel.append(abs(k_srv - k_seq) / abs(k_seq))
    return {"jobs": len(reqs), "ok": sum(1 for x in out["results"] if x.status == 0),
            "embeddings_per_s": len(reqs) / t_srv, "sequential_embeddings_per_s": len(reqs) / t_seq,
            "speedup": t_seq / t_srv, "kl_max_rel_diff": max(rel),
            "p50_latency_s": out["p50_s"], "p99_latency_s": out["p99_s"],
            "timing": "wall clock; the server from the first admission to the last result in host "
                      "memory, the loop from the first upload to the last result in host memory "
                      "(plan creation, P upload and Y read-back inside both)",
            "workload": f"the first {len(reqs)} requests of the served stream, all arriving at t = 0"}


def run_ours(a):
    import torch
    import paper_1712_09005_gb300 as pkg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1712_09005_gb300 import build as pbuild
    pbuild.build()
    num, N, s, fixed, over, desc = WORKLOADS[a.workload]
    N = a.n or N
    if a.n:
        desc = f"{desc} [N overridden to {N}]"
    K, W = a.steps, a.warmup
    n_iter = max(1000, K)
    sched = schedule(a.workload, n_iter)

    P, Y0 = make_inputs(a.workload, rank, "cuda", N)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    stream = torch.cuda.current_stream()
    plan = pkg.Plan(N, s, n_intervals=fixed, stream=stream.cuda_stream, force_mode=a.force_mode,
                    order_rounds=-1 if a.no_graph_order else a.order_rounds,
                    relabel_first=a.relabel_first)

    # one-time analysis of P (not per iteration): the graph order the run
    # starts in and the copy of P in that order, timed and reported as setup
    order_ms = None
    if not a.no_graph_order:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.order(Pd)
        e1.record(stream)
        torch.cuda.synchronize()
        order_ms = e0.elapsed_time(e1)

    # warm-up on a scratch copy of the job
    Yw = torch.as_tensor(Y0.copy(), device="cuda")
    plan.run_reset()
    if W > 0:
        plan.run_iters(Pd, Yw, sched, 0, W)
    torch.cuda.synchronize()

    # timed: iterations 0 .. K-1 of the job from Y0 (steady-state steps
    # replay the plan's step graph; no per-phase events in this pass)
    Y = torch.as_tensor(Y0.copy(), device="cuda")
    plan.run_reset()
    plan.profile(False)
    launches0 = plan.launch_count()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    plan.run_iters(Pd, Y, sched, 0, K)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = plan.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    info = plan.info()
    status = plan.status()
    if status != 0:
        raise RuntimeError(f"device status {status} after the timed run")
    # the same K iterations again with CUDA events around every phase on the
    # plan's stream (plain launches): the per-phase times and the force
    # kernel's duration for the roofline
    Yp = torch.as_tensor(Y0.copy(), device="cuda")
    plan.run_reset()
    plan.profile(True)
    plan.profile_read()
    plan.run_iters(Pd, Yp, sched, 0, K)
    prof = plan.profile_read()
    plan.profile(False)
    del Yp
    ms_max = max_over_ranks(ms)
    value = whole_job_rate(world, N, K, ms_max / 1e3)

    # roofline of the dominant kernel: attraction + interpolation + update
    n = info["n"]
    grid_bytes = 16 * (n ** s)
    bytes_force = 8 * P.nnz + 4 * (N + 1) + 24 * s * N + grid_bytes
    force_ms = prof["ms"]["force"] / max(1, prof["evals"])
    achieved = bytes_force / (force_ms / 1e3) / 1e9
    peak, peak_kind = peak_hbm()
    traffic = force_traffic(s, N)

    # the whole iteration against the same roofline (every kernel of a step):
    # 8 nnz + 4 (N + 1) + 24 s N + 8 (s + 5) n^s bytes (for s = 2: 56 n^2;
    # s = 1: 40 n; the grids are written and read once each)
    bytes_iter = 8 * P.nnz + 4 * (N + 1) + 24 * s * N + 8 * (s + 5) * (n ** s)
    iter_achieved = bytes_iter / (ms_max / K / 1e3) / 1e9

    # the whole job (iterations 0 .. n_iter - 1 from Y0, embedding
    # relabellings included) on the same plan, when the timed window is shorter
    full_job = None
    if K < n_iter and not a.no_full_job:
        Yf = torch.as_tensor(Y0.copy(), device="cuda")
        plan.run_reset()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        plan.run_iters(Pd, Yf, sched, 0, n_iter)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        finfo = plan.info()
        if plan.status() != 0:
            raise RuntimeError("device status after the full job")
        Yf = torch.as_tensor(Y0.copy(), device="cuda")  # phases of the whole job (events, plain launches)
        plan.run_reset()
        plan.profile(True)
        plan.profile_read()
        plan.run_iters(Pd, Yf, sched, 0, n_iter)
        fprof = plan.profile_read()
        plan.profile(False)
        full_job = {"iterations": [0, n_iter], "value": N * n_iter / (fms / 1e3), "unit": UNIT,
                    "ms_per_step": fms / n_iter,
                    "phases_ms_per_iter": {k: v / max(1, fprof["evals"]) for k, v in fprof["ms"].items()},
                    "final_n_int": finfo["n_int"], "final_fft_len": finfo["fft_len"],
                    "note": "the same job from Y0 over its whole schedule, CUDA events on the plan's "
                            "stream around the run; starts in the order prepared before the timed "
                            "region; phases from a second run with per-phase events"}
        del Yf

    # end to end through the C ABI with host buffers (pinned): upload P and
    # Y0, K iterations, download Y (the graph order of P is computed inside)
    e2e = None
    if not a.no_e2e:
        rp = torch.from_numpy(P.row_ptr).pin_memory()
        cl = torch.from_numpy(P.col).pin_memory()
        vl = torch.from_numpy(P.val).pin_memory()
        Yh = torch.from_numpy(Y0.copy()).pin_memory()
        sched_e2e = pkg.Schedule(n_iter=K, **over)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.run_host(rp.numpy(), cl.numpy(), vl.numpy(), Yh.numpy(), sched_e2e, want_kl=False)
        dt = max_over_ranks(time.perf_counter() - t0)
        h2d = 4 * (N + 1) + 8 * P.nnz + 4 * N * s
        d2h = 4 * N * s
        e2e = {"value": whole_job_rate(world, N, K, dt), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K,
               "note": "one tsne_run_host call: P and Y0 uploaded once, Y downloaded once; "
                       "bytes per step = call totals / K"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        oracle.build()
        it, dt, cores = oracle_iterations(P, Y0, a.workload, dict(n_iter=n_iter, **over),
                                          a.cpu_seconds, 10 ** 6)
        cpu = {"value": N * it / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{it} oracle iterations (FP64 interpolated gradient with radix-2 FFT + "
                         f"update) of this job from Y0, {dt:.1f} s"}

    batched = served = None
    plan.close()
    del Pd
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not a.no_batched:
        batched = run_batched_compare(a.batched_jobs, 1000)
    if rank == 0 and world == 1 and not a.no_served:
        served = run_served(a.served_jobs)
        served["saturated"] = run_served_saturated(a.served_jobs)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "N": N, "nnz": int(P.nnz), "s": s, "p": 3,
                       "iterations": [0, K], "final_n_int": info["n_int"],
                       "final_fft_len": info["fft_len"],
                       "l2": "inputs larger than L2 (CSR of %.2f GB streamed every iteration)"
                             % ((8 * P.nnz + 4 * (N + 1)) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "force_kernel (attraction + interpolation + update)",
                         "duration": "mean CUDA-event time of the force phase over a second pass of "
                                     "the same K iterations with per-phase events (the timed pass "
                                     "replays a graph)",
                         "algorithmic_bytes_per_launch": bytes_force,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "iteration_roofline": {"bound": "hbm", "achieved": iter_achieved, "peak": peak,
                                   "unit": "GB/s", "frac": iter_achieved / peak,
                                   "algorithmic_bytes_per_step": bytes_iter,
                                   "note": "every kernel of one step: 8 nnz + 4 (N + 1) + 24 s N + "
                                           "8 (s + 5) n^s bytes / ms_per_step"},
            "phases_ms_per_iter": {k: v / max(1, prof["evals"]) for k, v in prof["ms"].items()},
            "setup": {"graph_order_ms": order_ms,
                      "note": "once per P, before the timed region: the graph order a run starts "
                              "in and the copy of P in that order (tsne_plan_order)"},
            "full_job": full_job,
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "batched": batched,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_served_only(a):
    """--workload served: the whole 500-job stream (rank 0 only)."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    from paper_1712_09005_gb300 import build as pbuild
    pbuild.build()
    served = run_served(500)
    line = {"metric": "served p50/p99 latency (FIt-SNE jobs)", "value": served["p99_latency_s"],
            "unit": "s (p99)", "n_gpus": 1, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic", "config": {"workload": served["workload"]}, "served": served}
    print(json.dumps(line), flush=True)
    return 0


def run_affinity(a):
    """--workload affinity: P from X on the GPU (exact kNN k = 90, perplexity
    30, symmetrisation) for the N = 1M, D = 50 mixture of n1m_2d (rank 0 only).
    The roofline line is the kNN's. With the tensor-core kNN (the default at
    this size): 2 N (N - 1) D flops (one multiply-add per pair and
    dimension of the products the distances need) against the TF32 dense
    peak; the kernel issues 3 MMAs per K-step (head and tail terms) over D
    padded to a multiple of 8, so its ceiling is D / (3 * 8 ceil(D / 8)) of
    that peak (0.30 at D = 50). With the FP32-lane kernels: 3 flops
    (subtract, multiply, add) per pair and dimension over N (N - 1) D against
    the FP32 lanes' rate for that mix (152 SMs x 128 lanes x 1.5 flops per
    instruction x the sampled SM clock)."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    from paper_1712_09005_gb300 import build as pbuild
    pbuild.build()
    import paper_1712_09005_gb300 as pkg
    from paper_1712_09005_gb300 import inputs
    N = a.n or 1_000_000
    args = inputs.mixture_args(3, N=N)
    X = inputs.mixture(**args)
    D, k, perp = X.shape[1], 90, 30.0
    Xd = torch.as_tensor(X, device="cuda")
    warm, steps = max(3, a.warmup), a.steps
    sampler = ClockSampler(local)
    with pkg.Affinity(N, D, k) as aff:
        for _ in range(warm):
            aff.compute(Xd, perp)
        phases = []
        launches0 = aff.launch_count()
        sampler.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            P = aff.compute(Xd, perp)  # synchronises (nnz)
            phases.append(aff.phase_ms())
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        launches = aff.launch_count() - launches0
        knn_info = aff.knn_info()
        nnz = P.nnz
        # end to end: X from pinned host memory, P back to pinned host memory
        Xh = torch.from_numpy(X).pin_memory()
        rp_h = torch.empty(N + 1, dtype=torch.int32).pin_memory()
        col_h = torch.empty(2 * N * k, dtype=torch.int32).pin_memory()
        val_h = torch.empty(2 * N * k, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(steps):
            Xd.copy_(Xh, non_blocking=True)
            P = aff.compute(Xd, perp)
            rp_h.copy_(P.row_ptr, non_blocking=True)
            col_h[:P.nnz].copy_(P.col, non_blocking=True)
            val_h[:P.nnz].copy_(P.val, non_blocking=True)
            torch.cuda.synchronize()
        e2e_wall = time.perf_counter() - t1
    ms = {kk: statistics.median(ph[kk] for ph in phases) for kk in phases[0]}
    total_ms = sum(ms.values())
    clk = clocks.get("sm_mhz") or 2070.0
    if knn_info["kernel"] == "tc":
        peak, basis = peak_tensor_tf32()
        achieved = 2.0 * N * (N - 1) * D / (ms["knn"] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_basis": basis + " (TF32 dense)",
                "ceiling_3xtf32": D / (3 * 8 * ((D + 7) // 8))}
    else:
        peak = 152 * 128 * 1.5 * clk * 1e6 / 1e12  # TFLOP/s for the sub + fma mix
        achieved = 3.0 * N * (N - 1) * D / (ms["knn"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_basis": f"152 SMs x 128 FP32 lanes x 1.5 flop/instr x {clk:.0f} MHz (sampled)"}
    line = {"metric": "affinity builds/s (exact kNN k=90, perplexity 30, N=1M, D=50)",
            "value": 1e3 / total_ms, "unit": "builds/s", "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": total_ms, "higher_is_better": True, "dtype": "f32 (kNN), f64 (bandwidths)",
            "data": "synthetic", "config": {"workload": f"N={N} 50-d mixture (100 clusters + 5% background), "
                                                      "k=90, perplexity 30", "l2": "inputs larger than L2"},
            "phases_ms": ms, "nnz": nnz, "wall_s_per_step": wall / steps,
            "knn": knn_info, "roofline": roof,
            "e2e": {"value": steps / e2e_wall, "unit": "builds/s", "h2d_bytes_per_step": X.nbytes,
                    "d2h_bytes_per_step": 4 * (N + 1) + 8 * nnz},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_heatmap(a):
    """--workload heatmap: t-SNE heatmaps (Sec. 5) of N = 50,000 cells and
    G = 25,000 genes (synthetic counts, ~940 expressed genes per cell, a
    clustered 1-D layout), 100 bins, the nearest 4 genes of 3 genes of
    interest (the paper's example). One step = bin + gene x bin sums +
    nearest genes. The roofline line is the binning kernel's: it streams the
    expression CSR once (8 bytes per entry, plus y and row_ptr) and writes H
    (n_bins x G FP64)."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_1712_09005_gb300 import build as pbuild
    pbuild.build()
    import paper_1712_09005_gb300 as pkg
    from paper_1712_09005_gb300 import inputs
    N = a.n or 50_000
    G, n_bins, goi, m = 25_000, 100, [11, 12_345, 24_999], 4
    e = inputs.expression(N, G, mean_genes=1000, n_clusters=20, seed=5000)
    nnz = int(e.row_ptr[-1])
    E = pkg.DeviceCSR.from_host(*e.as_tuple())
    yd = torch.as_tensor(e.y, device="cuda")
    stream = torch.cuda.current_stream()
    warm, steps = max(3, a.warmup), a.steps
    with pkg.Heatmap(n_bins, G, max_goi=len(goi)) as hm:
        H = torch.empty((n_bins, G), dtype=torch.float64, device="cuda")
        for _ in range(warm):
            hm.bin(yd, E, H)
            hm.nearest(H, goi, m)
        launches0 = hm.launch_count()
        sampler = ClockSampler(local)
        sampler.start()
        torch.cuda.synchronize()
        phases = []
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            hm.bin(yd, E, H)  # synchronises (error flags)
            hm.nearest(H, goi, m)
            phases.append(hm.phase_ms())
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1) / steps
        launches = hm.launch_count() - launches0
        # end to end: y and E from pinned host memory, H and the gene lists back
        yh = torch.from_numpy(e.y).pin_memory()
        rph = torch.from_numpy(e.row_ptr).pin_memory()
        colh = torch.from_numpy(e.col).pin_memory()
        valh = torch.from_numpy(e.val).pin_memory()
        Hh = torch.empty((n_bins, G), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            yd.copy_(yh, non_blocking=True)
            E.row_ptr.copy_(rph, non_blocking=True)
            E.col.copy_(colh, non_blocking=True)
            E.val.copy_(valh, non_blocking=True)
            hm.bin(yd, E, H)
            idx, dist = hm.nearest(H, goi, m)
            Hh.copy_(H, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / steps
    ph = {k: statistics.median(p[k] for p in phases) for k in phases[0]}
    bytes_bin = 8 * nnz + 4 * (N + 1) + 4 * N + 8 * n_bins * G
    achieved = bytes_bin / (ph["bin_sums"] * 1e-3) / 1e9
    peak, peak_kind = peak_hbm()
    cpu = None
    if not a.no_cpu_baseline:
        from oracle import heatmap as ohm
        t0 = time.perf_counter()
        Ho, _ = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, G, n_bins)
        ohm.nearest(Ho, goi, m)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "builds/s", "cores": 1, "kind": "oracle",
               "sample": f"one whole build of this workload by the numpy oracle, {dt:.1f} s"}
    line = {"metric": f"t-SNE heatmap builds/s (N={N} cells, G={G} genes, {n_bins} bins, "
                      f"{len(goi)} genes of interest x {m} nearest)",
            "value": 1e3 / ms, "unit": "builds/s", "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bins), f64 (sums, distances)", "data": "synthetic",
            "config": {"workload": f"N={N} cells x G={G} genes synthetic counts (nnz {nnz}), "
                                   f"20-cluster 1-D layout, {n_bins} equal-width bins",
                       "l2": "expression CSR (%.2f GB) larger than L2, streamed every step" % (8 * nnz / 1e9)},
            "phases_ms": ph,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "hm_bin_kernel",
                         "algorithmic_bytes_per_launch": bytes_bin, "peak_source": f"{peak_kind} hbm_gbs"},
            "e2e": {"value": 1.0 / e2e_s, "unit": "builds/s",
                    "h2d_bytes_per_step": 4 * N + 4 * (N + 1) + 8 * nnz,
                    "d2h_bytes_per_step": 8 * n_bins * G + 12 * len(goi) * m},
            "gpu_launches": launches, "cpu_baseline": cpu, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def peak_tensor_tf32():
    """TF32 dense tensor peak: the measured bf16 burst peak times the nominal
    TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s dense)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16_tflops x 1.1/2.25"
    except (OSError, KeyError, ValueError):
        return 1900.0 * 1.1 / 2.25, "fallback 1.9 PFLOP/s bf16 x 1.1/2.25"


def run_oocpca(a):
    """--workload oocpca: the paper's oocPCA experiment shape (Sec. 6): a
    random m x n = 1,000,000 x 30,000 rank-50 FP32 matrix (planted singular
    values 100 .. 1), k = 50 components, l = k + 2 random vectors, its = 2
    (the defaults of the paper's experiment). One step = one decomposition
    (its + 2 = 4 passes over A). A sits in device memory (120 GB) for the
    timed value; e2e streams A from pinned host memory in blocks (the
    out-of-core mode) when the host can hold it, else a stated smaller m."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_1712_09005_gb300 import build as pbuild
    pbuild.build()
    import paper_1712_09005_gb300 as pkg
    from paper_1712_09005_gb300 import inputs
    m, n, r, k, its = (a.n or 1_000_000), 30_000, 50, 50, 2
    l = k + 2
    A, sig, _, _ = inputs.low_rank_matrix(m, n, r, seed=6000, device="cuda")
    Om = inputs.omega(n, l, seed=6000).astype(np.float32)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    warm, steps = max(3, a.warmup), a.steps
    with pkg.OocPca(m, n, k, l, its=its, stream=stream.cuda_stream) as p:
        for _ in range(warm):
            U, s_gpu, V = p.run(A, Om)
        launches0 = p.launch_count()
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        phase = {"passes_ms": 0.0, "renormalize_ms": 0.0, "qr_svd_ms": 0.0}
        for _ in range(steps):
            U, s_gpu, V = p.run(A, Om)  # synchronises
            ph = p.phase_ms()
            for key in phase:
                phase[key] += ph[key] / steps
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        sec = ev0.elapsed_time(ev1) / 1e3 / steps
        launches = p.launch_count() - launches0
        passes = ph["passes"]
        s_np = s_gpu.cpu().numpy()
        sigma_err = float(np.abs(s_np - sig[:k]).max() / sig[0])
        # orthonormality and the residual on sampled rows: ||A_S - U_S diag(s) V*||
        Vt = V.double()
        rows = torch.as_tensor(np.random.default_rng(1).choice(m, 2000, replace=False), device="cuda")
        resid = (A[rows].double() - (U[rows].double() * s_gpu) @ Vt.T).norm().item() / A[rows].double().norm().item()
        orth = float((U.double().T @ U.double() - torch.eye(k, device="cuda", dtype=torch.float64)).abs().max())
    del U, V
    bytes_pass = 4.0 * m * n  # A read once per pass (the fused pass)
    pass_s = phase["passes_ms"] / 1e3 / passes
    flops_pass = 2 * 2.0 * m * n * l  # A W and A* Y (algorithmic, l columns)
    peak_bw, bw_kind = peak_hbm()
    peak_tf, tf_kind = peak_tensor_tf32()
    e2e = None
    if not a.no_e2e:
        try:
            avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        except (ValueError, OSError):
            avail = 0
        # pinned host copy of A: at most 40 % of the free host memory
        m_h = m if 4 * m * n <= 0.4 * avail else max(4096, int(0.4 * avail / (4 * n)) // 128 * 128)
        Ah = torch.empty((m_h, n), dtype=torch.float32, pin_memory=True)
        Ah.copy_(A[:m_h])
        del A
        torch.cuda.empty_cache()
        with pkg.OocPca(m_h, n, k, l, its=its, stream=stream.cuda_stream) as p:
            p.run(Ah.numpy(), Om)  # warm-up (allocates the block buffers)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(max(1, steps // 2)):
                U, s_h, V = p.run(Ah.numpy(), Om)
                _ = (U.cpu(), s_h.cpu(), V.cpu())
            dt = (time.perf_counter() - t0) / max(1, steps // 2)
        e2e = {"value": dt * m / m_h, "unit": "s", "h2d_bytes_per_step": 4 * m_h * n * (its + 2) + 4 * n * l,
               "d2h_bytes_per_step": 4 * (m_h + n) * k + 8 * k,
               "note": (f"A ({m_h} x {n} FP32) in pinned host memory streamed in 1 GiB blocks ({its + 2} "
                        "passes), U, sigma, V read back" +
                        (f"; scaled to m = {m} by rows (host memory)" if m_h < m else ""))}
    cpu = None
    if not a.no_cpu_baseline:
        import oracle.oocpca as ooc
        m_c = 20_000
        Ac = inputs.low_rank_matrix(m_c, n, r, seed=6001)[0]
        Omc = inputs.omega(n, l, seed=6001)
        t0 = time.perf_counter()
        ooc.oocpca(Ac, k, its, Omc, b=4096)
        dt = time.perf_counter() - t0
        cpu = {"value": dt * m / m_c, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the FP64 numpy oracle on {m_c} x {n} (rank {r}, k {k}, its {its}) in "
                         f"{dt:.1f} s, scaled to m = {m} by rows (every pass is linear in m)"}
    line = {
        "metric": "oocPCA seconds per decomposition (1,000,000 x 30,000 rank-50, k=50, its=2)",
        "value": sec, "unit": "s", "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": sec * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (3xTF32 tensor)",
        "data": "synthetic",
        "config": {"workload": f"oocpca m={m} n={n} rank={r} k={k} l={l} its={its}, A FP32 in device "
                               f"memory (one block), planted singular values 100..1",
                   "l2": "inputs larger than L2 (A is %.0f GB)" % (4 * m * n / 1e9)},
        "roofline": {"bound": "hbm", "achieved": bytes_pass / pass_s / 1e9, "peak": peak_bw, "unit": "GB/s",
                     "frac": bytes_pass / pass_s / 1e9 / peak_bw, "traffic": None,
                     "kernel": "one pass over A (G1 A W + G2 A* Y, tensor cores)",
                     "algorithmic_bytes_per_pass": bytes_pass, "peak_source": f"{bw_kind} hbm_gbs",
                     "tensor": {"achieved_tflops": flops_pass / pass_s / 1e12, "peak_tflops": peak_tf,
                                "frac": flops_pass / pass_s / 1e12 / peak_tf, "peak_source": tf_kind,
                                "note": "algorithmic FLOPs 4 m n l per pass; the 3xTF32 split issues "
                                        "3 MMAs per product on 64 padded columns"}},
        "phases_ms_per_step": phase, "passes_per_step": passes,
        "accuracy": {"sigma_max_abs_err_over_sigma1": sigma_err, "sampled_row_residual": resid,
                     "U_orthonormality": orth},
        "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
        "paper": "15.9 min at 1 GB of memory ... 8.4 min at 300 GB (Sec. 6; CPU, MKL, FP64)",
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps [1000 iterations; 3 builds for --workload affinity]")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["served", "affinity", "heatmap", "oocpca"],
                    default="n1m_2d")
    ap.add_argument("--n", type=int, default=0, help="override the workload's N (smaller cases for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--force-mode", type=int, default=0,
                    help="force-kernel schedule: 0 auto, 1 grid, 2 region (profiling)")
    ap.add_argument("--no-graph-order", action="store_true",
                    help="runs start in the caller's labels (no graph order of P)")
    ap.add_argument("--order-rounds", type=int, default=0,
                    help="averaging rounds of the graph order (0: the library's default)")
    ap.add_argument("--relabel-first", type=int, default=0,
                    help="first embedding relabelling (0: the library's default, < 0: never)")
    ap.add_argument("--no-full-job", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--batched-jobs", type=int, default=64)
    ap.add_argument("--served-jobs", type=int, default=40,
                    help="requests of the served stream in the default run's sample")
    ap.add_argument("--ref-budget", type=float, default=120.0,
                    help="seconds of oracle iterations the reference arm times")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = {"affinity": 3, "heatmap": 20, "oocpca": 4}.get(a.workload, 1000)
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "served":
        return run_served_only(a)
    if a.workload == "affinity":
        return run_affinity(a)
    if a.workload == "heatmap":
        return run_heatmap(a)
    if a.workload == "oocpca":
        return run_oocpca(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
