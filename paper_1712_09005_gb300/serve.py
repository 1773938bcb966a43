"""Continuous-batching service of embedding jobs on one GPU.

Requests (each an embedding job: affinities P in host CSR, Y0, dimension s,
schedule) arrive over time. The server keeps every admitted job's P, Y,
optimizer state and grid scratch resident on the device inside one batch per
embedding dimension (include/fitsne_gb300.h, tsne_batch_*), admits queued
requests at iteration boundaries while slots and the HBM budget allow,
advances every resident job together (one graph replay per iteration and
batch; the batches of s = 1 and s = 2 run on their own streams, so their
iterations overlap on the device), and retires jobs as they finish. A job's
result does not depend on what else was resident (the kernels never mix
jobs), so it equals the job run alone at the same tuning.

Latency of a request = time from its arrival until its embedding is back in
host memory; the server also reports completed embeddings per second.

This module is host-side scheduling only: every arithmetic step of a job runs
in the library's CUDA kernels.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import Batch, DeviceCSR, Schedule, Tuning


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the stream
    s: int
    row_ptr: np.ndarray            # host CSR (int32, int32, float32)
    col: np.ndarray
    val: np.ndarray
    Y0: np.ndarray                 # host float32 [N, s]
    sched: Schedule
    n_intervals: int = 0

    @property
    def N(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def p_bytes(self) -> int:
        return 4 * len(self.row_ptr) + 8 * len(self.col)


@dataclass
class Result:
    rid: int
    N: int
    s: int
    arrival: float
    admitted: float
    finished: float
    Y: np.ndarray
    status: int

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Resident:
    req: Request
    job: int
    bytes: int
    admitted: float
    P: DeviceCSR
    Y0: torch.Tensor


class Server:
    """Admission under an HBM budget, continuous batching, retirement.

    budget_bytes bounds the device memory of resident jobs: each job counts
    its batch scratch (tsne_batch_job_bytes) plus its P. iters_per_round
    iterations run between two scheduling rounds (admission, completion poll).
    """

    def __init__(self, budget_bytes: int, max_jobs: int = 64, iters_per_round: int = 25,
                 tunings: dict | None = None, p: int = 3, batch_factory=None):
        self.budget = int(budget_bytes)
        self.iters_per_round = iters_per_round
        make = batch_factory or (lambda s: Batch(s, p=p, max_jobs=max_jobs))
        self.batches = {s: make(s) for s in (1, 2)}
        for s, b in self.batches.items():
            if tunings and s in tunings:
                b.set_tuning(tunings[s])
        self.resident: dict[tuple[int, int], _Resident] = {}
        self.used = 0
        self.peak_used = 0
        self.rounds = 0
        self.time_scale = 1.0
        self.admission_order: list[int] = []

    def close(self):
        for b in self.batches.values():
            b.close()

    def job_bytes(self, req: Request) -> int:
        return self.batches[req.s].job_bytes(req.N) + req.p_bytes

    def fits(self, req: Request) -> bool:
        b = self.batches[req.s]
        slots = sum(1 for (s, _) in self.resident if s == req.s)
        return slots < b.max_jobs and self.used + self.job_bytes(req) <= self.budget

    def admit(self, req: Request, now: float):
        b = self.batches[req.s]
        P, Y0 = b.upload(req)
        job = b.add(P, Y0, req.sched, req.n_intervals)
        nb = self.job_bytes(req)
        self.admission_order.append(req.rid)
        self.resident[(req.s, job)] = _Resident(req, job, nb, now, P, Y0)
        self.used += nb
        self.peak_used = max(self.peak_used, self.used)

    def step(self):
        """One round: every batch with resident jobs advances iters_per_round
        iterations (enqueued on both streams before any wait)."""
        for s, b in self.batches.items():
            if any(k[0] == s for k in self.resident):
                b.iterate(self.iters_per_round)
        self.rounds += 1

    def retire(self, now_fn) -> list[Result]:
        """Polls the batches (synchronises them) and returns the finished jobs."""
        out = []
        for s, b in self.batches.items():
            mine = [r for k, r in self.resident.items() if k[0] == s]
            if not mine:
                continue
            iters, status = b.poll()
            for r in mine:
                if iters[r.job] >= r.req.sched.n_iter or status[r.job] != 0:
                    Y = b.get_y(r.job)
                    Yh = Y.cpu().numpy()  # synchronises the copy
                    out.append(Result(r.req.rid, r.req.N, s, r.req.arrival * self.time_scale,
                                      r.admitted, now_fn(), Yh, int(status[r.job])))
                    b.remove(r.job)
                    del self.resident[(s, r.job)]
                    self.used -= r.bytes
        return out

    def serve(self, requests: list[Request], time_scale: float = 1.0) -> dict:
        """Serves a stream of requests arriving at req.arrival * time_scale
        seconds after the call; returns per-request results and summary."""
        for r in requests:
            if self.job_bytes(r) > self.budget:
                raise ValueError(f"request {r.rid} needs {self.job_bytes(r)} bytes, over the budget")
        self.time_scale = time_scale
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[tuple[float, int, Request]] = []
        results: list[Result] = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        k = 0
        while k < len(pending) or queue or self.resident:
            t = now()
            while k < len(pending) and pending[k].arrival * time_scale <= t:
                r = pending[k]
                heapq.heappush(queue, (r.arrival * time_scale, r.rid, r))
                k += 1
            # admission in arrival order while the head fits (no overtaking)
            while queue and self.fits(queue[0][2]):
                _, _, r = heapq.heappop(queue)
                self.admit(r, now())
            if self.resident:
                self.step()
                results.extend(self.retire(now))
            elif k < len(pending):
                time.sleep(max(0.0, min(0.01, pending[k].arrival * time_scale - now())))
        makespan = now()
        lat = np.array([r.latency for r in results])
        return {
            "results": results,
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "embeddings_per_s": len(results) / makespan if makespan > 0 else None,
            "makespan_s": makespan,
            "peak_bytes": self.peak_used,
            "rounds": self.rounds,
        }


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate (per second)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_alone(req: Request, tuning: Tuning | None = None, p: int = 3) -> np.ndarray:
    """The request run by itself in a batch of one job (same kernels, same tuning)."""
    with Batch(req.s, p=p, max_jobs=1) as b:
        if tuning is not None:
            b.set_tuning(tuning)
        P = DeviceCSR.from_host(req.row_ptr, req.col, req.val)
        j = b.add(P, torch.as_tensor(req.Y0, device="cuda"), req.sched, req.n_intervals)
        b.iterate(req.sched.n_iter)
        return b.get_y(j).cpu().numpy()
