"""GB300-native FIt-SNE gradient (arXiv 1712.09005): Python binding.

The functions below carry the names of the C-ABI entry points of
include/fitsne_gb300.h and only marshal arguments (torch tensors for device
buffers, numpy arrays for host buffers). All arithmetic of the gradient
(bounding box, sort, spread, FFT convolution, interpolation, attraction,
update, Z and KL) runs in the CUDA kernels of libfitsne_gb300.so; there is
no CPU fallback and the import fails if the library is missing.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, fields

import numpy as np
import torch

from . import _abi
from ._abi import TsneError, check

__all__ = ["Plan", "DeviceCSR", "Schedule", "tsne_plan_create", "tsne_plan_destroy",
           "tsne_plan_set_box", "tsne_gradient", "tsne_step", "tsne_run", "tsne_run_reset", "tsne_run_iters", "tsne_kl",
           "tsne_run_state_save", "tsne_run_state_load", "tsne_plan_order",
           "tsne_run_host", "tsne_validate_csr", "tsne_plan_status", "tsne_plan_info",
           "tsne_debug_copy", "tsne_plan_profile", "tsne_plan_profile_read",
           "tsne_plan_launch_count", "tsne_kl_noalloc", "TsneError", "Batch", "Tuning",
           "tsne_batch_create", "tsne_batch_destroy", "tsne_batch_job_bytes",
           "tsne_batch_bytes_in_use", "tsne_batch_add_job", "tsne_batch_remove_job",
           "tsne_batch_iterate", "tsne_batch_poll", "tsne_batch_get_y", "tsne_batch_kl",
           "tsne_batch_set_tuning", "tsne_batch_get_tuning", "tsne_batch_autotune",
           "tsne_batch_launch_count", "tsne_batch_stream", "Affinity", "tsne_affinity_create",
           "tsne_affinity_destroy", "tsne_affinity_compute", "tsne_affinity_knn_copy",
           "tsne_affinity_phase_ms", "tsne_affinity_launch_count", "tsne_affinity_knn_info", "Heatmap", "tsne_heatmap_create",
           "tsne_heatmap_destroy", "tsne_heatmap_bin", "tsne_heatmap_nearest", "tsne_heatmap_phase_ms",
           "tsne_heatmap_launch_count", "OocPca", "tsne_oocpca_create", "tsne_oocpca_destroy",
           "tsne_oocpca_run", "tsne_oocpca_debug_copy", "tsne_oocpca_phase_ms",
           "tsne_oocpca_launch_count"]


def lib():
    return _abi.load()


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@dataclass
class DeviceCSR:
    """P on the device: int32 row_ptr [N+1], int32 col [nnz], fp32 val [nnz]."""
    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor

    @staticmethod
    def from_host(row_ptr, col, val, device="cuda") -> "DeviceCSR":
        return DeviceCSR(torch.as_tensor(np.ascontiguousarray(row_ptr, np.int32), device=device),
                         torch.as_tensor(np.ascontiguousarray(col, np.int32), device=device),
                         torch.as_tensor(np.ascontiguousarray(val, np.float32), device=device))

    @property
    def N(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.col.numel()

    def c(self) -> _abi.tsne_csr:
        for t, dt in ((self.row_ptr, torch.int32), (self.col, torch.int32), (self.val, torch.float32)):
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError("DeviceCSR tensors must be contiguous CUDA int32/int32/float32")
        return _abi.tsne_csr(self.row_ptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr(),
                             self.nnz)


@dataclass
class Schedule:
    """tsne_step_params (exaggeration schedule and optimizer constants)."""
    n_iter: int = 1000
    early_iters: int = 250
    late_iters: int = 0
    mom_switch_iter: int = 250
    early_alpha: float = 12.0
    late_alpha: float = 1.0
    lr: float = 200.0
    momentum_early: float = 0.5
    momentum_late: float = 0.8
    min_gain: float = 0.01
    gain_inc: float = 0.2
    gain_dec: float = 0.8

    def c(self) -> _abi.tsne_step_params:
        return _abi.tsne_step_params(*[getattr(self, f.name) for f in fields(self)])


def _vec(t: torch.Tensor, N: int, s: int, name: str):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == N * s):
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor of {N}x{s}")
    return _ptr(t)


# ---- functions named after the C entry points --------------------------------

def tsne_plan_create(N: int, s: int, n_intervals: int = 0, p: int = 3, n_min: int = 0,
                     n_int_max: int = 0, stream: int | None = None, relabel_first: int = 0,
                     relabel_every: int = 0, force_mode: int = 0,
                     order_rounds: int = 0) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    opts = _abi.tsne_plan_opts(n_min, n_int_max, stream, relabel_first, relabel_every, force_mode,
                               order_rounds)
    out = ctypes.c_void_p()
    check(lib().tsne_plan_create(N, s, n_intervals, p, ctypes.byref(opts), ctypes.byref(out)))
    return out


def tsne_plan_destroy(plan) -> None:
    check(lib().tsne_plan_destroy(plan))


def tsne_plan_set_box(plan, y_min: float, width: float, n_int: int) -> None:
    check(lib().tsne_plan_set_box(plan, y_min, width, n_int))


def tsne_gradient(plan, P: DeviceCSR, Y, alpha, dY, Z=None) -> None:
    check(lib().tsne_gradient(plan, P.c(), _ptr(Y), alpha, _ptr(dY), _ptr(Z)))


def tsne_step(plan, P: DeviceCSR, Y, uY, gains, it: int, sched: Schedule) -> None:
    sp = sched.c()
    check(lib().tsne_step(plan, P.c(), _ptr(Y), _ptr(uY), _ptr(gains), it, ctypes.byref(sp)))


def tsne_run(plan, P: DeviceCSR, Y, sched: Schedule, want_kl: bool = True):
    sp = sched.c()
    kl = ctypes.c_double(float("nan"))
    check(lib().tsne_run(plan, P.c(), _ptr(Y), ctypes.byref(sp),
                         ctypes.byref(kl) if want_kl else None))
    return kl.value if want_kl else None


def tsne_run_reset(plan) -> None:
    check(lib().tsne_run_reset(plan))


def tsne_plan_order(plan, P: DeviceCSR) -> None:
    check(lib().tsne_plan_order(plan, P.c()))


def tsne_run_state_save(plan, uY: np.ndarray, gains: np.ndarray) -> None:
    for a in (uY, gains):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("uY and gains must be contiguous float32 host arrays")
    check(lib().tsne_run_state_save(plan, ctypes.c_void_p(uY.ctypes.data), ctypes.c_void_p(gains.ctypes.data)))


def tsne_run_state_load(plan, uY: np.ndarray, gains: np.ndarray) -> None:
    uY = np.ascontiguousarray(uY, np.float32)
    gains = np.ascontiguousarray(gains, np.float32)
    check(lib().tsne_run_state_load(plan, ctypes.c_void_p(uY.ctypes.data), ctypes.c_void_p(gains.ctypes.data)))


def tsne_run_iters(plan, P: DeviceCSR, Y, sched: Schedule, it_begin: int, count: int) -> None:
    sp = sched.c()
    check(lib().tsne_run_iters(plan, P.c(), _ptr(Y), ctypes.byref(sp), it_begin, count))


def tsne_kl(plan, P: DeviceCSR, Y) -> float:
    kl = ctypes.c_double()
    check(lib().tsne_kl(plan, P.c(), _ptr(Y), ctypes.byref(kl)))
    return kl.value


def tsne_run_host(plan, row_ptr: np.ndarray, col: np.ndarray, val: np.ndarray, Y: np.ndarray,
                  sched: Schedule, want_kl: bool = True):
    """Y (host float32, N x s) is overwritten with the embedding."""
    for a, dt in ((row_ptr, np.int32), (col, np.int32), (val, np.float32), (Y, np.float32)):
        if a.dtype != dt or not a.flags.c_contiguous:
            raise TypeError("host arrays must be contiguous int32/int32/float32/float32")
    sp = sched.c()
    kl = ctypes.c_double(float("nan"))
    P_ = ctypes.c_void_p
    check(lib().tsne_run_host(plan, P_(row_ptr.ctypes.data), P_(col.ctypes.data),
                              P_(val.ctypes.data), len(col), P_(Y.ctypes.data), ctypes.byref(sp),
                              ctypes.byref(kl) if want_kl else None))
    return kl.value if want_kl else None


def tsne_validate_csr(plan, P: DeviceCSR) -> None:
    check(lib().tsne_validate_csr(plan, P.c()))


def tsne_plan_status(plan) -> int:
    return int(lib().tsne_plan_status(plan))


def tsne_plan_info(plan) -> dict:
    info = _abi.tsne_plan_info_t()
    check(lib().tsne_plan_info(plan, ctypes.byref(info)))
    return {f[0]: getattr(info, f[0]) for f in info._fields_ if f[0] != "pad"}


def tsne_debug_copy(plan, which: int, s: int) -> np.ndarray:
    need = ctypes.c_size_t()
    check(lib().tsne_debug_copy(plan, which, None, 0, ctypes.byref(need)))
    if which == 2:
        out = np.empty(need.value // 4, dtype=np.int32)
    elif which == 1:
        out = np.empty((need.value // 16, 4), dtype=np.float32)
    else:
        out = np.empty(need.value // 8, dtype=np.float64)
    check(lib().tsne_debug_copy(plan, which, ctypes.c_void_p(out.ctypes.data), out.nbytes, None))
    return out


PHASES = ("box", "sort_spread", "fft_conv", "force")


def tsne_plan_profile(plan, enable: bool) -> None:
    check(lib().tsne_plan_profile(plan, 1 if enable else 0))


def tsne_plan_profile_read(plan) -> dict:
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    check(lib().tsne_plan_profile_read(plan, ms, cnt))
    return {"ms": dict(zip(PHASES, list(ms))), "evals": int(cnt[0])}


def tsne_plan_launch_count(plan) -> int:
    return int(lib().tsne_plan_launch_count(plan))


def tsne_kl_noalloc(P: DeviceCSR, Y: torch.Tensor, s: int, Z: float, kl_out: torch.Tensor,
                    stream: int | None = None) -> None:
    """KL without device allocation; kl_out is a 1-element float64 CUDA tensor."""
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    if not (kl_out.is_cuda and kl_out.dtype == torch.float64 and kl_out.numel() >= 1):
        raise TypeError("kl_out must be a float64 CUDA tensor")
    N = P.N
    if s in (1, 2):
        _vec(Y, N, s, "Y")  # the kernel reads Y[col[e]] for every stored entry of P
    rc = lib().tsne_kl_noalloc(P.c(), _ptr(Y), N, s, float(Z), _ptr(kl_out),
                               ctypes.c_void_p(stream))
    if rc != 0:
        raise TsneError(rc, lib().tsne_noalloc_last_error_string().decode())


# ---- input affinities ------------------------------------------------------------

def tsne_affinity_create(N: int, D: int, k: int, stream: int | None = None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    check(lib().tsne_affinity_create(N, D, k, ctypes.c_void_p(stream), ctypes.byref(out)))
    return out


def tsne_affinity_destroy(aff) -> None:
    check(lib().tsne_affinity_destroy(aff))


def tsne_affinity_compute(aff, X: torch.Tensor, perplexity: float) -> _abi.tsne_csr:
    if not (X.is_cuda and X.dtype == torch.float32 and X.is_contiguous() and X.dim() == 2):
        raise TypeError("X must be a contiguous 2-D CUDA float32 tensor")
    out = _abi.tsne_csr()
    check(lib().tsne_affinity_compute(aff, _ptr(X), float(perplexity), ctypes.byref(out)))
    return out


def tsne_affinity_knn_copy(aff, idx=None, d2=None, pcond=None) -> None:
    def host(a):
        return None if a is None else ctypes.c_void_p(a.ctypes.data)
    check(lib().tsne_affinity_knn_copy(aff, host(idx), host(d2), host(pcond)))


def tsne_affinity_phase_ms(aff) -> list[float]:
    ms = (ctypes.c_double * 4)()
    check(lib().tsne_affinity_phase_ms(aff, ms))
    return list(ms)


def tsne_affinity_launch_count(aff) -> int:
    return lib().tsne_affinity_launch_count(aff)


def tsne_affinity_knn_info(aff) -> tuple[int, int]:
    """(kNN kernel: 0 rows, 1 tiled, 2 tensor cores; queries of the last
    compute recomputed by the row kernel)."""
    kind = ctypes.c_int32()
    rec = ctypes.c_int64()
    check(lib().tsne_affinity_knn_info(aff, ctypes.byref(kind), ctypes.byref(rec)))
    return kind.value, rec.value


class Affinity:
    """Workspace for P from data X (N x D float32 on the device): exact kNN,
    perplexity calibration and symmetrisation in the library's kernels.

    compute() returns a DeviceCSR whose tensors view the workspace's memory:
    valid until the next compute() or close()."""

    def __init__(self, N: int, D: int, k: int, stream: int | None = None):
        self.N, self.D, self.k = N, D, k
        self._h = tsne_affinity_create(N, D, k, stream)

    def compute(self, X: torch.Tensor, perplexity: float = 30.0) -> DeviceCSR:
        if X.shape != (self.N, self.D):
            raise ValueError(f"X must be {self.N} x {self.D}")
        c = tsne_affinity_compute(self._h, X, perplexity)
        dev = X.device

        def view(ptr, n, dtype):
            # a zero-copy view of workspace memory (kept alive by this object)
            return _device_view(ptr, n, dtype, dev)
        return DeviceCSR(view(c.row_ptr, self.N + 1, torch.int32), view(c.col, c.nnz, torch.int32),
                         view(c.val, c.nnz, torch.float32))

    def knn(self):
        """(idx int32 N x k, d2 float32 N x k, p_{j|i} float64 N x k) of the last compute, on the host."""
        idx = np.empty((self.N, self.k), np.int32)
        d2 = np.empty((self.N, self.k), np.float32)
        pc = np.empty((self.N, self.k), np.float64)
        tsne_affinity_knn_copy(self._h, idx, d2, pc)
        return idx, d2, pc

    def launch_count(self) -> int:
        return tsne_affinity_launch_count(self._h)

    def phase_ms(self) -> dict:
        """Device time of the last compute's phases (CUDA events on its stream)."""
        return dict(zip(("knn", "bandwidths", "edge_sort", "symmetrise"), tsne_affinity_phase_ms(self._h)))

    def knn_info(self) -> dict:
        """The kNN kernel in use ("rows", "tiled", "tc") and the queries of the
        last compute that the tensor-core kernel left to the row kernel."""
        kind, rec = tsne_affinity_knn_info(self._h)
        return {"kernel": ("rows", "tiled", "tc")[kind], "recomputed": rec}

    def close(self):
        if self._h is not None:
            tsne_affinity_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tsne_heatmap_create(n_bins: int, G: int, max_goi: int = 64, stream: int | None = None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    check(lib().tsne_heatmap_create(n_bins, G, max_goi, ctypes.c_void_p(stream), ctypes.byref(out)))
    return out


def tsne_heatmap_destroy(hm) -> None:
    check(lib().tsne_heatmap_destroy(hm))


def tsne_heatmap_bin(hm, y: torch.Tensor, E: "DeviceCSR", H: torch.Tensor, bin_count: torch.Tensor) -> None:
    if not (y.is_cuda and y.dtype == torch.float32 and y.is_contiguous() and y.dim() == 1):
        raise TypeError("y must be a contiguous 1-D CUDA float32 tensor")
    if not (H.is_cuda and H.dtype == torch.float64 and H.is_contiguous()):
        raise TypeError("H must be a contiguous CUDA float64 tensor")
    if not (bin_count.is_cuda and bin_count.dtype == torch.int32 and bin_count.is_contiguous()):
        raise TypeError("bin_count must be a contiguous CUDA int32 tensor")
    if H.numel() != H.shape[0] * H.shape[-1] or bin_count.numel() != H.shape[0]:
        raise ValueError("H must be n_bins x G and bin_count n_bins long")
    if E.row_ptr.numel() != y.numel() + 1:
        raise ValueError("E must have one row per cell")
    check(lib().tsne_heatmap_bin(hm, _ptr(y), y.numel(), E.c(), _ptr(H), _ptr(bin_count)))


def tsne_heatmap_nearest(hm, H: torch.Tensor, goi: np.ndarray, m: int, idx: np.ndarray, dist: np.ndarray) -> None:
    goi = np.ascontiguousarray(goi, dtype=np.int32)
    if idx.dtype != np.int32 or dist.dtype != np.float64 or idx.size < goi.size * m or dist.size < goi.size * m:
        raise TypeError("idx must be int32 and dist float64, n_goi x m each")
    check(lib().tsne_heatmap_nearest(hm, _ptr(H), ctypes.c_void_p(goi.ctypes.data), goi.size, m,
                                     ctypes.c_void_p(idx.ctypes.data), ctypes.c_void_p(dist.ctypes.data)))


def tsne_heatmap_phase_ms(hm) -> list[float]:
    ms = (ctypes.c_double * 4)()
    check(lib().tsne_heatmap_phase_ms(hm, ms))
    return list(ms)


def tsne_heatmap_launch_count(hm) -> int:
    return lib().tsne_heatmap_launch_count(hm)


class Heatmap:
    """t-SNE heatmaps (Sec. 5) of a 1-D embedding of N cells and a cells x
    genes expression matrix E (DeviceCSR over cells, column = gene index):
    bin() sums every gene's expression per equal-width bin of the embedding
    (H, n_bins x G, FP64) and counts the cells per bin; nearest() returns, for
    each gene of interest, the m genes nearest to it in the Euclidean distance
    of those per-bin vectors (the rows of the heatmap)."""

    def __init__(self, n_bins: int, G: int, max_goi: int = 64, stream: int | None = None):
        self.n_bins, self.G, self.max_goi = n_bins, G, max_goi
        self._h = tsne_heatmap_create(n_bins, G, max_goi, stream)

    def bin(self, y: torch.Tensor, E: "DeviceCSR", H: torch.Tensor | None = None):
        if H is None:
            H = torch.empty((self.n_bins, self.G), dtype=torch.float64, device=y.device)
        if H.shape != (self.n_bins, self.G):
            raise ValueError(f"H must be {self.n_bins} x {self.G}")
        counts = torch.empty(self.n_bins, dtype=torch.int32, device=y.device)
        tsne_heatmap_bin(self._h, y, E, H, counts)
        return H, counts

    def nearest(self, H: torch.Tensor, goi, m: int):
        goi = np.asarray(goi, dtype=np.int32).ravel()
        idx = np.empty((goi.size, m), np.int32)
        dist = np.empty((goi.size, m), np.float64)
        tsne_heatmap_nearest(self._h, H, goi, m, idx, dist)
        return idx, dist

    def phase_ms(self) -> dict:
        """Device time of the last calls' phases (CUDA events on the workspace's stream)."""
        return dict(zip(("range", "bin_sums", "distances", "selection"), tsne_heatmap_phase_ms(self._h)))

    def launch_count(self) -> int:
        return tsne_heatmap_launch_count(self._h)

    def close(self):
        if self._h is not None:
            tsne_heatmap_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr: int, n: int, dtype: torch.dtype, device) -> torch.Tensor:
    """A torch tensor over n elements of library-owned device memory (no copy)."""
    elem = torch.tensor([], dtype=dtype).element_size()

    class _Iface:
        __cuda_array_interface__ = {
            "shape": (n,), "typestr": {torch.int32: "<i4", torch.float32: "<f4"}[dtype],
            "data": (int(ptr or 0), False), "version": 3, "strides": None}
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    t = torch.as_tensor(_Iface(), device=device)
    assert t.element_size() == elem
    return t


# ---- batched jobs ---------------------------------------------------------------

@dataclass
class Tuning:
    """tsne_batch_tuning: spread work item, FFT threads per CTA, interval policy."""
    chunk: int = 64
    fft_threads: int = 0
    n_int_policy: int = _abi.TSNE_NINT_RULE
    ms_per_iter: float = 0.0

    def c(self) -> _abi.tsne_batch_tuning:
        return _abi.tsne_batch_tuning(self.chunk, self.fft_threads, self.n_int_policy,
                                      self.ms_per_iter)

    @staticmethod
    def of(t: _abi.tsne_batch_tuning) -> "Tuning":
        return Tuning(t.chunk, t.fft_threads, t.n_int_policy, t.ms_per_iter)


def tsne_batch_create(s: int, p: int = 3, n_min: int = 0, n_int_max: int = 0, max_jobs: int = 64,
                      use_graph: bool = True, stream: int | None = None) -> ctypes.c_void_p:
    opts = _abi.tsne_batch_opts()
    lib().tsne_batch_opts_default(ctypes.byref(opts))
    opts.n_min, opts.n_int_max, opts.max_jobs = n_min, n_int_max, max_jobs
    opts.use_graph = 1 if use_graph else 0
    opts.stream = stream
    out = ctypes.c_void_p()
    check(lib().tsne_batch_create(s, p, ctypes.byref(opts), ctypes.byref(out)))
    return out


def tsne_batch_destroy(batch) -> None:
    check(lib().tsne_batch_destroy(batch))


def tsne_batch_job_bytes(batch, N: int) -> int:
    return int(lib().tsne_batch_job_bytes(batch, N))


def tsne_batch_bytes_in_use(batch) -> int:
    return int(lib().tsne_batch_bytes_in_use(batch))


def tsne_batch_add_job(batch, P: DeviceCSR, Y0: torch.Tensor, sched: Schedule,
                       n_intervals: int = 0) -> int:
    sp = sched.c()
    jid = ctypes.c_int32(-1)
    check(lib().tsne_batch_add_job(batch, P.N, P.c(), _ptr(Y0), n_intervals, ctypes.byref(sp),
                                   ctypes.byref(jid)))
    return jid.value


def tsne_batch_remove_job(batch, job: int) -> None:
    check(lib().tsne_batch_remove_job(batch, job))


def tsne_batch_iterate(batch, count: int) -> None:
    check(lib().tsne_batch_iterate(batch, count))


def tsne_batch_poll(batch, max_jobs: int):
    it = (ctypes.c_int32 * max_jobs)()
    st = (ctypes.c_int32 * max_jobs)()
    check(lib().tsne_batch_poll(batch, it, st))
    return list(it), list(st)


def tsne_batch_get_y(batch, job: int, Y_out: torch.Tensor) -> None:
    check(lib().tsne_batch_get_y(batch, job, _ptr(Y_out)))


def tsne_batch_kl(batch, job: int) -> float:
    kl = ctypes.c_double()
    check(lib().tsne_batch_kl(batch, job, ctypes.byref(kl)))
    return kl.value


def tsne_batch_set_tuning(batch, t: Tuning) -> None:
    tc = t.c()
    check(lib().tsne_batch_set_tuning(batch, ctypes.byref(tc)))


def tsne_batch_get_tuning(batch) -> Tuning:
    tc = _abi.tsne_batch_tuning()
    check(lib().tsne_batch_get_tuning(batch, ctypes.byref(tc)))
    return Tuning.of(tc)


def tsne_batch_autotune(batch, iters: int = 3) -> Tuning:
    tc = _abi.tsne_batch_tuning()
    check(lib().tsne_batch_autotune(batch, iters, ctypes.byref(tc)))
    return Tuning.of(tc)


def tsne_batch_launch_count(batch) -> int:
    return int(lib().tsne_batch_launch_count(batch))


def tsne_batch_stream(batch) -> int:
    return int(lib().tsne_batch_stream(batch) or 0)


class Batch:
    """Owns a tsne_batch: many embedding jobs iterated together (one launch
    per phase for all jobs, one CUDA graph per iteration)."""

    def __init__(self, s: int, p: int = 3, n_min: int = 0, n_int_max: int = 0,
                 max_jobs: int = 64, use_graph: bool = True, stream: int | None = None):
        self.s, self.max_jobs = s, max_jobs
        self.handle = tsne_batch_create(s, p, n_min, n_int_max, max_jobs, use_graph, stream)
        self.N = {}
        self._P = {}  # the batch reads each job's P until the job is removed
        self._ext = torch.cuda.ExternalStream(self.stream)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            tsne_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stream(self) -> int:
        return tsne_batch_stream(self.handle)

    def job_bytes(self, N: int) -> int:
        return tsne_batch_job_bytes(self.handle, N)

    def bytes_in_use(self) -> int:
        return tsne_batch_bytes_in_use(self.handle)

    def add(self, P: DeviceCSR, Y0: torch.Tensor, sched: Schedule, n_intervals: int = 0) -> int:
        _vec(Y0, P.N, self.s, "Y0")
        self._ext.wait_stream(torch.cuda.current_stream())  # P and Y0 are ready
        jid = tsne_batch_add_job(self.handle, P, Y0, sched, n_intervals)
        self.N[jid] = P.N
        self._P[jid] = (P, Y0)
        return jid

    def upload(self, req):
        """Copies a request's host CSR and Y0 to the device on the batch's
        stream (pinned staging, asynchronous)."""
        with torch.cuda.stream(self._ext):
            up = lambda a: torch.from_numpy(a).pin_memory().to("cuda", non_blocking=True)
            P = DeviceCSR(up(req.row_ptr), up(req.col), up(req.val))
            Y0 = up(req.Y0)
        return P, Y0

    def remove(self, job: int):
        tsne_batch_remove_job(self.handle, job)
        self.N.pop(job, None)
        self._P.pop(job, None)

    def iterate(self, count: int = 1):
        tsne_batch_iterate(self.handle, count)

    def poll(self):
        return tsne_batch_poll(self.handle, self.max_jobs)

    def get_y(self, job: int, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.N[job], self.s), dtype=torch.float32, device="cuda")
        _vec(out, self.N[job], self.s, "Y_out")
        self._ext.wait_stream(torch.cuda.current_stream())
        tsne_batch_get_y(self.handle, job, out)
        torch.cuda.current_stream().wait_stream(self._ext)
        return out

    def kl(self, job: int) -> float:
        return tsne_batch_kl(self.handle, job)

    def set_tuning(self, t: Tuning):
        tsne_batch_set_tuning(self.handle, t)

    def tuning(self) -> Tuning:
        return tsne_batch_get_tuning(self.handle)

    def autotune(self, iters: int = 3) -> Tuning:
        return tsne_batch_autotune(self.handle, iters)

    def launch_count(self) -> int:
        return tsne_batch_launch_count(self.handle)


# ---- convenience object -------------------------------------------------------

class Plan:
    """Owns a tsne_plan; methods forward to the functions above."""

    def __init__(self, N: int, s: int, n_intervals: int = 0, p: int = 3, n_min: int = 0,
                 n_int_max: int = 0, stream: int | None = None, relabel_first: int = 0,
                 relabel_every: int = 0, force_mode: int = 0, order_rounds: int = 0):
        self.N, self.s = N, s
        self.handle = tsne_plan_create(N, s, n_intervals, p, n_min, n_int_max, stream,
                                       relabel_first, relabel_every, force_mode, order_rounds)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            tsne_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_box(self, y_min: float, width: float, n_int: int):
        tsne_plan_set_box(self.handle, y_min, width, n_int)

    def gradient(self, P: DeviceCSR, Y: torch.Tensor, alpha: float = 1.0, dY=None, Z=None):
        _vec(Y, self.N, self.s, "Y")
        if dY is None:
            dY = torch.empty_like(Y)
        if Z is None:
            Z = torch.empty(1, dtype=torch.float64, device=Y.device)
        tsne_gradient(self.handle, P, Y, alpha, dY, Z)
        return dY, Z

    def step(self, P: DeviceCSR, Y, uY, gains, it: int, sched: Schedule):
        for t, nm in ((Y, "Y"), (uY, "uY"), (gains, "gains")):
            _vec(t, self.N, self.s, nm)
        tsne_step(self.handle, P, Y, uY, gains, it, sched)

    def run(self, P: DeviceCSR, Y: torch.Tensor, sched: Schedule, want_kl: bool = True):
        _vec(Y, self.N, self.s, "Y")
        return tsne_run(self.handle, P, Y, sched, want_kl)

    def run_reset(self):
        tsne_run_reset(self.handle)

    def order(self, P: DeviceCSR):
        if P.N != self.N:
            raise ValueError(f"P has {P.N} rows, the plan {self.N} points")
        tsne_plan_order(self.handle, P)

    def run_state_save(self):
        """(uY, gains) of the run, N x s float32 host arrays in the caller's labels."""
        uY = np.empty((self.N, self.s), np.float32)
        gains = np.empty((self.N, self.s), np.float32)
        tsne_run_state_save(self.handle, uY, gains)
        return uY, gains

    def run_state_load(self, uY: np.ndarray, gains: np.ndarray):
        if np.shape(uY) != (self.N, self.s) or np.shape(gains) != (self.N, self.s):
            raise ValueError(f"uY and gains must be {self.N} x {self.s}")
        tsne_run_state_load(self.handle, uY, gains)

    def run_iters(self, P: DeviceCSR, Y: torch.Tensor, sched: Schedule, it_begin: int, count: int):
        _vec(Y, self.N, self.s, "Y")
        tsne_run_iters(self.handle, P, Y, sched, it_begin, count)

    def kl(self, P: DeviceCSR, Y: torch.Tensor) -> float:
        _vec(Y, self.N, self.s, "Y")
        return tsne_kl(self.handle, P, Y)

    def run_host(self, row_ptr, col, val, Y: np.ndarray, sched: Schedule, want_kl: bool = True):
        return tsne_run_host(self.handle, row_ptr, col, val, Y, sched, want_kl)

    def validate(self, P: DeviceCSR):
        tsne_validate_csr(self.handle, P)

    def status(self) -> int:
        return tsne_plan_status(self.handle)

    def info(self) -> dict:
        return tsne_plan_info(self.handle)

    def debug(self, which: int) -> np.ndarray:
        return tsne_debug_copy(self.handle, which, self.s)

    def profile(self, enable: bool = True):
        tsne_plan_profile(self.handle, enable)

    def profile_read(self) -> dict:
        return tsne_plan_profile_read(self.handle)

    def launch_count(self) -> int:
        return tsne_plan_launch_count(self.handle)


# ---- out-of-core randomized PCA (Sec. 6, Algorithm oocPCA) ---------------------

def tsne_oocpca_create(m: int, n: int, k: int, l: int, its: int = 0, center: bool = False,
                       block_rows: int = 0, stream: int | None = None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    opts = _abi.tsne_oocpca_opts(its, 1 if center else 0, block_rows, stream)
    out = ctypes.c_void_p()
    check(lib().tsne_oocpca_create(m, n, k, l, ctypes.byref(opts), ctypes.byref(out)))
    return out


def tsne_oocpca_destroy(plan) -> None:
    check(lib().tsne_oocpca_destroy(plan))


def tsne_oocpca_run(plan, A_ptr: int, lda: int, a_on_host: bool, Omega: torch.Tensor, U: torch.Tensor,
                    sigma: torch.Tensor, V: torch.Tensor) -> None:
    check(lib().tsne_oocpca_run(plan, ctypes.c_void_p(A_ptr), lda, 1 if a_on_host else 0, _ptr(Omega),
                                _ptr(U), _ptr(sigma), _ptr(V)))


def tsne_oocpca_debug_copy(plan, which: int, rows: int, l: int) -> np.ndarray:
    out = np.empty((rows, l), np.float64)
    check(lib().tsne_oocpca_debug_copy(plan, which, out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
    return out


def tsne_oocpca_phase_ms(plan) -> tuple[list[float], int]:
    ms = (ctypes.c_double * 4)()
    passes = ctypes.c_int32()
    check(lib().tsne_oocpca_phase_ms(plan, ms, ctypes.byref(passes)))
    return list(ms), passes.value


def tsne_oocpca_launch_count(plan) -> int:
    return int(lib().tsne_oocpca_launch_count(plan))


class OocPca:
    """Owns a tsne_oocpca plan: top-k PCA of an m x n FP32 matrix held on the
    device (a torch tensor) or in host memory (a numpy array, pinned or not),
    read block by block."""

    def __init__(self, m: int, n: int, k: int, l: int | None = None, its: int = 0,
                 center: bool = False, block_rows: int = 0, stream: int | None = None):
        self.m, self.n, self.k = m, n, k
        self.l = k + 2 if l is None else l
        self.handle = tsne_oocpca_create(m, n, k, self.l, its, center, block_rows, stream)

    def run(self, A, Omega):
        """A: torch CUDA float32 (m x n, row stride a multiple of 4) or a host
        float32 array; Omega: n x l. Returns (U, sigma, V) as CUDA tensors."""
        if isinstance(A, torch.Tensor) and A.is_cuda:
            if A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1 or tuple(A.shape) != (self.m, self.n):
                raise TypeError("A must be a CUDA float32 m x n tensor with unit column stride")
            ptr, lda, host = A.data_ptr(), A.stride(0), False
        else:
            if isinstance(A, torch.Tensor):
                A = A.numpy()
            if A.dtype != np.float32 or A.ndim != 2 or A.shape != (self.m, self.n) or A.strides[1] != 4:
                raise TypeError("A must be a float32 m x n array with unit column stride")
            ptr, lda, host = A.ctypes.data, A.strides[0] // 4, True
        Om = torch.as_tensor(np.asarray(Omega, np.float32) if not isinstance(Omega, torch.Tensor) else Omega,
                             device="cuda", dtype=torch.float32).contiguous()
        if tuple(Om.shape) != (self.n, self.l):
            raise ValueError(f"Omega must be {self.n} x {self.l}")
        U = torch.empty((self.m, self.k), device="cuda", dtype=torch.float32)
        V = torch.empty((self.n, self.k), device="cuda", dtype=torch.float32)
        sig = torch.empty(self.k, device="cuda", dtype=torch.float64)
        tsne_oocpca_run(self.handle, ptr, lda, host, Om, U, sig, V)
        return U, sig, V

    def debug(self, which: int) -> np.ndarray:
        rows = self.n if which == 1 else self.m
        return tsne_oocpca_debug_copy(self.handle, which, rows, self.l)

    def phase_ms(self):
        ms, passes = tsne_oocpca_phase_ms(self.handle)
        return {"passes_ms": ms[0], "renormalize_ms": ms[1], "qr_svd_ms": ms[2], "means_ms": ms[3],
                "passes": passes}

    def launch_count(self) -> int:
        return tsne_oocpca_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            tsne_oocpca_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
