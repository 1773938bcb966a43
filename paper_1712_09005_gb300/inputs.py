"""Seeded synthetic inputs: Gaussian-mixture data, kNN affinities P, Y0.

This module only prepares inputs; it computes nothing of the per-iteration
gradient. Both the CUDA path's tests/benchmark and the oracle's tests draw
their inputs from here (the oracle checks the affinities independently with
its own builder).

Workloads (stand-ins shaped like the paper's 50-dimensional PCA inputs of
10^5 - 10^6 points; no dataset item is reproduced):

  mixture(N, n_clusters, ...)   X ~ sum of isotropic unit-variance Gaussians in
                                50-d, centres ~ N(0, centre_std^2 I); sizes
                                equal or ~ Multinomial(N, Dirichlet(1)); an
                                optional fraction of uniform background points
                                on the per-dimension [min, max] of the centres
                                widened by 3.
  affinities(X, perplexity, k)  exact kNN (k = 3 * perplexity by default),
                                per-point bandwidth by bisection to the target
                                perplexity, symmetrised p_ij = (p_j|i + p_i|j)/2N
                                (Sec. 1.1 and Sec. 3), CSR int32/int32/fp32.
  initial_embedding(N, s)       Y0 ~ N(0, 1e-4 I), fp32.
  expression(N, G, ...)         a cells x genes count matrix (CSR over cells)
                                and a clustered 1-D layout of the cells, for
                                the t-SNE heatmaps of Sec. 5 (shaped like a
                                single-cell RNA-seq count matrix; synthetic).

Random numbers come from numpy's PCG64 with the seed given.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass

import numpy as np
import torch

_CACHE = os.environ.get(
    "FITSNE_INPUT_CACHE",
    os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".cache"))


@dataclass
class CSR:
    row_ptr: np.ndarray  # int32 [N+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float32 [nnz]

    @property
    def N(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnz(self) -> int:
        return len(self.col)

    def as_tuple(self):
        return self.row_ptr, self.col, self.val


def mixture(N: int, n_clusters: int, dim: int = 50, centre_std: float = 5.0,
            sizes: str = "equal", background: float = 0.0, seed: int = 0) -> np.ndarray:
    """N points of an isotropic unit-variance Gaussian mixture in `dim` dimensions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_bg = int(round(background * N))
    n_cl = N - n_bg
    centres = rng.normal(0.0, centre_std, size=(n_clusters, dim))
    if sizes == "equal":
        counts = np.full(n_clusters, n_cl // n_clusters)
        counts[: n_cl - counts.sum()] += 1
    elif sizes == "dirichlet":
        counts = rng.multinomial(n_cl, rng.dirichlet(np.ones(n_clusters)))
    else:
        raise ValueError(sizes)
    X = np.empty((N, dim), dtype=np.float32)
    pos = 0
    for c, cnt in enumerate(counts):
        X[pos:pos + cnt] = centres[c] + rng.standard_normal((cnt, dim))
        pos += cnt
    if n_bg:
        lo = centres.min(axis=0) - 3.0
        hi = centres.max(axis=0) + 3.0
        X[pos:] = rng.uniform(lo, hi, size=(n_bg, dim))
    perm = rng.permutation(N)
    return X[perm]


def initial_embedding(N: int, s: int, seed: int = 0) -> np.ndarray:
    """Y0 ~ N(0, 1e-4 I) as fp32 [N, s]."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return (rng.standard_normal((N, s)) * 1e-2).astype(np.float32)


def _knn(X: torch.Tensor, k: int, chunk: int):
    """Exact k nearest neighbours (self excluded); returns (idx int64, d2)."""
    N = X.shape[0]
    sq = (X * X).sum(1)
    idx = torch.empty((N, k), dtype=torch.int64, device=X.device)
    d2 = torch.empty((N, k), dtype=X.dtype, device=X.device)
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        D = sq[a:b, None] + sq[None, :] - 2.0 * (X[a:b] @ X.T)
        D[torch.arange(b - a, device=X.device), torch.arange(a, b, device=X.device)] = float("inf")
        vals, ids = torch.topk(D, k, dim=1, largest=False, sorted=True)
        idx[a:b] = ids
        # recompute the selected distances in difference form (no cancellation)
        diff = X[a:b, None, :] - X[ids]
        d2[a:b] = (diff * diff).sum(-1)
        del D, vals, diff
    return idx, d2


def _bandwidths(d2: torch.Tensor, perplexity: float, tol: float = 1e-5, max_iter: int = 200):
    """Row-wise bisection on beta = 1/(2 sigma^2) to the target perplexity."""
    target = float(np.log(perplexity))
    x = d2 - d2.min(dim=1, keepdim=True).values
    beta = torch.ones(x.shape[0], dtype=x.dtype, device=x.device)
    lo = torch.full_like(beta, -float("inf"))
    hi = torch.full_like(beta, float("inf"))
    for _ in range(max_iter):
        e = torch.exp(-beta[:, None] * x)
        ssum = e.sum(1)
        pr = e / ssum[:, None]
        H = torch.log(ssum) + beta * (pr * x).sum(1)
        active = (H - target).abs() >= tol
        if not bool(active.any()):
            break
        flat = active & (H > target)
        sharp = active & (H <= target)
        lo = torch.where(flat, beta, lo)
        hi = torch.where(sharp, beta, hi)
        up = torch.where(torch.isinf(hi), beta * 2.0, (beta + hi) * 0.5)
        down = torch.where(torch.isinf(lo), beta * 0.5, (beta + lo) * 0.5)
        beta = torch.where(flat, up, torch.where(sharp, down, beta))
    e = torch.exp(-beta[:, None] * x)
    return e / e.sum(1, keepdim=True)


def affinities(X: np.ndarray, perplexity: float = 30.0, k: int | None = None,
               device: str = "cpu", dtype=None, chunk: int | None = None) -> CSR:
    """Symmetric normalised kNN affinities of X as fp32 CSR (sorted columns)."""
    if k is None:
        k = int(3 * perplexity)
    dev = torch.device(device)
    if dtype is None:
        dtype = torch.float64 if dev.type == "cpu" else torch.float32
    Xt = torch.as_tensor(np.asarray(X), device=dev).to(dtype)
    N = Xt.shape[0]
    if chunk is None:
        chunk = 1024 if dev.type != "cpu" else 512
    idx, d2 = _knn(Xt, k, chunk)
    pc = _bandwidths(d2, perplexity)
    rows = torch.arange(N, device=dev, dtype=torch.int64).repeat_interleave(k)
    cols = idx.reshape(-1)
    v = pc.reshape(-1).to(torch.float64 if dev.type == "cpu" else torch.float32)
    key = torch.cat([rows * N + cols, cols * N + rows])
    vv = torch.cat([v, v])
    key, order = torch.sort(key)
    vv = vv[order]
    ukey, inv = torch.unique_consecutive(key, return_inverse=True)
    sums = torch.zeros(ukey.shape[0], dtype=vv.dtype, device=dev).index_add_(0, inv, vv)
    sums = sums / (2.0 * N)
    r = ukey // N
    c = ukey % N
    counts = torch.bincount(r, minlength=N)
    row_ptr = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return CSR(row_ptr.to(torch.int32).cpu().numpy(), c.to(torch.int32).cpu().numpy(),
               sums.to(torch.float32).cpu().numpy())


@dataclass
class Workload:
    name: str
    X_args: dict
    perplexity: float
    k: int
    s: int
    seed: int


def _key(*parts) -> str:
    return hashlib.sha1(repr(parts).encode()).hexdigest()[:16]


def cached_affinities(name: str, X_args: dict, perplexity: float, k: int, device: str = "cpu") -> CSR:
    """affinities(mixture(**X_args)) cached on disk (inputs only; safe to delete)."""
    os.makedirs(_CACHE, exist_ok=True)
    path = os.path.join(_CACHE, f"P_{name}_{_key(X_args, perplexity, k)}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return CSR(z["row_ptr"], z["col"], z["val"])
    X = mixture(**X_args)
    P = affinities(X, perplexity, k, device=device)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, row_ptr=P.row_ptr, col=P.col, val=P.val)
    os.replace(tmp, path)
    return P


# The five workloads, seeds 1000 * workload + job.
def mixture_args(workload: int, job: int = 0, N: int | None = None) -> dict:
    seed = 1000 * workload + job
    if workload == 1:
        return dict(N=N or 2000, n_clusters=10, sizes="equal", seed=seed)
    if workload == 2:
        return dict(N=N or 100_000, n_clusters=30, sizes="dirichlet", seed=seed)
    if workload == 3:
        return dict(N=N or 1_000_000, n_clusters=100, sizes="equal", background=0.05, seed=seed)
    if workload in (4, 5):
        rng = np.random.Generator(np.random.PCG64(seed))
        n_cl = int(rng.integers(10, 31))
        return dict(N=N, n_clusters=n_cl, sizes="dirichlet", seed=seed)
    raise ValueError(workload)


def log_uniform_sizes(n_jobs: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_jobs)).astype(np.int64)


@dataclass
class Expression:
    """Cells x genes counts as CSR over cells (int32 row_ptr, int32 gene
    index, fp32 count) and a 1-D layout y (fp32) of the cells."""
    y: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    G: int
    label: np.ndarray

    def as_tuple(self):
        return self.row_ptr, self.col, self.val


def expression(N: int, G: int, mean_genes: float = 1000.0, n_clusters: int = 20,
               markers: int = 25, seed: int = 0) -> Expression:
    """Synthetic single-cell counts: cluster c of the cells raises the rate
    of its own `markers` genes 20-fold over log-normal base rates; a cell of
    cluster c draws Poisson(mean_genes) reads from its cluster's gene
    distribution (with replacement), and its row holds each distinct gene
    with its read count. y places cluster c at 10 c + N(0, 1) along a line, in
    a shuffled cluster order (a 1-D embedding's layout)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    label = rng.integers(0, n_clusters, size=N)
    order = rng.permutation(n_clusters)
    y = (10.0 * order[label] + rng.normal(0.0, 1.0, size=N)).astype(np.float32)
    base = rng.lognormal(0.0, 1.0, size=G)
    reads = np.clip(rng.poisson(mean_genes, size=N), 1, None)
    keys = []
    for c in range(n_clusters):
        cells = np.nonzero(label == c)[0]
        if cells.size == 0:
            continue
        w = base.copy()
        w[rng.choice(G, size=min(markers, G), replace=False)] *= 20.0
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        r = reads[cells]
        owner = np.repeat(cells, r)
        gene = np.minimum(np.searchsorted(cdf, rng.random(owner.size), side="right"), G - 1)
        keys.append(owner.astype(np.int64) * G + gene)
    keys = np.concatenate(keys) if keys else np.zeros(0, np.int64)
    uk, cnt = np.unique(keys, return_counts=True)
    cell = uk // G
    row_ptr = np.zeros(N + 1, np.int64)
    np.cumsum(np.bincount(cell, minlength=N), out=row_ptr[1:])
    return Expression(y, row_ptr.astype(np.int32), (uk % G).astype(np.int32), cnt.astype(np.float32), G,
                      label)


# ---- out-of-core PCA inputs (Sec. 6) -------------------------------------------

def planted_spectrum(rank: int, top: float = 100.0, ratio: float = 1e-2) -> np.ndarray:
    """Singular values decaying geometrically from top to top * ratio."""
    if rank == 1:
        return np.array([top])
    return top * ratio ** (np.arange(rank) / (rank - 1))


def low_rank_matrix(m: int, n: int, rank: int, seed: int, sigma=None, noise: float = 0.0,
                    device: str = "cpu", dtype=None):
    """A = U0 diag(sigma) V0* (+ noise * N(0, 1) entries) with U0, V0
    orthonormal (QR of Gaussian matrices), the shape of the paper's random
    rank-50 test matrix. Returns (A, sigma, U0, V0): numpy FP64 on the CPU;
    on a CUDA device, torch tensors (A in dtype, default float32) built with
    torch on that device (the paper's 1,000,000 x 30,000 size needs 120 GB
    in FP32, so it is generated where it is used)."""
    sigma = planted_spectrum(rank) if sigma is None else np.asarray(sigma, np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    if device == "cpu":
        U0, _ = np.linalg.qr(rng.standard_normal((m, rank)))
        V0, _ = np.linalg.qr(rng.standard_normal((n, rank)))
        A = (U0 * sigma) @ V0.T
        if noise:
            A += noise * rng.standard_normal((m, n))
        if dtype is not None:
            A = A.astype(dtype)
        return A, sigma, U0, V0
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    # orthonormal factors by numpy's QR on the host (m x rank and n x rank are small)
    U0 = torch.as_tensor(np.linalg.qr(rng.standard_normal((m, rank)))[0], device=device)
    V0 = torch.as_tensor(np.linalg.qr(rng.standard_normal((n, rank)))[0], device=device)
    s = torch.as_tensor(sigma, device=device)
    dt = dtype or torch.float32
    A = torch.empty((m, n), device=device, dtype=dt)
    step = max(1, (1 << 28) // max(1, n))  # rows per slab of the product (FP64 slab <= 2 GB)
    for r0 in range(0, m, step):
        slab = (U0[r0:r0 + step] * s) @ V0.T
        if noise:
            slab += noise * torch.randn(slab.shape, generator=g, device=device, dtype=torch.float64)
        A[r0:r0 + step] = slab.to(dt)
    return A, sigma, U0, V0


def omega(n: int, l: int, seed: int) -> np.ndarray:
    """Omega of Algorithm oocPCA: n x l uniform on [-1, 1) (FP64)."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    return rng.uniform(-1.0, 1.0, size=(n, l))
