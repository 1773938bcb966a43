"""Oracle t-SNE heatmaps (Sec. 5), plain numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py): only the tests, smoke() and the
CPU legs of bench.py use it; it shares no code with the CUDA library.

Sec. 5 cuts the cells' 1-D t-SNE embedding into bins, sums each gene's
expression over the cells of every bin (gene g -> a vector h_g with one entry
per bin), compares genes by the Euclidean distance between those vectors, and
enriches each gene of interest with the genes closest to it; the vectors of
that gene set are the heatmap's rows. The paper does not say how the bins are
cut; the reading used here is equal-width bins over [min y, max y]:

  w = (max y - min y) / n_bins,   bin(y) = floor((y - min y) * (1 / w)),

each operation rounded once in FP32 (round to nearest, no fused multiply-add)
because the result is an integer decision that the GPU must take the same
way; bins are clamped to [0, n_bins - 1], and w = 0 (or 1 / w not finite)
puts every cell in bin 0. Everything after the bin decision is FP64. Nearest
genes exclude the gene itself; equal distances are ordered by gene index.
"""
from __future__ import annotations

import numpy as np


def bins(y, n_bins: int) -> np.ndarray:
    """Bin index of every cell (int64), decided in FP32 as described above."""
    y = np.asarray(y, dtype=np.float32)
    if y.size == 0:
        return np.zeros(0, np.int64)
    if not np.all(np.isfinite(y)):
        raise ValueError("non-finite coordinate")
    lo, hi = np.float32(y.min()), np.float32(y.max())
    w = np.float32(np.float32(hi - lo) / np.float32(n_bins))
    inv = np.float32(0.0)
    if w > 0:
        with np.errstate(over="ignore"):
            inv = np.float32(np.float32(1.0) / w)
        if not np.isfinite(inv):
            inv = np.float32(0.0)
    t = (y - lo).astype(np.float32) * inv
    t = t.astype(np.float32)
    b = np.zeros(y.size, np.int64)
    ok = t >= 0
    b[ok] = np.minimum(np.floor(t[ok]).astype(np.int64), n_bins - 1)
    return b


def gene_bin_sums(y, row_ptr, col, val, G: int, n_bins: int):
    """H[b, g] = sum of E[i, g] over the cells i of bin b (FP64), and the
    number of cells per bin. E is a cells x genes CSR (row_ptr, col, val)."""
    b = bins(y, n_bins)
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    val = np.asarray(val, np.float64)
    cell = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    H = np.zeros((n_bins, G), np.float64)
    np.add.at(H, (b[cell], col), val)
    counts = np.bincount(b, minlength=n_bins).astype(np.int64)
    return H, counts


def gene_distances(H, goi) -> np.ndarray:
    """|h_q - h_g| for every gene of interest q (rows) and every gene g."""
    H = np.asarray(H, np.float64)
    out = np.empty((len(goi), H.shape[1]), np.float64)
    for r, q in enumerate(goi):
        d = H - H[:, [q]]
        out[r] = np.sqrt(np.einsum("bg,bg->g", d, d))
    return out


def nearest(H, goi, m: int):
    """The m genes nearest to each gene of interest (itself excluded), in
    increasing (distance, gene index); returns (idx, dist), n_goi x m."""
    D = gene_distances(H, goi)
    G = D.shape[1]
    idx = np.empty((len(goi), m), np.int64)
    dist = np.empty((len(goi), m), np.float64)
    for r, q in enumerate(goi):
        order = sorted((g for g in range(G) if g != q), key=lambda g: (D[r, g], g))[:m]
        idx[r] = order
        dist[r] = D[r, order]
    return idx, dist
