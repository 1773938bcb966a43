"""t-SNE heatmaps (Sec. 5) on the GPU, through the C ABI, against the oracle
on the same seeded inputs.

What is compared:
  - cells per bin: exactly (the bin of a cell is decided in FP32 by the same
    rounded operations on both sides);
  - H (gene x bin sums): the GPU sums in FP64 with atomics, in an order that
    varies; for non-negative values every partial sum is below the final one,
    so each entry is within (n - 1) u H of the exact sum (n terms, u = 2^-53):
    below 1e-11 relative for the sizes here (n <= 10^5), tested at 1e-11;
  - distances |h_q - h_g|: both sides start from such H, so a distance
    differs by at most ~1e-11 (|h_q| + |h_g|) (the test's bound);
  - nearest genes: equal, except where two candidates' oracle distances are
    within that bound of each other (a near-tie either order may take).
"""
import numpy as np
import pytest
import torch

from oracle import heatmap as ohm
import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs
from paper_1712_09005_gb300._abi import TsneError, TSNE_ERR_INVALID_ARG, TSNE_ERR_NONFINITE

pytestmark = pytest.mark.gpu

RTOL_H = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_heatmap(y, row_ptr, col, val, G, n_bins, goi=None, m=4):
    E = pkg.DeviceCSR.from_host(row_ptr, col, val)
    yd = torch.as_tensor(np.asarray(y, np.float32), device="cuda")
    with pkg.Heatmap(n_bins, G, max_goi=max(1, len(goi) if goi is not None else 1)) as hm:
        H, counts = hm.bin(yd, E)
        near = hm.nearest(H, goi, m) if goi is not None else None
        assert hm.launch_count() >= 2
        ph = hm.phase_ms()
        assert ph["bin_sums"] >= 0.0
        return H.cpu().numpy(), counts.cpu().numpy(), near


def check_nearest(Ho, goi, m, idx, dist):
    D = ohm.gene_distances(Ho, goi)
    scale = np.sqrt((Ho ** 2).sum(0))
    for r, q in enumerate(goi):
        tol = RTOL_H * (scale[q] + scale[idx[r]]) + 1e-300
        np.testing.assert_allclose(dist[r], D[r, idx[r]], rtol=0, atol=float(tol.max()) * 4)
        oi, od = ohm.nearest(Ho, [q], m)
        if idx[r].tolist() != oi[0].tolist():
            # every difference must be a near-tie at the m-th distance
            kth = od[0, -1]
            for g in set(idx[r].tolist()) ^ set(oi[0].tolist()):
                assert abs(D[r, g] - kth) <= RTOL_H * 8 * (scale[q] + scale[g])
        assert np.all(np.diff(dist[r]) >= -float(tol.max()) * 4)
        assert q not in idx[r].tolist()


def log_normalised(e):
    """log(1 + 10^4 x / cell total): non-integer values (the usual scRNA-seq
    normalisation), so the FP64 sums round."""
    tot = np.add.reduceat(e.val.astype(np.float64), e.row_ptr[:-1]) if e.val.size else np.zeros(0)
    per = np.repeat(tot, np.diff(e.row_ptr))
    return np.log1p(1e4 * e.val / per).astype(np.float32)


@pytest.mark.parametrize("N,G,n_bins,seed", [
    (5003, 1501, 37, 1),    # ragged against warps and blocks
    (2048, 300, 1, 2),      # one bin: H = gene totals
    (777, 64, 500, 3),      # more bins than cells fill (many empty bins)
])
@pytest.mark.parametrize("norm", [False, True])
def test_matches_oracle(N, G, n_bins, seed, norm):
    e = inputs.expression(N, G, mean_genes=60, n_clusters=9, markers=6, seed=seed)
    if norm:
        e.val = log_normalised(e)
    goi = [0, G // 3, G - 1]  # the paper's example: three genes, each with its 4 nearest
    H, counts, (idx, dist) = gpu_heatmap(e.y, e.row_ptr, e.col, e.val, G, n_bins, goi, 4)
    Ho, co = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, G, n_bins)
    assert counts.tolist() == co.tolist()
    np.testing.assert_allclose(H, Ho, rtol=RTOL_H, atol=0)
    check_nearest(Ho, goi, 4, idx, dist)


def test_integer_counts_are_exact_and_repeatable():
    """Counts are integers: every partial sum is exact in FP64, so H equals the
    oracle bit for bit and two calls agree bit for bit."""
    e = inputs.expression(3000, 400, mean_genes=80, n_clusters=5, seed=7)
    H1, c1, _ = gpu_heatmap(e.y, e.row_ptr, e.col, e.val, 400, 25)
    H2, c2, _ = gpu_heatmap(e.y, e.row_ptr, e.col, e.val, 400, 25)
    Ho, co = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, 400, 25)
    assert np.array_equal(H1, Ho) and np.array_equal(H2, Ho)
    assert np.array_equal(c1, co) and np.array_equal(c2, co)


def test_fp32_bin_decision_and_degenerate_layouts():
    # y = fl(10/3) falls in bin 1 of 3 by the FP32 rule (bin 0 in exact arithmetic)
    y = np.array([0.0, np.float32(10.0) / np.float32(3.0), 10.0], np.float32)
    rp = np.array([0, 1, 2, 3], np.int32)
    col = np.array([0, 1, 2], np.int32)
    val = np.array([1.0, 2.0, 4.0], np.float32)
    H, counts, _ = gpu_heatmap(y, rp, col, val, 3, 3)
    assert counts.tolist() == [1, 1, 1]
    assert H.tolist() == [[1, 0, 0], [0, 2, 0], [0, 0, 4]]
    # one cell; all cells equal; cells without any expressed gene
    H, counts, _ = gpu_heatmap(np.array([3.5], np.float32), np.array([0, 2], np.int32),
                               np.array([0, 4], np.int32), np.array([1.5, 2.5], np.float32), 5, 8)
    assert counts.tolist() == [1] + [0] * 7 and H[0].tolist() == [1.5, 0, 0, 0, 2.5]
    y = np.full(40, -2.0, np.float32)
    rp = np.zeros(41, np.int32)  # no expression at all
    H, counts, _ = gpu_heatmap(y, rp, np.zeros(0, np.int32), np.zeros(0, np.float32), 6, 4)
    assert counts.tolist() == [40, 0, 0, 0] and not H.any()


def test_errors_are_reported():
    e = inputs.expression(500, 50, mean_genes=10, n_clusters=3, seed=8)
    E = pkg.DeviceCSR.from_host(*e.as_tuple())
    with pkg.Heatmap(10, 50, max_goi=2) as hm:
        y = torch.as_tensor(e.y.copy(), device="cuda")
        y[7] = float("nan")
        with pytest.raises(TsneError) as ex:
            hm.bin(y, E)
        assert ex.value.code == TSNE_ERR_NONFINITE
        H, _ = hm.bin(torch.as_tensor(e.y, device="cuda"), E)
        for goi, m in (([50], 2), ([-1], 2), ([0], 0), ([0], 50), ([0, 1, 2], 2)):
            with pytest.raises(TsneError) as ex:
                hm.nearest(H, goi, m)
            assert ex.value.code == TSNE_ERR_INVALID_ARG
    with pkg.Heatmap(10, 40, max_goi=1) as hm:  # gene indices up to 49 with G = 40
        with pytest.raises(TsneError) as ex:
            hm.bin(torch.as_tensor(e.y, device="cuda"), E)
        assert ex.value.code == TSNE_ERR_INVALID_ARG


def test_bench_size_sampled():
    """The benchmark's shape (N = 50,000 cells, G = 25,000 genes, ~940 genes
    per cell, 100 bins): counts exactly, H on 64 sampled genes, and the
    nearest genes of three genes of interest against the oracle's full H."""
    N, G, n_bins = 50_000, 25_000, 100
    e = inputs.expression(N, G, mean_genes=1000, n_clusters=20, seed=5000)
    goi = [11, 12_345, 24_999]
    H, counts, (idx, dist) = gpu_heatmap(e.y, e.row_ptr, e.col, e.val, G, n_bins, goi, 4)
    Ho, co = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, G, n_bins)
    assert counts.tolist() == co.tolist()
    g = np.random.default_rng(0).choice(G, 64, replace=False)
    np.testing.assert_allclose(H[:, g], Ho[:, g], rtol=RTOL_H, atol=0)
    check_nearest(Ho, goi, 4, idx, dist)
