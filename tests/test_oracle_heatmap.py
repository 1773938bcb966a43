"""Pins of the oracle's t-SNE heatmaps (Sec. 5): bins of the 1-D embedding,
gene x bin sums, gene distances and nearest genes, each against something
other than the oracle itself (hand-worked values, a sparse one-hot product,
scipy's cdist, brute force, invariants)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial.distance import cdist

from oracle import heatmap as ohm
from paper_1712_09005_gb300 import inputs


def test_bins_worked_examples():
    # w = 2, 1 / w = 0.5 exactly: t = 0, 0.5, 1, 1.5, 2 -> the top edge joins the last bin
    assert ohm.bins(np.array([-2, -1, 0, 1, 2], np.float32), 2).tolist() == [0, 0, 1, 1, 1]
    # w = 1: integer coordinates sit on the lower edge of their bin
    assert ohm.bins(np.array([0, 1, 2, 3, 4], np.float32), 4).tolist() == [0, 1, 2, 3, 3]
    # one bin, one cell, all cells equal (w = 0)
    assert ohm.bins(np.array([5, -3, 7], np.float32), 1).tolist() == [0, 0, 0]
    assert ohm.bins(np.array([1.5], np.float32), 10).tolist() == [0]
    assert ohm.bins(np.full(6, 2.25, np.float32), 8).tolist() == [0] * 6
    # order of the cells does not matter
    y = np.array([4, 0, 3, 1, 2], np.float32)
    assert ohm.bins(y, 4).tolist() == [3, 0, 3, 1, 2]


def test_bin_is_decided_in_fp32():
    """max - min = 10, 3 bins: w = fl(10/3) = 3.33333325..., 1/w = fl(0.3000000119...).
    For y = fl(10/3) the FP32 product rounds up to exactly 1 (bin 1), while
    exact arithmetic gives y / w_exact = 0.99999998 (bin 0); the rule is the
    FP32 one, which the GPU follows."""
    y = np.array([0.0, np.float32(10.0) / np.float32(3.0), 10.0], np.float32)
    assert float(y[1]) * 0.3 < 1.0  # the exact ratio is below 1
    assert ohm.bins(y, 3).tolist() == [0, 1, 2]


def test_bins_are_monotone_and_cover_every_bin():
    rng = np.random.default_rng(2)
    y = rng.normal(size=5000).astype(np.float32)
    b = ohm.bins(y, 50)
    order = np.argsort(y, kind="stable")
    assert np.all(np.diff(b[order]) >= 0)
    assert b.min() == 0 and b.max() == 49
    yl = np.linspace(-1, 1, 1001).astype(np.float32)
    assert np.bincount(ohm.bins(yl, 10), minlength=10).min() > 90


def _small(N=700, G=90, seed=3):
    return inputs.expression(N, G, mean_genes=25, n_clusters=6, markers=8, seed=seed)


def test_sums_equal_the_one_hot_product():
    """H = B^T E with B the cells x bins one-hot matrix (a sparse product)."""
    e = _small()
    n_bins = 13
    H, counts = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, e.G, n_bins)
    N = e.y.size
    b = ohm.bins(e.y, n_bins)
    B = sp.csr_matrix((np.ones(N), (np.arange(N), b)), shape=(N, n_bins))
    E = sp.csr_matrix((e.val.astype(np.float64), e.col, e.row_ptr), shape=(N, e.G))
    np.testing.assert_allclose(H, (B.T @ E).toarray(), rtol=1e-13, atol=0)
    assert counts.tolist() == np.bincount(b, minlength=n_bins).tolist()
    # invariants: every gene's total expression and every cell are counted once
    np.testing.assert_allclose(H.sum(0), np.asarray(E.sum(0)).ravel(), rtol=1e-13)
    assert counts.sum() == N


def test_integer_counts_are_summed_exactly():
    e = _small(seed=4)
    H, _ = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, e.G, 7)
    assert np.all(H == np.round(H))
    assert H.sum() == e.val.astype(np.float64).sum()


def test_distances_match_cdist_and_metric_axioms():
    e = _small(seed=5)
    H, _ = ohm.gene_bin_sums(e.y, e.row_ptr, e.col, e.val, e.G, 11)
    goi = [0, 17, 42]
    D = ohm.gene_distances(H, goi)
    np.testing.assert_allclose(D, cdist(H.T[goi], H.T), rtol=1e-12, atol=1e-9)
    for r, q in enumerate(goi):
        assert D[r, q] == 0.0
    full = ohm.gene_distances(H, list(range(e.G)))
    np.testing.assert_allclose(full, full.T, rtol=1e-12, atol=1e-9)
    i, j, k = 3, 50, 77
    assert full[i, k] <= full[i, j] + full[j, k] + 1e-9


def test_nearest_planted_and_brute_force():
    n_bins, G = 6, 12
    rng = np.random.default_rng(6)
    H = rng.uniform(10, 20, size=(n_bins, G))
    H[:, 5] = H[:, 0] + 0.5          # nearest to gene 0 ...
    H[:, 3] = H[:, 0] + 0.5          # ... tied with gene 5: the smaller index first
    H[:, 9] = H[:, 0] - 1.0          # then gene 9
    idx, dist = ohm.nearest(H, [0], 3)
    assert idx[0].tolist() == [3, 5, 9]
    np.testing.assert_allclose(dist[0], [0.5 * np.sqrt(n_bins)] * 2 + [np.sqrt(n_bins)], rtol=1e-14)
    # brute force on random data, several genes of interest, the gene itself excluded
    H = rng.normal(size=(9, 40))
    goi = [1, 7, 39]
    idx, dist = ohm.nearest(H, goi, 5)
    for r, q in enumerate(goi):
        d = np.sqrt(((H - H[:, [q]]) ** 2).sum(0))
        d[q] = np.inf
        want = np.lexsort((np.arange(40), d))[:5]
        assert idx[r].tolist() == want.tolist()
        np.testing.assert_allclose(dist[r], d[want], rtol=1e-13)


def test_rejects_non_finite_embedding():
    with pytest.raises(ValueError):
        ohm.bins(np.array([0.0, np.nan], np.float32), 3)


def test_expression_generator_is_a_valid_count_matrix():
    """The synthetic cells x genes counts: a well-formed CSR (rows in cell
    order, distinct sorted genes per row, positive integer counts), seeded,
    with a 1-D layout that keeps each cluster's cells together."""
    e = inputs.expression(1500, 300, mean_genes=40, n_clusters=5, markers=6, seed=9)
    assert e.row_ptr[0] == 0 and np.all(np.diff(e.row_ptr) >= 1)
    assert e.row_ptr[-1] == e.col.size == e.val.size
    for i in range(e.y.size):
        c = e.col[e.row_ptr[i]:e.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < e.G
    assert np.all(e.val >= 1) and np.all(e.val == np.round(e.val))
    again = inputs.expression(1500, 300, mean_genes=40, n_clusters=5, markers=6, seed=9)
    assert np.array_equal(again.col, e.col) and np.array_equal(again.y, e.y)
    # clusters sit 10 apart with unit spread: each cluster's cells span < 10
    for c in range(5):
        yc = e.y[e.label == c]
        assert yc.max() - yc.min() < 10.0
