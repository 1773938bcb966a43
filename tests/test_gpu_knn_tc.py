"""The tensor-core kNN (shortlists from 3xTF32 tile products, exact FP32
re-rank) against the row kernel: the same neighbour lists and the same FP32
distances, bit for bit, on every input; the queries it cannot prove complete
(exact ties beyond its shortlist, non-finite data) go to the row kernel, and
on ordinary data there are none, so the tensor-core path is the one that
produced the lists.

The row kernel's lists are themselves pinned to the oracle's FP64 kNN by
tests/test_gpu_affinity.py (which also runs every oracle case with this
kernel)."""
import numpy as np
import pytest
import torch

import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def knn(X, k, kernel, monkeypatch, perplexity=None):
    monkeypatch.setenv("FITSNE_KNN_KERNEL", kernel)
    N, D = X.shape
    with pkg.Affinity(N, D, k) as aff:
        P = aff.compute(torch.as_tensor(X, device="cuda"), perplexity or max(1.0, k / 3.0))
        torch.cuda.synchronize()
        vals = P.val.cpu().numpy().copy()
        idx, d2, _ = aff.knn()
        info = aff.knn_info()
    assert info["kernel"] == kernel
    return idx, d2, vals, info


def same_as_rows(X, k, monkeypatch, max_recomputed=0):
    it, dt, vt, info = knn(X, k, "tc", monkeypatch)
    ir, dr, vr, _ = knn(X, k, "rows", monkeypatch)
    assert np.array_equal(it, ir)
    assert np.array_equal(dt.view(np.uint32), dr.view(np.uint32))
    assert np.array_equal(vt.view(np.uint32), vr.view(np.uint32))
    assert info["recomputed"] <= max_recomputed, info
    return info


@pytest.mark.parametrize("N,D,k,seed,left", [
    (3001, 50, 90, 1, 0),     # several query and candidate tiles, ragged tail
    (1537, 3, 30, 2, 0),      # low dimension: one K-step
    (2000, 64, 150, 3, 0),    # D at its maximum, eight K-steps, the norm added in FP32
    (1000, 10, 256, 4, 0),    # k at its maximum
    (200, 33, 1, 5, 0),       # k = 1, D just past one 32-column chunk
    (91, 20, 90, 6, 0),       # N = k + 1: every other point
    # D = 1: one K-step, the norm in column 1; coordinates up to ~15 give a
    # band (6e-5 of the norms) wider than the neighbour spacing, so the final
    # shortlists of the dense clusters overflow their 128-entry slots and go
    # to the row kernel (still the same lists)
    (3000, 1, 30, 13, 3000),
    (2500, 63, 2, 14, 0),     # D = 63: the norm in the last column, eight K-steps
    (2049, 56, 90, 15, 0),    # D = 56: with the norm column, 57 columns round up to 64
])
def test_tc_equals_rows_on_mixtures(N, D, k, seed, left, monkeypatch):
    X = inputs.mixture(N=N, n_clusters=7, dim=D, seed=seed)
    same_as_rows(X, k, monkeypatch, max_recomputed=left)


def test_far_from_origin_is_centred(monkeypatch):
    """An offset of 1000 in every coordinate: without centring the products'
    cancellation would leave no usable shortlist; the centre removes it."""
    X = inputs.mixture(N=2500, n_clusters=5, dim=50, seed=7) + np.float32(1000.0)
    same_as_rows(X, 90, monkeypatch)


def test_exact_ties_beyond_the_shortlist_go_to_the_row_kernel(monkeypatch):
    """600 copies of one point: each copy has 599 candidates at distance 0,
    more than a shortlist can hold, so those queries are recomputed by the
    row kernel; the other queries are not."""
    X = inputs.mixture(N=3000, n_clusters=5, dim=16, seed=8)
    X[1000:1600] = X[1000]
    info = same_as_rows(X, 30, monkeypatch, max_recomputed=3000)
    assert 600 <= info["recomputed"] < 3000


def test_integer_data_with_duplicates(monkeypatch):
    rng = np.random.default_rng(9)
    X = rng.integers(0, 4, size=(1200, 6)).astype(np.float32)
    X[600:700] = X[0:100]
    same_as_rows(X, 15, monkeypatch, max_recomputed=1200)


def test_non_finite_row_sends_every_query_to_the_row_kernel(monkeypatch):
    X = inputs.mixture(N=700, n_clusters=3, dim=8, seed=10)
    X[17, 3] = np.nan
    info = same_as_rows(X, 30, monkeypatch, max_recomputed=700)
    assert info["recomputed"] == 700


def test_large_ragged_n_bitwise(monkeypatch):
    """N = 131,101 (1025 query tiles, a ragged last one), D = 50, k = 90."""
    X = inputs.mixture(N=131_101, n_clusters=10, dim=50, seed=11)
    same_as_rows(X, 90, monkeypatch)


def test_default_choice_and_repeatability(monkeypatch):
    monkeypatch.delenv("FITSNE_KNN_KERNEL", raising=False)
    X = torch.as_tensor(inputs.mixture(N=40_000, n_clusters=6, dim=50, seed=12), device="cuda")
    with pkg.Affinity(40_000, 50, 90) as aff:
        a = aff.compute(X, 30.0).val.cpu().numpy().copy()
        b = aff.compute(X, 30.0).val.cpu().numpy().copy()
        assert aff.knn_info() == {"kernel": "tc", "recomputed": 0}
    assert np.array_equal(a, b)
