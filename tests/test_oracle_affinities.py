"""Pins of the oracle's input affinities (Sec. 1.1, Eq. p_ij) and the check
of the product's input generator against them."""
import numpy as np
import pytest

from oracle import affinities as oaff


def test_perplexity_symmetry_normalisation():
    from paper_1712_09005_gb300 import inputs
    X = inputs.mixture(N=600, n_clusters=4, seed=11)
    idx, d2 = oaff.exact_knn(X, 45)
    Pc, beta = oaff.calibrate(d2, 15.0)
    np.testing.assert_allclose(oaff.perplexity_of(Pc), 15.0, rtol=1e-4)
    np.testing.assert_allclose(Pc.sum(1), 1.0, rtol=1e-12)
    rp, col, val = oaff.build_P(X, 15.0)
    N = 600
    import scipy.sparse as sp
    S = sp.csr_matrix((val, col, rp), shape=(N, N))
    assert abs(S.sum() - 1.0) < 1e-12
    assert abs(S - S.T).max() < 1e-15
    assert S.diagonal().max() == 0.0
    assert (val > 0).all()


def test_knn_brute_force():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(50, 7))
    idx, d2 = oaff.exact_knn(X, 6)
    for i in range(50):
        d = ((X - X[i]) ** 2).sum(1)
        d[i] = np.inf
        order = sorted(range(50), key=lambda j: (d[j], j))[:6]
        assert list(idx[i]) == order
        np.testing.assert_allclose(d2[i], d[order], rtol=1e-12)


def test_full_neighbourhood_matches_definition():
    """k = N - 1: p_{j|i} over all other points, bisected to the target perplexity."""
    rng = np.random.default_rng(4)
    X = rng.normal(size=(25, 3))
    idx, d2 = oaff.exact_knn(X, 24)
    Pc, beta = oaff.calibrate(d2, 5.0)
    for i in range(25):
        e = np.exp(-beta[i] * d2[i])
        np.testing.assert_allclose(Pc[i], e / e.sum(), rtol=1e-12)


def test_product_generator_matches_oracle():
    """The product's torch affinity builder reproduces the oracle's P."""
    from paper_1712_09005_gb300 import inputs
    X = inputs.mixture(N=800, n_clusters=5, seed=21)
    rp, col, val = oaff.build_P(X.astype(np.float64), 30.0)
    Pg = inputs.affinities(X, 30.0, device="cpu")
    assert np.array_equal(Pg.row_ptr, rp) and np.array_equal(Pg.col, col)
    np.testing.assert_allclose(Pg.val, val, rtol=2e-6)
    assert Pg.row_ptr.dtype == np.int32 and Pg.col.dtype == np.int32 and Pg.val.dtype == np.float32
