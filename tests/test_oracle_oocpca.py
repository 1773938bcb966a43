"""Pins of the oocPCA oracle (Sec. 6, Algorithm oocPCA) against what the
mathematics fixes, independent of the oracle's own code:

* a planted rank-r matrix (r <= k): the singular values are the planted
  ones, U and V span the planted subspaces, and the residual is zero;
* a full-rank matrix with a decaying spectrum: the top-k singular values and
  vectors agree with a dense SVD (LAPACK through numpy) within the
  randomized error bound (tiny here: the spectrum decays fast);
* blocking: the result does not depend on b;
* the LU renormalization: Y = L U with |L| <= 1 (partial pivoting);
* column centring equals the oracle on the explicitly centred matrix, and
  the leading singular vector of a centred rank-one cloud is its direction;
* the power iterations matter: with its = 0 the error against the dense SVD
  is much larger than with its = 2 on a slowly decaying spectrum.
"""
import numpy as np
import pytest

from oracle import oocpca as ooc
from paper_1712_09005_gb300 import inputs


def subspace_cos(U, U0):
    """Cosines of the principal angles between span(U) and span(U0)."""
    return np.linalg.svd(U.T @ U0, compute_uv=False)


@pytest.mark.parametrize("its", [0, 1, 2])
def test_planted_rank_is_recovered(its):
    m, n, r, k = 700, 300, 8, 8
    A, sig, U0, V0 = inputs.low_rank_matrix(m, n, r, seed=3)
    Om = inputs.omega(n, k + 2, seed=3)
    U, s, V = ooc.oocpca(A, k, its, Om, b=64)
    assert np.allclose(s, sig, rtol=1e-11, atol=0)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-12)
    assert np.all(subspace_cos(U, U0) > 1 - 1e-12)
    assert np.all(subspace_cos(V, V0) > 1 - 1e-12)
    assert ooc.spectral_error(A, U, s, V) <= 1e-11 * sig[0]


def test_matches_dense_svd_on_decaying_spectrum():
    m, n, k = 500, 260, 10
    rng = np.random.default_rng(5)
    Ud, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vd, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = 0.6 ** np.arange(n)
    A = (Ud * sig) @ Vd.T
    U, s, V = ooc.oocpca(A, k, 2, inputs.omega(n, k + 2, seed=5), b=100)
    Uf, sf, Vfh = np.linalg.svd(A, full_matrices=False)
    # randomized bound with l = k + 2 and 2 power iterations: the error in
    # sigma_j is of order (sigma_{k+1} / sigma_j)^(2 its + 1) sigma_j
    assert np.allclose(s, sf[:k], rtol=1e-6)
    assert np.allclose(s[:5], sf[:5], rtol=1e-12)
    # vectors up to sign
    for j in range(5):
        assert abs(abs(U[:, j] @ Uf[:, j]) - 1) < 1e-10
        assert abs(abs(V[:, j] @ Vfh[j]) - 1) < 1e-10
    # the residual is the (k+1)-th singular value, up to the same bound
    assert ooc.spectral_error(A, U, s, V) <= 1.01 * sf[k]


def test_power_iterations_sharpen_a_slow_spectrum():
    m, n, k = 400, 200, 6
    rng = np.random.default_rng(9)
    Ud, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vd, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = 1.0 / (1.0 + np.arange(n)) ** 0.5
    A = (Ud * sig) @ Vd.T
    sf = np.linalg.svd(A, compute_uv=False)
    Om = inputs.omega(n, k + 2, seed=9)
    e0 = np.abs(ooc.oocpca(A, k, 0, Om)[1] - sf[:k]).max()
    e2 = np.abs(ooc.oocpca(A, k, 2, Om)[1] - sf[:k]).max()
    assert e2 < 0.25 * e0


def test_blocking_does_not_change_the_result():
    A, _, _, _ = inputs.low_rank_matrix(331, 120, 12, seed=11, noise=1e-3)
    Om = inputs.omega(120, 9, seed=11)
    a = ooc.oocpca(A, 7, 2, Om, b=331)
    for b in (1, 37, 100):
        c = ooc.oocpca(A, 7, 2, Om, b=b)
        assert np.allclose(a[1], c[1], rtol=1e-12)
        assert np.allclose(np.abs(a[0].T @ c[0]), np.eye(7), atol=1e-9)


def test_lu_renormalization_properties():
    Y = np.random.default_rng(2).standard_normal((50, 7))
    L, U = ooc.lu_renormalize(Y)
    assert np.allclose(L @ U, Y, atol=1e-13)
    assert np.all(np.abs(L) <= 1 + 1e-15)
    assert np.allclose(U, np.triu(U))
    # L is a row permutation of a unit lower-trapezoidal matrix
    piv = [int(np.argmax(np.isclose(L[:, j], 1.0) & np.all(np.abs(L[:, j + 1:]) == 0, axis=1)))
           for j in range(7)]
    assert len(set(piv)) == 7


def test_column_centring():
    m, n = 400, 90
    rng = np.random.default_rng(4)
    direction = rng.standard_normal(n)
    direction /= np.linalg.norm(direction)
    t = rng.standard_normal(m) * 5.0
    A = 3.0 + np.outer(t, direction) + 1e-3 * rng.standard_normal((m, n))
    Om = inputs.omega(n, 4, seed=4)
    U, s, V = ooc.oocpca(A, 2, 2, Om, center=True)
    Uc, sc, Vc = ooc.oocpca(A - A.mean(axis=0), 2, 2, Om)
    assert np.allclose(s, sc, rtol=1e-12)
    assert abs(abs(V[:, 0] @ direction) - 1) < 1e-6
    # without centring the constant offset dominates the first component
    _, s_raw, V_raw = ooc.oocpca(A, 2, 2, Om)
    assert abs(V_raw[:, 0] @ np.ones(n)) / np.sqrt(n) > 0.5


def test_argument_checks():
    A = np.zeros((10, 8))
    with pytest.raises(ValueError):
        ooc.oocpca(A, 0, 1, np.zeros((8, 2)))
    with pytest.raises(ValueError):
        ooc.oocpca(A, 3, 1, np.zeros((8, 2)))
    with pytest.raises(ValueError):
        ooc.oocpca(A, 2, 1, np.zeros((7, 3)))
