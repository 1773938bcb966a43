"""Oracle input affinities P (Sec. 1.1, Eq. p_ij), plain FP64 numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py). Written independently of the
product's input generator so that the generator can be checked against it.

  p_{j|i} = exp(-|x_i - x_j|^2 / 2 sigma_i^2) / sum_{k != i} exp(-|x_i - x_k|^2 / 2 sigma_i^2)
  p_ij    = (p_{j|i} + p_{i|j}) / (2N)

restricted, as in Sec. 3, to the k exact nearest neighbours of each point.
sigma_i is set by bisection on beta_i = 1 / (2 sigma_i^2) so that the
perplexity exp(H(P_i)) (natural log) matches the target; the paper gives no
tolerance, so bisection stops at |H - log(perplexity)| < 1e-5 or after 200
steps (a reading, see the design notes).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def exact_knn(X: np.ndarray, k: int):
    """k nearest neighbours of every row of X (Euclidean, FP64, self excluded).

    Ties are broken by the smaller index. Returns (idx N x k int64, d2 N x k).
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    if k >= N:
        raise ValueError("k must be < N")
    sq = np.einsum("ij,ij->i", X, X)
    idx = np.empty((N, k), dtype=np.int64)
    d2 = np.empty((N, k), dtype=np.float64)
    for start in range(0, N, 512):
        stop = min(N, start + 512)
        D = sq[start:stop, None] + sq[None, :] - 2.0 * X[start:stop] @ X.T
        np.maximum(D, 0.0, out=D)
        D[np.arange(stop - start), np.arange(start, stop)] = np.inf
        order = np.argsort(D, axis=1, kind="stable")[:, :k]
        idx[start:stop] = order
        d2[start:stop] = np.take_along_axis(D, order, axis=1)
    return idx, d2


def calibrate(d2: np.ndarray, perplexity: float, tol: float = 1e-5, max_iter: int = 200):
    """Bisection on beta per row so that exp(H(P_i)) = perplexity.

    d2 is N x k squared distances to the neighbours. Returns (P_cond, beta).
    """
    N, k = d2.shape
    target = np.log(perplexity)
    shifted = d2 - d2[:, :1]  # the normalisation cancels any per-row shift
    beta = np.ones(N)
    lo = np.full(N, -np.inf)
    hi = np.full(N, np.inf)
    done = np.zeros(N, dtype=bool)
    P = np.empty_like(d2)
    for _ in range(max_iter):
        E = np.exp(-beta[:, None] * shifted)
        S = E.sum(axis=1)
        P = E / S[:, None]
        H = np.log(S) + beta * (P * shifted).sum(axis=1)
        done |= np.abs(H - target) < tol
        if done.all():
            break
        up = (H > target) & ~done   # too flat: sharpen
        down = (H <= target) & ~done
        lo[up] = beta[up]
        beta[up] = np.where(np.isinf(hi[up]), beta[up] * 2.0, (beta[up] + hi[up]) / 2.0)
        hi[down] = beta[down]
        beta[down] = np.where(np.isinf(lo[down]), beta[down] / 2.0, (beta[down] + lo[down]) / 2.0)
    E = np.exp(-beta[:, None] * shifted)
    P = E / E.sum(axis=1, keepdims=True)
    return P, beta


def perplexity_of(P_cond: np.ndarray) -> np.ndarray:
    """exp of the Shannon entropy (natural log) of each row."""
    with np.errstate(divide="ignore", invalid="ignore"):
        H = -np.where(P_cond > 0, P_cond * np.log(P_cond), 0.0).sum(axis=1)
    return np.exp(H)


def build_P(X: np.ndarray, perplexity: float = 30.0, k: int | None = None):
    """Symmetric, normalised kNN affinities as CSR (row_ptr, col, val).

    k defaults to 3 * perplexity. Values are FP64 here; the caller casts.
    Columns are sorted within each row; there are no diagonal entries.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    if k is None:
        k = int(3 * perplexity)
    idx, d2 = exact_knn(X, k)
    Pc, _ = calibrate(d2, perplexity)
    rows = np.repeat(np.arange(N), k)
    C = sp.csr_matrix((Pc.ravel(), (rows, idx.ravel())), shape=(N, N))
    S = ((C + C.T) / (2.0 * N)).tocsr()
    S.sort_indices()
    S.eliminate_zeros()
    return S.indptr.astype(np.int64), S.indices.astype(np.int64), S.data.astype(np.float64)
