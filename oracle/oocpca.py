"""Oracle out-of-core randomized PCA (Sec. 6, Algorithm oocPCA), plain numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py): only the tests, smoke() and the
CPU legs of bench.py use it; it shares no code with the CUDA library.

Everything is FP64. The steps follow Algorithm oocPCA in the paper's order:

  1. Omega, n x l uniform random (drawn by the caller and passed in, so that
     the GPU path and this oracle start from the same vectors);
  2. Y_0 = A Omega, formed b rows of A at a time;
  3. L_0 U_0 = Y_0, the LU factorization with partial pivoting (L_0 holds the
     row permutation: L_0 = P L for Y_0 = P L U);
  4. for i = 1 .. its: Y_i = A A* L_{i-1}, formed b rows at a time; for
     i < its, L_i U_i = Y_i;
  5. Q R = Y_its (QR factorization);
  6. U' Sigma V* = Q* A (SVD of the small l x n matrix);
  7. U = Q U'; the first k columns of U and V and the first k singular
     values are returned.

"b rows at a time" is the block-wise matrix product of the implementation
notes: A B is filled in block after block of rows of A, and A* C is the sum
over blocks of A_blk* C_blk; neither changes the result beyond rounding.
Optional column centring (Sec. 6: PCA works on the column-centred matrix;
the implementation offers the centring as preprocessing) subtracts the
column means from A before step 2.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def block_product(A: np.ndarray, B: np.ndarray, b: int) -> np.ndarray:
    """A B, b rows of A at a time."""
    m = A.shape[0]
    out = np.empty((m, B.shape[1]))
    for r0 in range(0, m, b):
        out[r0:r0 + b] = A[r0:r0 + b] @ B
    return out


def block_adjoint_product(A: np.ndarray, C: np.ndarray, b: int) -> np.ndarray:
    """A* C = sum over blocks of b rows of A_blk* C_blk."""
    acc = np.zeros((A.shape[1], C.shape[1]))
    for r0 in range(0, A.shape[0], b):
        acc += A[r0:r0 + b].T @ C[r0:r0 + b]
    return acc


def lu_renormalize(Y: np.ndarray):
    """L, U with Y = L U: partial pivoting, L = P L' (unit lower trapezoidal
    up to the row permutation P, every entry of magnitude <= 1)."""
    P, Lp, U = scipy.linalg.lu(Y)
    return P @ Lp, U


def oocpca(A, k: int, its: int, Omega, b: int | None = None, center: bool = False):
    """Top-k PCA of A (m x n) by Algorithm oocPCA with l = Omega.shape[1]
    random vectors; returns U (m x k), sigma (k), V (n x k)."""
    A = np.asarray(A, dtype=np.float64)
    Omega = np.asarray(Omega, dtype=np.float64)
    m, n = A.shape
    l = Omega.shape[1]
    if not (0 < k <= l < min(m, n)):
        raise ValueError("need 0 < k <= l < min(m, n)")
    if Omega.shape[0] != n:
        raise ValueError("Omega must have n rows")
    b = b or m
    if center:
        A = A - A.mean(axis=0)
    Y = block_product(A, Omega, b)                                   # step 2
    L, _ = lu_renormalize(Y)                                         # step 3
    for i in range(1, its + 1):                                      # step 4
        Y = block_product(A, block_adjoint_product(A, L, b), b)
        if i < its:
            L, _ = lu_renormalize(Y)
    Q, _ = np.linalg.qr(Y)                                           # step 5
    B = block_adjoint_product(A, Q, b).T                             # Q* A
    Up, s, Vh = np.linalg.svd(B, full_matrices=False)                # step 6
    U = Q @ Up                                                       # step 7
    return U[:, :k], s[:k], Vh[:k].T


def spectral_error(A, U, s, V, iters: int = 200, seed: int = 0) -> float:
    """||A - U diag(s) V*||_2 by power iteration on the residual (FP64)."""
    A = np.asarray(A, dtype=np.float64)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.shape[1])
    x /= np.linalg.norm(x)
    est = 0.0
    for _ in range(iters):
        y = A @ x - U @ (s * (V.T @ x))
        z = A.T @ y - V @ (s * (U.T @ y))
        nz = np.linalg.norm(z)
        if nz == 0.0:
            return 0.0
        est = np.sqrt(nz)
        x = z / nz
    return float(est)
