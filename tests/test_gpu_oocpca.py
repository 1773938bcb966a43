"""Parity of the GPU oocPCA (Sec. 6, Algorithm oocPCA) with the FP64 oracle.

Tolerances, from the arithmetic: A and Omega are FP32 on both sides (the
oracle reads the same FP32 values in FP64). The GPU forms every product with
A on the tensor cores from TF32 heads and tails (three MMAs per step, FP32
accumulation), i.e. each product term within about 2^-21 of its value and
the sums rounded in FP32: the first pass's Y = A Omega and G = A* Y agree
with FP64 to about 1e-6 of their largest entries (bar 1e-5). Everything
after the passes is FP64, so the singular values agree to a few 1e-6 of
sigma_1 (bar 1e-5 sigma_1) and the rank-k approximation U diag(sigma) V* to
the same relative Frobenius bar; individual vectors are compared through
that product (their signs and rotations inside near-equal singular values
are not unique).

Shapes are ragged on purpose: m not a multiple of the 128-row tile or the
32-row stage, n not a multiple of the 128-column tile.
"""
import numpy as np
import pytest
import torch

import oracle.oocpca as ooc
import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def decaying(m, n, seed, decay=0.8, noise=1e-3):
    """Full-rank FP32 matrix with a geometric spectrum plus noise."""
    rng = np.random.default_rng(seed)
    r = min(m, n, 80)
    U0, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, r)))
    A = (U0 * (50.0 * decay ** np.arange(r))) @ V0.T + noise * rng.standard_normal((m, n))
    return A.astype(np.float32)


def compare(A32, Om, k, its, got, center=False, tol=1e-5):
    U, s, V = (t.cpu().numpy().astype(np.float64) for t in got)
    Uo, so, Vo = ooc.oocpca(A32.astype(np.float64), k, its, Om.astype(np.float64), center=center)
    assert np.all(np.diff(s) <= 0)
    assert np.abs(s - so).max() <= tol * so[0], (s, so)
    Rg = (U * s) @ V.T
    Ro = (Uo * so) @ Vo.T
    assert np.linalg.norm(Rg - Ro) <= tol * np.linalg.norm(Ro)
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-5
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-5
    return s, so


def test_first_pass_products_elementwise():
    m, n, k, l = 1000, 520, 6, 8
    A = np.random.default_rng(1).standard_normal((m, n)).astype(np.float32)
    Om = inputs.omega(n, l, seed=1).astype(np.float32)
    with pkg.OocPca(m, n, k, l, its=-1) as p:
        p.run(torch.as_tensor(A, device="cuda"), Om)
        Y0 = p.debug(0)
        G0 = p.debug(1)
    Yr = A.astype(np.float64) @ Om.astype(np.float64)
    assert np.abs(Y0 - Yr).max() <= 1e-5 * np.abs(Yr).max()
    Gr = A.astype(np.float64).T @ Y0
    assert np.abs(G0 - Gr).max() <= 1e-5 * np.abs(Gr).max()


@pytest.mark.parametrize("its", [0, 1, 2])
def test_planted_rank_matches_oracle(its):
    m, n, r = 3001, 1000, 10
    A, sig, _, _ = inputs.low_rank_matrix(m, n, r, seed=7, dtype=np.float32)
    Om = inputs.omega(n, r + 2, seed=7).astype(np.float32)
    with pkg.OocPca(m, n, r, its=its if its else -1) as p:
        got = p.run(torch.as_tensor(A, device="cuda"), Om)
        torch.cuda.synchronize()
    s, so = compare(A, Om, r, its, got)
    assert np.abs(s - sig).max() <= 1e-5 * sig[0]


@pytest.mark.parametrize("center", [False, True])
@pytest.mark.parametrize("where,block_rows", [("device", 0), ("device", 333), ("host", 500)])
def test_decaying_spectrum_matches_oracle(where, block_rows, center):
    m, n, k = 2077, 644, 12
    A = decaying(m, n, seed=3)
    if center:
        A = A + np.linspace(-2.0, 5.0, n, dtype=np.float32)  # column means to remove
    Om = inputs.omega(n, k + 2, seed=3).astype(np.float32)
    with pkg.OocPca(m, n, k, center=center, block_rows=block_rows) as p:
        src = torch.as_tensor(A, device="cuda") if where == "device" else A
        got = p.run(src, Om)
        torch.cuda.synchronize()
        passes = p.phase_ms()["passes"]
    compare(A, Om, k, 2, got, center=center)
    # its = 2: Y_0, Y_1, Y_2, then Q* A; one more for the column means
    assert passes == 4 + (1 if center else 0)


def test_repeated_runs_are_identical():
    m, n, k = 1500, 400, 8
    A = torch.as_tensor(decaying(m, n, seed=5), device="cuda")
    Om = inputs.omega(n, k + 2, seed=5).astype(np.float32)
    with pkg.OocPca(m, n, k) as p:
        a = [t.clone() for t in p.run(A, Om)]
        b = p.run(A, Om)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_bad_arguments_are_rejected():
    with pytest.raises(pkg.TsneError):
        pkg.OocPca(100, 102, 4)  # n not a multiple of 4
    with pkg.OocPca(200, 100, 4) as p:
        A = torch.zeros((200, 100), device="cuda")
        with pytest.raises(ValueError):
            p.run(A, np.zeros((100, 5), np.float32))  # Omega must be n x l
        with pytest.raises(TypeError):
            p.run(torch.zeros((200, 100), device="cuda", dtype=torch.float64), np.zeros((100, 6), np.float32))
