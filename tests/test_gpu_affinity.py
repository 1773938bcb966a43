"""Input affinities built on the GPU (exact kNN, perplexity calibration,
symmetrisation; Sec. 1.1 Eq. p_ij with the k nearest neighbours of Sec. 3)
against the oracle's FP64 builder on the same seeded data.

What is unique is compared exactly; what rounding may legitimately change is
bounded:
  - the sorted k smallest distances of every row are unique: the GPU's
    (FP32, difference form) agree with the oracle's (FP64) to 1e-5 relative;
  - the neighbour lists agree exactly except where two candidates' FP64
    distances are within that tolerance of each other (a near-tie that FP32
    may order either way: each differing row must hold such a pair among the
    oracle's k + 1 nearest); on integer-valued data every distance is exact
    in both precisions and the lists, ties included, agree bit for bit;
  - the CSR structure (row_ptr, col) is equal wherever no near-tie touches
    the row or column;
  - values: both sides stop the bisection at |H - log perplexity| < 1e-5, so
    beta may differ by one bisection step; with dH/dbeta = -beta Var(d^2) that
    moves log p_{j|i} by at most 2e-5 |z_j| / (beta sd(d^2)) for a neighbour z_j
    standard deviations from the mean, below 1e-3 for the data here (checked
    by the entropy of every GPU row, which must itself be within 1e-5);
  - P is symmetric bit for bit and sums to 1.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from oracle import affinities as oaff
import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL_D2 = 1e-5
RTOL_P = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(params=["tc", "tiled", "rows"])
def knn_kernel(request, monkeypatch):
    """Every kNN kernel on every case (the library picks by N otherwise:
    the small cases here would all take the row kernel)."""
    monkeypatch.setenv("FITSNE_KNN_KERNEL", request.param)
    return request.param


def gpu_affinities(X, perplexity, k):
    N, D = X.shape
    with pkg.Affinity(N, D, k) as aff:
        P = aff.compute(torch.as_tensor(X, device="cuda"), perplexity)
        torch.cuda.synchronize()
        rp, col, val = (t.cpu().numpy().copy() for t in (P.row_ptr, P.col, P.val))
        idx, d2, pc = aff.knn()
        assert aff.launch_count() >= 10
    return rp, col, val, idx, d2, pc


def near_tie_rows(X, idx_g, idx_o, d2_o):
    """Rows whose lists differ; each must be explained by a near-tie."""
    bad = np.nonzero((idx_g != idx_o).any(axis=1))[0]
    X64 = X.astype(np.float64)
    for i in bad:
        dg = ((X64[idx_g[i]] - X64[i]) ** 2).sum(axis=1)  # FP64 distances of the GPU's picks
        assert np.allclose(dg, d2_o[i], rtol=RTOL_D2, atol=0), i
        assert len(set(idx_g[i])) == len(idx_g[i]) and i not in set(idx_g[i])
    return set(bad.tolist())


def check(X, perplexity, k, expect_exact_lists=False):
    N = X.shape[0]
    rp, col, val, idx_g, d2_g, pc = gpu_affinities(X, perplexity, k)
    idx_o, d2_o = oaff.exact_knn(X, k)
    # sorted distances: unique
    assert np.allclose(d2_g, d2_o, rtol=RTOL_D2, atol=1e-30)
    order_bad = near_tie_rows(X, idx_g, idx_o, d2_o)
    if expect_exact_lists:
        assert not order_bad
    # FP32 can reorder two neighbours only where their FP64 distances lie
    # within its rounding: every differing row has such a pair among the
    # oracle's k + 1 nearest
    _, d2_more = oaff.exact_knn(X, min(k + 1, N - 1))
    close = (np.diff(d2_more, axis=1) <= RTOL_D2 * d2_more[:, 1:]).any(axis=1)
    assert all(close[i] for i in order_bad), sorted(i for i in order_bad if not close[i])
    # P depends on the neighbour sets only; rows whose sets differ (a near-tie at
    # the k-th place) are left out of the comparison below with their columns
    bad = {i for i in order_bad if set(idx_g[i].tolist()) != set(idx_o[i].tolist())}
    # calibration reached on every row where it can be (more exact ties at the
    # smallest distance than the perplexity allows make it unreachable: the
    # oracle's own bisection then ends after 200 steps, and so must the GPU's)
    def entropy(p):
        with np.errstate(divide="ignore", invalid="ignore"):
            return -np.where(p > 0, p * np.log(p), 0.0).sum(axis=1)
    pc_o, _ = oaff.calibrate(d2_o, perplexity)
    ok = np.abs(entropy(pc_o) - np.log(perplexity)) < 1e-5
    assert ok.mean() > 0.9
    assert np.all(np.abs(entropy(pc)[ok] - np.log(perplexity)) < 1.1e-5)
    same = np.ones(N, bool)
    same[list(order_bad)] = False
    assert np.allclose(pc[~ok & same], pc_o[~ok & same], rtol=RTOL_P, atol=1e-12)
    assert np.allclose(pc.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    # structure and values
    G = sp.csr_matrix((val.astype(np.float64), col, rp), shape=(N, N))
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= k)
    for i in range(0, N, max(1, N // 64)):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i not in set(c.tolist())
    assert (G != G.T).nnz == 0  # symmetric bit for bit
    assert abs(G.sum() - 1.0) < 1e-5
    rp_o, col_o, val_o = oaff.build_P(X, perplexity, k)
    O = sp.csr_matrix((val_o, col_o, rp_o), shape=(N, N))
    keep = np.ones(N, bool)
    keep[list(bad)] = False
    # a near-tie changes the rows of the two points and the columns pointing at them
    for i in bad:
        keep[idx_g[i]] = False
        keep[idx_o[i]] = False
    Gk = G[keep][:, keep].tocsr()
    Ok = O[keep][:, keep].tocsr()
    # the GPU keeps the kNN graph's structure, including entries whose value
    # underflowed to 0 (the oracle drops those): compare at the GPU's positions
    r = np.repeat(np.arange(Gk.shape[0]), np.diff(Gk.indptr))
    o_at = np.asarray(Ok[r, Gk.indices]).ravel()
    assert np.count_nonzero(o_at) == Ok.nnz  # every oracle entry is present
    assert np.allclose(Gk.data, o_at, rtol=RTOL_P, atol=1e-30)
    return bad


@pytest.mark.parametrize("N,D,perp,seed", [
    (3001, 50, 30.0, 1),    # several kNN tiles and query blocks, ragged tail
    (1537, 3, 10.0, 2),     # D not a multiple of 4, small k (30)
    (2000, 64, 50.0, 3),    # D at its maximum, k = 150
])
def test_matches_oracle(N, D, perp, seed, knn_kernel):
    X = inputs.mixture(N=N, n_clusters=7, dim=D, seed=seed)
    check(X, perp, int(3 * perp))


def test_integer_data_with_exact_ties_is_bit_exact_in_structure(knn_kernel):
    """Small-integer coordinates: every squared distance is an exact integer in
    FP32 and FP64, duplicates give zero distances; the neighbour order
    (distance, then index) must agree exactly."""
    rng = np.random.default_rng(5)
    X = rng.integers(0, 4, size=(1200, 6)).astype(np.float32)
    X[600:700] = X[0:100]  # exact duplicates
    check(X, 5.0, 15, expect_exact_lists=True)


def test_k_is_everyone_else_and_k_at_maximum(knn_kernel):
    # N = k + 1: every point's list is all other points; P is dense
    X = inputs.mixture(N=91, n_clusters=3, dim=20, seed=9)
    check(X, 30.0, 90)
    # k = 256 (the largest), N ragged against the 64-query blocks
    X = inputs.mixture(N=1000, n_clusters=4, dim=10, seed=10)
    check(X, 80.0, 256)
    # D = 64 with k = 256: the register-tiled kernel's buffers exceed shared
    # memory, the one-candidate-per-lane kernel runs whatever the override
    X = inputs.mixture(N=700, n_clusters=4, dim=64, seed=15)
    check(X, 80.0, 256)


def test_recompute_and_bitwise_determinism(knn_kernel):
    X = inputs.mixture(N=2500, n_clusters=5, dim=50, seed=11)
    Xd = torch.as_tensor(X, device="cuda")
    with pkg.Affinity(2500, 50, 90) as aff:
        a = [t.cpu().numpy().copy() for t in aff.compute(Xd, 30.0).__dict__.values()]
        b = [t.cpu().numpy().copy() for t in aff.compute(Xd, 30.0).__dict__.values()]
        c = [t.cpu().numpy().copy() for t in aff.compute(Xd, 20.0).__dict__.values()]
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])  # same kNN graph
    assert not np.array_equal(a[2], c[2])


def test_tiled_and_row_kernels_agree_bitwise(monkeypatch):
    """Both kNN kernels sum the same squared differences in the same order of
    d and sort by (distance, index): the lists, distances and P are equal bit
    for bit (N ragged against both kernels' tiles)."""
    X = inputs.mixture(N=3001, n_clusters=6, dim=50, seed=21)
    out = {}
    for kern in ("tiled", "rows"):
        monkeypatch.setenv("FITSNE_KNN_KERNEL", kern)
        out[kern] = gpu_affinities(X, 30.0, 90)
    for a, b in zip(out["tiled"], out["rows"]):
        assert np.array_equal(a, b)


def test_rejects_bad_perplexity_and_shape():
    X = torch.zeros((200, 5), device="cuda")
    with pkg.Affinity(200, 5, 30) as aff:
        for perp in (0.5, 31.0, float("nan")):
            with pytest.raises(pkg.TsneError):
                aff.compute(X, perp)
        with pytest.raises(ValueError):
            aff.compute(torch.zeros((199, 5), device="cuda"), 10.0)


def test_non_finite_input_keeps_a_valid_structure():
    """A NaN row ranks last for everyone (its distances count as +inf) and gets
    the nearest points by index; the CSR stays well formed."""
    X = inputs.mixture(N=500, n_clusters=3, dim=8, seed=12)
    X[17, 3] = np.nan
    rp, col, val, idx, d2, pc = gpu_affinities(X, 10.0, 30)
    assert np.all((idx >= 0) & (idx < 500))
    assert rp[-1] == col.size and np.all(np.diff(rp) >= 30)
    assert np.all((col >= 0) & (col < 500))
    assert 17 not in set(idx[np.arange(500) != 17].ravel().tolist())


def test_gpu_p_drives_the_gradient_like_the_oracle_p():
    """End to end: the gradient from the GPU-built P equals the one from the
    oracle-built P (both on the GPU path) to the P tolerance."""
    N = 3000
    X = inputs.mixture(N=N, n_clusters=6, dim=50, seed=13)
    Y = torch.as_tensor(inputs.initial_embedding(N, 2, seed=13) * 300.0, device="cuda")
    with pkg.Affinity(N, 50, 90) as aff, pkg.Plan(N, 2) as plan:
        Pg = aff.compute(torch.as_tensor(X, device="cuda"), 30.0)
        dg, _ = plan.gradient(Pg, Y, alpha=1.0)
        Po = pkg.DeviceCSR.from_host(*oaff.build_P(X, 30.0))
        do, _ = plan.gradient(Po, Y, alpha=1.0)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(dg - do) / torch.linalg.norm(do))
    assert err < RTOL_P


def test_sampled_rows_at_one_million_points():
    """N = 1M, D = 50, perplexity 30: 48 sampled rows' neighbour distances
    against brute force in FP64, the sums and symmetry of P on the sample."""
    N, D, k = 1_000_000, 50, 90
    X = inputs.mixture(N=N, n_clusters=10, dim=D, seed=14)
    with pkg.Affinity(N, D, k) as aff:
        P = aff.compute(torch.as_tensor(X, device="cuda"), 30.0)
        torch.cuda.synchronize()
        rp, col, val = (t.cpu().numpy().copy() for t in (P.row_ptr, P.col, P.val))
        idx, d2, pc = aff.knn()
    rng = np.random.default_rng(0)
    X64 = X.astype(np.float64)
    for i in rng.choice(N, 48, replace=False):
        dd = ((X64 - X64[i]) ** 2).sum(axis=1)
        dd[i] = np.inf
        want = np.sort(dd)[:k]
        got = ((X64[idx[i]] - X64[i]) ** 2).sum(axis=1)
        assert np.allclose(got, want, rtol=RTOL_D2, atol=0), i
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and set(idx[i].tolist()) <= set(c.tolist())
        for j, v in zip(c[:8], val[rp[i]:rp[i + 1]][:8]):  # symmetric entries
            cj = col[rp[j]:rp[j + 1]]
            pos = np.searchsorted(cj, i)
            assert cj[pos] == i and val[rp[j] + pos] == v
    assert abs(val.astype(np.float64).sum() - 1.0) < 1e-4
    assert np.all(np.abs(-np.where(pc > 0, pc * np.log(pc), 0).sum(1)[:1000] - np.log(30.0)) < 1.1e-5)


@pytest.mark.parametrize("case", ["mixture", "integer_ties", "k256"])
def test_fp32_prefilter_keeps_the_fp64_bisection_path(case, monkeypatch):
    """The bandwidth search evaluates each step with FP32 exponentials first
    and in FP64 only near the target; every decision is the FP64 one, so
    beta and p_{j|i} are bit for bit those of the all-FP64 search
    (FITSNE_CALIB_FP64=1): ordinary rows, exact ties with unreachable
    perplexity (beta doubled to overflow), and k at its maximum."""
    if case == "mixture":
        X, k, perp = inputs.mixture(N=5000, n_clusters=7, dim=50, seed=31), 90, 30.0
    elif case == "integer_ties":
        rng = np.random.default_rng(32)
        X = rng.integers(0, 3, size=(2000, 4)).astype(np.float32)
        X[1000:1200] = X[0:200]
        k, perp = 30, 10.0
    else:
        X, k, perp = inputs.mixture(N=3000, n_clusters=4, dim=10, seed=33), 256, 80.0
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("FITSNE_CALIB_FP64", flag)
        out[flag] = gpu_affinities(X, perp, k)
    for a, b in zip(out["1"], out["0"]):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
