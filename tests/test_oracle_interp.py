"""Pins of the oracle's interpolated gradient (Sec. 2.1-2.5, Appendix).

What fixes each part, independently of the oracle's own code:
  * Step 1 (spread), node placement and Lagrange basis: moments of degree < p
    are conserved (Lagrange interpolation reproduces polynomials of degree
    < p), with the nodes placed by Eq. (equinodes) in the test.
  * Steps 2-3, the circulant embedding and the h -> F_rep assembly: points put
    exactly on nodes make every Lagrange weight 0 or 1, so the interpolated
    gradient must equal the exact O(N^2) one (self term included in h_1).
  * The FFT mode: equals the literal Toeplitz sum.
  * The approximation: its error obeys the bound of Sec. 2.1 with eps measured
    from the kernel interpolant, and falls as N_int or p grow (Sec. 2.3).
"""
import numpy as np
import pytest
from scipy.interpolate import BarycentricInterpolator


def knn_P(rng, N, k=5):
    """A small symmetric normalised P on random neighbours (values only need to be valid)."""
    A = np.zeros((N, N))
    for i in range(N):
        nb = rng.choice(np.delete(np.arange(N), i), size=k, replace=False)
        A[i, nb] = rng.random(k)
    A = A + A.T
    A /= A.sum()
    rows, cols = np.nonzero(A)
    rp = np.searchsorted(rows, np.arange(N + 1)).astype(np.int32)
    return rp, cols.astype(np.int32), A[rows, cols].astype(np.float32)


def nodes(box):
    n = box.n_int * box.p
    return np.float64(box.y_min) + (np.arange(n) + 0.5) * box.delta


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_spread_conserves_moments_1d(orc, p):
    rng = np.random.default_rng(p)
    Y = rng.normal(0, 4, size=(300, 1)).astype(np.float32).astype(np.float64)
    o = orc.InterpOptions(p=p, n_int_fixed=7, use_fft=False)
    out = orc.interp_gradient(Y, knn_P(rng, 300), opts=o, want_grids=True)
    x = nodes(out["box"])
    w = out["w"]
    for a in range(p):
        ref0 = np.sum(Y[:, 0] ** a)
        ref1 = np.sum(Y[:, 0] * Y[:, 0] ** a)
        assert abs(np.sum(w[0] * x ** a) - ref0) <= 1e-10 * max(1.0, np.sum(np.abs(Y[:, 0]) ** a))
        assert abs(np.sum(w[1] * x ** a) - ref1) <= 1e-10 * max(1.0, np.sum(np.abs(Y[:, 0]) ** (a + 1)))
    # degree p is not reproduced in general
    assert abs(np.sum(w[0] * x ** p) - np.sum(Y[:, 0] ** p)) > 1e-8


@pytest.mark.parametrize("p", [2, 3, 4])
def test_spread_conserves_moments_2d(orc, p):
    rng = np.random.default_rng(20 + p)
    Y = rng.normal(0, 3, size=(200, 2)).astype(np.float32).astype(np.float64)
    o = orc.InterpOptions(p=p, n_int_fixed=5, use_fft=False)
    out = orc.interp_gradient(Y, knn_P(rng, 200), opts=o, want_grids=True)
    x = nodes(out["box"])
    w = out["w"]
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    for a in range(p):
        for b in range(p):
            mono = X1 ** a * X2 ** b
            pts = Y[:, 0] ** a * Y[:, 1] ** b
            scale = max(1.0, np.sum(np.abs(pts) * (1 + np.abs(Y).sum(1))))
            assert abs(np.sum(w[0] * mono) - pts.sum()) <= 1e-10 * scale
            assert abs(np.sum(w[1] * mono) - (Y[:, 0] * pts).sum()) <= 1e-10 * scale
            assert abs(np.sum(w[2] * mono) - (Y[:, 1] * pts).sum()) <= 1e-10 * scale


@pytest.mark.parametrize("s", [1, 2])
@pytest.mark.parametrize("use_fft", [False, True])
def test_points_on_nodes_are_exact(orc, s, use_fft):
    """With every point on a node, Lagrange weights are 0/1 and the scheme is exact."""
    rng = np.random.default_rng(7 + s)
    n_int, p = 8, 3
    # box [0, 6]: b = 0.75 and delta = 0.25 are exact binary fractions
    o = orc.InterpOptions(p=p, n_int_fixed=n_int, force_box=(0.0, 6.0), use_fft=use_fft)
    n = n_int * p
    N = 120 if s == 2 else 60
    g = rng.integers(0, n, size=(N, s))
    Y = (g + 0.5) * 0.25
    P = knn_P(rng, N)
    ex = orc.exact_gradient(Y, P, alpha=2.0)
    it = orc.interp_gradient(Y, P, alpha=2.0, opts=o)
    assert it["box"].delta == 0.25
    assert abs(it["Z"] - ex["Z"]) <= 1e-12 * ex["Z"]
    np.testing.assert_allclose(it["dY"], ex["dY"], rtol=0, atol=1e-11 * np.abs(ex["dY"]).max())
    np.testing.assert_allclose(it["rep"], ex["rep"], rtol=0, atol=1e-11 * np.abs(ex["rep"]).max())


@pytest.mark.parametrize("s", [1, 2])
def test_fft_equals_direct(orc, s):
    rng = np.random.default_rng(40 + s)
    N = 400
    Y = rng.normal(0, 5, size=(N, s)).astype(np.float32).astype(np.float64)
    P = knn_P(rng, N)
    d = orc.interp_gradient(Y, P, opts=orc.InterpOptions(n_int_fixed=9, use_fft=False))
    f = orc.interp_gradient(Y, P, opts=orc.InterpOptions(n_int_fixed=9, use_fft=True))
    np.testing.assert_allclose(f["h"], d["h"], rtol=1e-11, atol=1e-12 * np.abs(d["h"]).max())
    assert abs(f["Z"] - d["Z"]) <= 1e-12 * d["Z"]
    np.testing.assert_allclose(f["dY"], d["dY"], rtol=0, atol=1e-10 * np.abs(d["dY"]).max())


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("s", [1, 2])
def test_error_falls_with_intervals_and_nodes(orc, s):
    """Sec. 2.3: accuracy improves as N_int grows at fixed p, and as p grows once
    the intervals are narrow against the kernel's width (with wide intervals the
    equispaced nodes suffer the Runge effect that Sec. 2.3 warns about)."""
    rng = np.random.default_rng(50 + s)
    N = 250
    Y = rng.normal(0, 6, size=(N, s)).astype(np.float32).astype(np.float64)
    P = knn_P(rng, N)
    ex = orc.exact_gradient(Y, P)
    errs = [rel_l2(orc.interp_gradient(Y, P, opts=orc.InterpOptions(p=3, n_int_fixed=m))["dY"], ex["dY"])
            for m in (5, 10, 20, 40, 80)]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 5e-3
    errs_p = [rel_l2(orc.interp_gradient(Y, P, opts=orc.InterpOptions(p=p, n_int_fixed=40))["dY"], ex["dY"])
              for p in (2, 3, 4, 5, 6)]
    assert all(a > b for a, b in zip(errs_p, errs_p[1:])), errs_p


def test_error_bound_1d(orc):
    """|phi~ - phi| <= eps sum|q| (Sec. 2.1) with eps = sup |K_p - K| over the box."""
    rng = np.random.default_rng(61)
    N, n_int, p = 300, 6, 3
    Y = rng.uniform(-4, 4, size=(N, 1)).astype(np.float32).astype(np.float64)
    P = knn_P(rng, N)
    out = orc.interp_gradient(Y, P, opts=orc.InterpOptions(p=p, n_int_fixed=n_int))
    bx = out["box"]
    b = float(bx.b)
    # sample each interval and build K_p(y, z) = sum_jl K(y~_j, z~_l) L_j(y) L_l(z)
    per = 60
    t = (np.arange(per) + 0.5) / per
    samples, basis = [], []
    for ell in range(n_int):
        left = bx.y_min + ell * b
        nd = left + (np.arange(p) + 0.5) * bx.delta
        ys = left + t * b
        B = np.stack([BarycentricInterpolator(nd, np.eye(p)[j])(ys) for j in range(p)], axis=1)
        samples.append((ys, nd, B))
    worst = {1: 0.0, 2: 0.0}
    for ys, ndy, By in samples:
        for zs, ndz, Bz in samples:
            D = ndy[:, None] - ndz[None, :]
            for kk, K in ((1, lambda r2: 1 / (1 + r2)), (2, lambda r2: 1 / (1 + r2) ** 2)):
                Kp = By @ K(D ** 2) @ Bz.T
                Kt = K((ys[:, None] - zs[None, :]) ** 2)
                worst[kk] = max(worst[kk], np.abs(Kp - Kt).max())
    # exact potentials, self term included as in the grid sums
    R2 = (Y[:, 0][:, None] - Y[:, 0][None, :]) ** 2
    h1 = (1 / (1 + R2)).sum(1)
    h3 = (1 / (1 + R2) ** 2).sum(1)
    h2 = (Y[:, 0][None, :] / (1 + R2) ** 2).sum(1)
    slack = 1.05  # the sampled sup is slightly below the true sup
    assert np.abs(out["h"][:, 0] - h1).max() <= slack * worst[1] * N
    assert np.abs(out["h"][:, 2] - h3).max() <= slack * worst[2] * N
    assert np.abs(out["h"][:, 1] - h2).max() <= slack * worst[2] * np.abs(Y).sum()
    # and the bound is not vacuous: the error is a sizeable fraction of it
    assert np.abs(out["h"][:, 0] - h1).max() > 1e-3 * worst[1] * N


def test_brute_force_small_n(orc):
    """N <= 50: fine grids reproduce the exact gradient, Z and KL."""
    rng = np.random.default_rng(70)
    for s in (1, 2):
        N = 40
        Y = rng.normal(0, 2, size=(N, s)).astype(np.float32).astype(np.float64)
        P = knn_P(rng, N, k=6)
        ex = orc.exact_gradient(Y, P, alpha=4.0)
        it = orc.interp_gradient(Y, P, alpha=4.0, opts=orc.InterpOptions(n_int_fixed=200))
        assert rel_l2(it["dY"], ex["dY"]) < 2e-6
        assert abs(it["Z"] - ex["Z"]) < 5e-7 * ex["Z"]
        assert abs(orc.kl(Y, P, it["Z"]) - orc.kl(Y, P, ex["Z"])) < 5e-7


def test_box_rule(orc):
    """N_int = max(n_min, ceil(width)) capped (Sec. 2.5); FP32 box decisions."""
    o = orc.InterpOptions(n_min=50, n_int_max=1000)
    Y = np.array([[-1.5], [71.7]])
    bx = orc.box(Y, o)
    assert bx.n_int == 74 and np.float32(bx.width) == np.float32(71.7) - np.float32(-1.5)
    assert orc.box(np.array([[0.0], [10.0]]), o).n_int == 50
    assert orc.box(np.array([[0.0], [5000.0]]), o).n_int == 1000
    assert orc.box(np.array([[2.0, 2.0], [2.0, 2.0]]), o).width == 1.0  # degenerate box
    assert orc.box(np.array([[0.0], [10.0]]), orc.InterpOptions(n_int_fixed=13)).n_int == 13


def test_edge_points(orc):
    """Points on the upper edge belong to the last interval (t = p, extrapolation-free)."""
    rng = np.random.default_rng(80)
    Y = np.concatenate([rng.uniform(0, 1, size=(30, 2)), [[0.0, 0.0], [1.0, 1.0], [1.0, 0.0]]])
    Y = Y.astype(np.float32).astype(np.float64)
    P = knn_P(rng, len(Y))
    ex = orc.exact_gradient(Y, P)
    it = orc.interp_gradient(Y, P, opts=orc.InterpOptions(n_int_fixed=30))
    assert rel_l2(it["dY"], ex["dY"]) < 2e-5
    # the corner points (last rows) are no worse than the interior ones
    err = np.abs(it["rep"] - ex["rep"]).max(axis=1)
    assert err[-3:].max() <= 4 * err[:-3].max()
