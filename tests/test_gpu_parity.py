"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: dY relative L2 <= 1e-5, Z relative <= 1e-6 (FP32 spreading, FFT
and gather against the FP64 oracle on the same box); the spread grids and the
node potentials element by element relative to their largest magnitude.
Sizes span many tiles with ragged tails (N not a multiple of 32 or 256).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs

pytestmark = pytest.mark.gpu

DY_TOL = 1e-5
Z_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def clustered_Y(N, s, scale, seed, n_clusters=6):
    """Embedding-like coordinates: clusters of relative width 0.1 around N(0, scale^2)."""
    rng = np.random.default_rng(seed)
    c = rng.normal(0, scale, size=(n_clusters, s))
    lab = rng.integers(0, n_clusters, size=N)
    return (c[lab] + rng.normal(0, 0.1 * scale, size=(N, s))).astype(np.float32)


_P_CACHE = {}


def affinities(N, seed, perp=30.0):
    key = (N, seed, perp)
    if key not in _P_CACHE:
        X = inputs.mixture(N=N, n_clusters=6, seed=seed)
        _P_CACHE[key] = inputs.affinities(X, perp, device="cpu")
    return _P_CACHE[key]


def oracle_opts(plan_s, n_int_fixed=0):
    return oracle.InterpOptions(p=3, n_int_fixed=n_int_fixed, n_min=50,
                                n_int_max=400 if plan_s == 2 else 1000, use_fft=True)


CASES = [(2000, 20.0), (3001, 0.05), (1537, 90.0), (4099, 3.0)]


@pytest.mark.parametrize("s", [1, 2])
@pytest.mark.parametrize("N,scale", CASES)
def test_gradient_and_Z(s, N, scale):
    P = affinities(N, 1)
    Y = clustered_Y(N, s, scale, seed=N + s)
    with pkg.Plan(N, s) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        Yd = torch.as_tensor(Y, device="cuda")
        dY, Z = plan.gradient(Pd, Yd, alpha=12.0)
        rep, _ = plan.gradient(Pd, Yd, alpha=0.0)
        torch.cuda.synchronize()
        assert plan.status() == 0
        info = plan.info()
    ref = oracle.interp_gradient(Y.astype(np.float64), P.as_tuple(), alpha=12.0, opts=oracle_opts(s))
    bx = ref["box"]
    assert info["n_int"] == bx.n_int
    assert np.float32(info["y_min"]) == np.float32(bx.y_min)
    assert np.float32(info["b"]) == np.float32(bx.b)
    assert info["fft_len"] >= 2 * bx.n_int * 3
    assert rel_l2(dY.cpu().numpy(), ref["dY"]) <= DY_TOL
    assert abs(Z.item() - ref["Z"]) <= Z_TOL * ref["Z"]
    assert rel_l2(rep.cpu().numpy(), 4.0 * ref["rep"]) <= DY_TOL


@pytest.mark.parametrize("s", [1, 2])
def test_spread_grids(s):
    """Step 1: the charge grid w0 and the dipole grids d_m = (w_{y(m)} - y~(m) w0) / delta
    against the oracle's spread of the charges 1 and y(m)."""
    N = 2500
    P = affinities(N, 2)
    Y = clustered_Y(N, s, 15.0, seed=7)
    with pkg.Plan(N, s) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        plan.gradient(Pd, torch.as_tensor(Y, device="cuda"), alpha=1.0)
        info = plan.info()
        w = plan.debug(0)
    ref = oracle.interp_gradient(Y.astype(np.float64), P.as_tuple(), opts=oracle_opts(s),
                                 want_grids=True)
    bx = ref["box"]
    n = info["n"]
    G = n ** s
    w = w.reshape(s + 1, G)
    rw = ref["w"].reshape(s + 1, G)
    x = np.float64(bx.y_min) + (np.arange(n) + 0.5) * bx.delta  # node positions
    if s == 1:
        coords = [x]
    else:
        X1, X2 = np.meshgrid(x, x, indexing="ij")
        coords = [X1.ravel(), X2.ravel()]
    expect = [rw[0]] + [(rw[m] - coords[m - 1] * rw[0]) / bx.delta for m in range(1, s + 1)]
    for ch in range(s + 1):
        scale = np.abs(expect[ch]).max()
        assert np.abs(w[ch] - expect[ch]).max() <= 1e-6 * scale, ch


@pytest.mark.parametrize("s", [1, 2])
def test_fft_convolution_against_cufft(s):
    """Step 2: the hand-written FFT convolution equals cuFFT (torch.fft, FP64) applied
    to the same spread grids: (u'_1, u'_2, v) = (K2*d1 - G1*w0, K2*d2 - G2*w0, K2*w0), and
    Z + N = w0 . (K1 * w0)."""
    N = 3000
    P = affinities(N, 3)
    Y = clustered_Y(N, s, 40.0, seed=11)
    with pkg.Plan(N, s) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        plan.gradient(Pd, torch.as_tensor(Y, device="cuda"), alpha=1.0)
        info = plan.info()
        w = plan.debug(0)
        h = plan.debug(1)
    n, delta = info["n"], np.float64(info["delta"])
    L = 2 * n
    dev = torch.device("cuda")
    f64 = torch.float64
    off = torch.arange(L, device=dev, dtype=f64)
    off = torch.where(off < n, off, off - L)  # signed offsets; index n is never reached
    if s == 1:
        K1 = 1 / (1 + (off * delta) ** 2)
        K2 = K1 ** 2
        G1 = off * K2
        pad = torch.zeros((2, L), dtype=f64, device=dev)
        pad[:, :n] = torch.as_tensor(w.reshape(2, n), device=dev)
        F = torch.fft.fft(pad)
        conv = lambda a, K: torch.fft.ifft(F[a] * torch.fft.fft(K)).real[:n]
        zero = torch.zeros(n, dtype=f64, device=dev)
        want_h1 = conv(0, K1)
        want = torch.stack([want_h1, conv(1, K2) - conv(0, G1), zero, conv(0, K2)], dim=1)
    else:
        O1, O2 = off[:, None].expand(L, L), off[None, :].expand(L, L)
        K1 = 1 / (1 + (O1 * delta) ** 2 + (O2 * delta) ** 2)
        K2 = K1 ** 2
        pad = torch.zeros((3, L, L), dtype=f64, device=dev)
        pad[:, :n, :n] = torch.as_tensor(w.reshape(3, n, n), device=dev)
        F = torch.fft.fft2(pad)
        conv = lambda a, K: torch.fft.ifft2(F[a] * torch.fft.fft2(K)).real[:n, :n].reshape(-1)
        want_h1 = conv(0, K1)
        want = torch.stack([want_h1, conv(1, K2) - conv(0, O1 * K2),
                            conv(2, K2) - conv(0, O2 * K2), conv(0, K2)], dim=1)
    want = want.cpu().numpy()
    for k in ([1, 3] if s == 1 else [1, 2, 3]):
        scale = np.abs(want[:, k]).max()
        assert np.abs(h[:, k] - want[:, k]).max() <= 5e-6 * scale, k
    zn = float((torch.as_tensor(w.reshape(s + 1, -1)[0], device=dev) * want_h1).sum())
    assert abs(info["Z"] + N - zn) <= 5e-7 * zn


@pytest.mark.parametrize("s", [1, 2])
def test_points_on_nodes_match_exact(s):
    """Forced box [0, 6], 8 intervals, delta = 1/4: nodes are exact floats, so
    the interpolated gradient equals the exact O(N^2) one up to FP32 rounding."""
    rng = np.random.default_rng(5)
    N = 700
    g = rng.integers(0, 24, size=(N, s))
    Y = ((g + 0.5) * 0.25).astype(np.float32)
    P = affinities(N, 4, perp=10.0)
    with pkg.Plan(N, s) as plan:
        plan.set_box(0.0, 6.0, 8)
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        dY, Z = plan.gradient(Pd, torch.as_tensor(Y, device="cuda"), alpha=2.0)
        torch.cuda.synchronize()
    ex = oracle.exact_gradient(Y.astype(np.float64), P.as_tuple(), alpha=2.0)
    assert rel_l2(dY.cpu().numpy(), ex["dY"]) <= DY_TOL
    assert abs(Z.item() - ex["Z"]) <= Z_TOL * ex["Z"]


@pytest.mark.parametrize("s", [1, 2])
def test_step_matches_oracle_step(s):
    N = 2100
    P = affinities(N, 5)
    rng = np.random.default_rng(9)
    Y = clustered_Y(N, s, 10.0, seed=13)
    uY = (rng.normal(0, 0.05, size=(N, s))).astype(np.float32)
    gains = rng.uniform(0.5, 2.0, size=(N, s)).astype(np.float32)
    sched = pkg.Schedule()
    with pkg.Plan(N, s) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        Yd, ud, gd = (torch.as_tensor(a.copy(), device="cuda") for a in (Y, uY, gains))
        plan.step(Pd, Yd, ud, gd, 300, sched)
        torch.cuda.synchronize()
    ref = oracle.interp_gradient(Y.astype(np.float64), P.as_tuple(), alpha=1.0, opts=oracle_opts(s))
    Yo, uo, go = Y.astype(np.float64), uY.astype(np.float64), gains.astype(np.float64)
    oracle.step(Yo, uo, go, ref["dY"], oracle.Schedule(), 300)
    # an update moves Y by lr * gain * dY; the dY tolerance bounds the difference
    step_scale = np.linalg.norm(200.0 * go * ref["dY"])
    assert np.linalg.norm(Yd.cpu().numpy() - Yo) <= 2 * DY_TOL * step_scale + 1e-6 * np.linalg.norm(Yo)
    # gains follow the sign rule exactly wherever the signs agree
    same = np.sign(ref["dY"]) != 0
    assert (np.abs(gd.cpu().numpy() - go)[same] < 1e-6).mean() > 0.999


@pytest.mark.parametrize("s", [1, 2])
def test_kl(s):
    N = 2400
    P = affinities(N, 6)
    Y = clustered_Y(N, s, 12.0, seed=17)
    with pkg.Plan(N, s) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        kl = plan.kl(Pd, torch.as_tensor(Y, device="cuda"))
    ref = oracle.interp_gradient(Y.astype(np.float64), P.as_tuple(), opts=oracle_opts(s))
    want = oracle.kl(Y.astype(np.float64), P.as_tuple(), ref["Z"])
    assert abs(kl - want) <= 1e-6 * abs(want)


def test_two_points_and_degenerate_box():
    # N = 2 (the smallest plan), and all points on one location (width 0 -> 1)
    P = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([0.5, 0.5], np.float32))
    for Y in (np.array([[0.3, -0.2], [1.3, 0.8]], np.float32), np.full((2, 2), 4.0, np.float32)):
        with pkg.Plan(2, 2) as plan:
            dY, Z = plan.gradient(pkg.DeviceCSR.from_host(*P), torch.as_tensor(Y, device="cuda"), 3.0)
            torch.cuda.synchronize()
        ref = oracle.interp_gradient(Y.astype(np.float64), P, alpha=3.0, opts=oracle_opts(2))
        # coincident points: the exact forces vanish; FP32 leaves O(1e-6) residue
        np.testing.assert_allclose(dY.cpu().numpy(), ref["dY"], rtol=1e-5, atol=1e-5)
        # with N = 2, Z (about 0.67) is the small difference sum h1 - N of two
        # O(1) terms, so its error is bounded relative to sum h1 = Z + N
        assert abs(Z.item() - ref["Z"]) <= Z_TOL * (abs(ref["Z"]) + 2)


def test_empty_rows_and_ragged():
    rng = np.random.default_rng(21)
    N = 1031
    Y = clustered_Y(N, 2, 25.0, seed=3)
    # rows with no neighbours, and a few heavy rows
    rows, cols = [], []
    for i in range(N):
        k = 0 if i % 7 == 0 else (200 if i % 101 == 0 else 5)
        nb = rng.choice(np.delete(np.arange(N), i), size=k, replace=False)
        rows += [i] * k
        cols += list(nb)
    import scipy.sparse as sp
    A = sp.csr_matrix((rng.random(len(rows)), (rows, cols)), shape=(N, N))
    A = A + A.T
    A = (A / A.sum()).tocsr()
    A.sort_indices()
    P = (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float32))
    with pkg.Plan(N, 2) as plan:
        dY, Z = plan.gradient(pkg.DeviceCSR.from_host(*P), torch.as_tensor(Y, device="cuda"), 5.0)
        torch.cuda.synchronize()
    ref = oracle.interp_gradient(Y.astype(np.float64), P, alpha=5.0, opts=oracle_opts(2))
    assert rel_l2(dY.cpu().numpy(), ref["dY"]) <= DY_TOL


def test_interval_cap_and_fixed_count():
    N = 1200
    P = affinities(N, 7)
    Y = clustered_Y(N, 2, 400.0, seed=23)  # width far above the 2-D cap of 400
    for fixed in (0, 37):
        with pkg.Plan(N, 2, n_intervals=fixed) as plan:
            dY, Z = plan.gradient(pkg.DeviceCSR.from_host(*P.as_tuple()), torch.as_tensor(Y, device="cuda"), 1.0)
            info = plan.info()
        ref = oracle.interp_gradient(Y.astype(np.float64), P.as_tuple(), opts=oracle_opts(2, fixed))
        assert info["n_int"] == ref["box"].n_int == (400 if fixed == 0 else 37)
        assert rel_l2(dY.cpu().numpy(), ref["dY"]) <= DY_TOL


@pytest.mark.parametrize("scale,fixed,n_int_want", [(140.0, 0, None), (900.0, 0, 1000), (15.0, 1000, 1000)])
def test_1d_large_grid(scale, fixed, n_int_want):
    """Workload 3's 1-D grid (Algorithm 1, Sec. 2.5): the interval rule at a
    width of several hundred, the rule capped at 1000 intervals, and a fixed
    count of 1000 on a narrow embedding: 3000 nodes and an FFT length of at
    least 6000 convolved in one CTA. dY, its repulsive part and Z against the
    oracle at the same tolerances as the small grids; N_int, y_min and b bit
    for bit."""
    N = 5003
    P = affinities(N, 17)
    Y = clustered_Y(N, 1, scale, seed=int(scale) + fixed, n_clusters=9)
    with pkg.Plan(N, 1, n_intervals=fixed) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        Yd = torch.as_tensor(Y, device="cuda")
        dY, Z = plan.gradient(Pd, Yd, alpha=4.0)
        rep, _ = plan.gradient(Pd, Yd, alpha=0.0)
        torch.cuda.synchronize()
        assert plan.status() == 0
        info = plan.info()
    ref = oracle.interp_gradient(Y.astype(np.float64), P.as_tuple(), alpha=4.0, opts=oracle_opts(1, fixed))
    bx = ref["box"]
    assert info["n_int"] == bx.n_int
    if n_int_want is not None:
        assert bx.n_int == n_int_want
        assert info["fft_len"] >= 6000
    else:
        assert 300 < bx.n_int < 1000
    assert np.float32(info["y_min"]) == np.float32(bx.y_min)
    assert np.float32(info["b"]) == np.float32(bx.b)
    assert rel_l2(dY.cpu().numpy(), ref["dY"]) <= DY_TOL
    assert rel_l2(rep.cpu().numpy(), 4.0 * ref["rep"]) <= DY_TOL
    assert abs(Z.item() - ref["Z"]) <= Z_TOL * ref["Z"]


def test_errors_are_reported():
    with pytest.raises(pkg.TsneError) as e:
        pkg.Plan(100, 3)
    assert e.value.code == pkg._abi.TSNE_ERR_INVALID_ARG
    with pytest.raises(pkg.TsneError):
        pkg.Plan(100, 2, p=1)
    with pytest.raises(pkg.TsneError):
        pkg.Plan(1, 2)
    N = 300
    P = affinities(N, 8, perp=10.0)
    Y = clustered_Y(N, 2, 5.0, seed=1)
    Y[17, 1] = np.nan
    with pkg.Plan(N, 2) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        plan.gradient(Pd, torch.as_tensor(Y, device="cuda"), 1.0)
        assert plan.status() == pkg._abi.TSNE_ERR_NONFINITE
        assert plan.status() == 0  # the latch clears
        bad_col = P.col.copy()
        bad_col[5] = N + 3
        with pytest.raises(pkg.TsneError):
            plan.validate(pkg.DeviceCSR.from_host(P.row_ptr, bad_col, P.val))
        plan.validate(Pd)


@pytest.mark.parametrize("s", [1, 2])
def test_run_host_equals_run(s):
    N = 1500
    P = affinities(N, 9)
    Y0 = inputs.initial_embedding(N, s, seed=4)
    sched = pkg.Schedule(n_iter=20)
    with pkg.Plan(N, s) as plan:
        Yd = torch.as_tensor(Y0.copy(), device="cuda")
        kl_d = plan.run(pkg.DeviceCSR.from_host(*P.as_tuple()), Yd, sched)
        Yh = Y0.copy()
        kl_h = plan.run_host(P.row_ptr, P.col, P.val, Yh, sched)
    # every kernel is deterministic (integer spread sums, fixed-order reductions)
    assert kl_d == kl_h
    assert np.array_equal(Yh, Yd.cpu().numpy())


@pytest.mark.parametrize("s", [1, 2])
def test_bitwise_reproducible(s):
    """Two evaluations on the same input give identical bits (the counting sort
    orders points within a box arbitrarily; the spread sums do not depend on it)."""
    N = 5000
    P = affinities(N, 10)
    Y = clustered_Y(N, s, 0.3, seed=2)  # tight: many boxes hold several chunks
    with pkg.Plan(N, s) as plan:
        Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
        Yd = torch.as_tensor(Y, device="cuda")
        a, Za = plan.gradient(Pd, Yd, alpha=12.0)
        a = a.clone(); Za = Za.clone()
        b, Zb = plan.gradient(Pd, Yd, alpha=12.0)
        torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(Za, Zb)


@pytest.mark.parametrize("s", [1, 2])
def test_locality_relabelling(s):
    """A run that relabels its points (iterations 5, 15, 25) equals the run that
    does not, bit for bit: relabelling permutes the rows and maps the columns
    but keeps each row's entry order, the attraction's lane order depends only
    on that, and the spread, FFT and reductions do not depend on the order of
    the points. Y comes back in the caller's labels."""
    N = 6000
    P = affinities(N, 11)
    Y0 = clustered_Y(N, s, 3.0, seed=31)
    sched = pkg.Schedule(n_iter=30)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    out = {}
    for tag, first in (("plain", -1), ("relabel", 5), ("relabel2", 5)):
        with pkg.Plan(N, s, relabel_first=first, relabel_every=10, order_rounds=-1) as plan:
            Y = torch.as_tensor(Y0.copy(), device="cuda")
            kl = plan.run(Pd, Y, sched)
            assert plan.status() == 0
            out[tag] = (kl, Y.cpu().numpy())
    assert np.array_equal(out["relabel"][1], out["relabel2"][1])
    assert np.array_equal(out["relabel"][1], out["plain"][1])
    assert out["relabel"][0] == out["plain"][0]


@pytest.mark.parametrize("s", [1, 2])
def test_graph_order_is_bitwise_neutral(s):
    """Runs that start in the graph order of P (computed at the run's start,
    kept for the next run of the same P, or prepared by tsne_plan_order and
    reused without copying P again; with and without later embedding
    relabellings; 1 and 8 averaging rounds) equal the run in the caller's
    labels bit for bit, Y and KL. Rows of very different lengths and an
    empty row are included."""
    N = 6000
    P = affinities(N, 14)
    # an empty row: drop row 17's entries (P need not be symmetric here)
    a, b = int(P.row_ptr[17]), int(P.row_ptr[18])
    col = np.delete(P.col, np.s_[a:b])
    val = np.delete(P.val, np.s_[a:b])
    rp = P.row_ptr.copy()
    rp[18:] -= b - a
    Pd = pkg.DeviceCSR.from_host(rp, col, val)
    Y0 = clustered_Y(N, s, 3.0, seed=35)
    sched = pkg.Schedule(n_iter=30)

    def run(plan):
        Y = torch.as_tensor(Y0.copy(), device="cuda")
        kl = plan.run(Pd, Y, sched)
        assert plan.status() == 0
        return kl, Y.cpu().numpy()

    with pkg.Plan(N, s, relabel_first=-1, order_rounds=-1) as plan:
        want = run(plan)
    cases = []
    for rounds in (1, 8):
        for first in (-1, 5):
            with pkg.Plan(N, s, relabel_first=first, relabel_every=10, order_rounds=rounds) as plan:
                cases.append(run(plan))          # order computed at the start
                cases.append(run(plan))          # order kept, copy of P rebuilt
                plan.order(Pd)                   # prepared: copy of P reused
                cases.append(run(plan))
                cases.append(run(plan))
    for kl, Y in cases:
        assert np.array_equal(Y, want[1])
        assert kl == want[0]


def test_plan_order_during_a_run():
    """tsne_plan_order between two pieces of a relabelled run (its copy of P
    replaced by the graph-ordered one) leaves the run's result bitwise equal
    to the uninterrupted run."""
    N = 3000
    P = affinities(N, 16)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    Y0 = inputs.initial_embedding(N, 2, seed=3)
    sched = pkg.Schedule(n_iter=20)
    with pkg.Plan(N, 2, relabel_first=2, relabel_every=6) as plan:
        Ya = torch.as_tensor(Y0.copy(), device="cuda")
        plan.run_reset()
        plan.run_iters(Pd, Ya, sched, 0, 20)
        Yb = torch.as_tensor(Y0.copy(), device="cuda")
        plan.run_reset()
        plan.run_iters(Pd, Yb, sched, 0, 5)
        plan.order(Pd)
        plan.run_iters(Pd, Yb, sched, 5, 15)
        assert plan.status() == 0
    assert torch.equal(Ya, Yb)


def test_plan_order_rejections():
    N = 500
    P = affinities(N, 15)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    with pkg.Plan(N, 2, order_rounds=-1) as plan:
        with pytest.raises(pkg.TsneError):
            plan.order(Pd)  # the plan has no graph order
    with pkg.Plan(N, 2) as plan:
        with pytest.raises(ValueError):
            plan.order(pkg.DeviceCSR.from_host(*affinities(N + 1, 15).as_tuple()))


@pytest.mark.parametrize("s", [1, 2])
def test_checkpoint_resume_is_bitwise(s):
    """A run saved after iteration 26 (uY, gains in the caller's labels, after
    relabellings at 5, 15 and 25) and resumed in a new plan, and in the same
    plan, ends with the uninterrupted run's Y bit for bit; so does a run saved
    before any relabelling (iteration 3). The late-exaggeration window and the
    momentum switch fall after the resume point."""
    N = 6000
    P = affinities(N, 13)
    Y0 = clustered_Y(N, s, 3.0, seed=33)
    sched = pkg.Schedule(n_iter=60, early_iters=20, mom_switch_iter=30, late_iters=10, late_alpha=4.0)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    kw = dict(relabel_first=5, relabel_every=10)
    with pkg.Plan(N, s, **kw) as plan:
        Ya = torch.as_tensor(Y0.copy(), device="cuda")
        plan.run_reset()
        plan.run_iters(Pd, Ya, sched, 0, 60)
        ya = Ya.cpu().numpy()
    for cut in (27, 3):
        with pkg.Plan(N, s, **kw) as plan:
            Yb = torch.as_tensor(Y0.copy(), device="cuda")
            plan.run_reset()
            plan.run_iters(Pd, Yb, sched, 0, cut)
            uY, gains = plan.run_state_save()
            Ymid = Yb.clone()
            assert np.all(gains > 0) and np.any(uY != 0)
            plan.run_iters(Pd, Yb, sched, cut, 60 - cut)  # same plan, no save/load
            assert np.array_equal(Yb.cpu().numpy(), ya)
            plan.run_state_load(uY, gains)  # same plan, back to the checkpoint
            Yc = Ymid.clone()
            plan.run_iters(Pd, Yc, sched, cut, 60 - cut)
            assert np.array_equal(Yc.cpu().numpy(), ya)
        with pkg.Plan(N, s, **kw) as plan2:  # a fresh plan
            plan2.run_state_load(uY, gains)
            Yd = Ymid.clone()
            plan2.run_iters(Pd, Yd, sched, cut, 60 - cut)
            assert plan2.status() == 0
            assert np.array_equal(Yd.cpu().numpy(), ya)


@pytest.mark.parametrize("s", [1, 2])
def test_force_schedules_agree(s):
    """The force kernel's work schedules (grid-stride chunks, SM-local regions)
    change which warp computes a row, not the arithmetic or its order:
    relabelled runs under both schedules are bitwise equal (N = 20,000, rows
    of many lengths, relabelled at iterations 5 and 20)."""
    N = 20000
    X = inputs.mixture(N=N, n_clusters=40, seed=12)
    P = inputs.affinities(X, 30.0, device="cuda")
    Y0 = clustered_Y(N, s, 3.0, seed=41)
    sched = pkg.Schedule(n_iter=40)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    out = {}
    modes = (pkg._abi.TSNE_FORCE_GRID, pkg._abi.TSNE_FORCE_REGION)
    for mode in modes:
        with pkg.Plan(N, s, relabel_first=5, relabel_every=15, force_mode=mode) as plan:
            Y = torch.as_tensor(Y0.copy(), device="cuda")
            out[mode] = plan.run(Pd, Y, sched)
            assert plan.status() == 0
            out[(mode, "Y")] = Y.cpu().numpy()
            dY, Z = plan.gradient(Pd, Y, alpha=3.0)
            out[(mode, "dY")] = dY.cpu().numpy()
    assert np.array_equal(out[(modes[0], "Y")], out[(modes[1], "Y")])
    assert np.array_equal(out[(modes[0], "dY")], out[(modes[1], "dY")])
    assert out[modes[0]] == out[modes[1]]


@pytest.mark.parametrize("s", [1, 2])
def test_step_graph_equals_plain_launches(s):
    """Steady-state steps of a run replay one captured CUDA graph (on the
    plan's own stream, fenced to the caller's); with phase tracing on they
    are plain launches. Both give the same Y bit for bit, with relabellings
    inside the run and the run split over two calls."""
    N = 5000
    P = affinities(N, 18)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    Y0 = clustered_Y(N, s, 3.0, seed=37)
    sched = pkg.Schedule(n_iter=40)
    out = []
    for trace in (False, True):
        with pkg.Plan(N, s, relabel_first=7, relabel_every=12) as plan:
            plan.profile(trace)
            Y = torch.as_tensor(Y0.copy(), device="cuda")
            plan.run_reset()
            plan.run_iters(Pd, Y, sched, 0, 17)
            plan.run_iters(Pd, Y, sched, 17, 23)
            assert plan.status() == 0
            out.append(Y.cpu().numpy())
            if trace:
                assert plan.profile_read()["evals"] == 40
    assert np.array_equal(out[0], out[1])
