"""Pin of the oracle's whole run (orc_run) against a plain t-SNE written here
in numpy from the paper's definitions: the exact gradient of Sec. 1.1,
4 sum_j (alpha p_ij - w_ij / Z) w_ij (y_i - y_j) with w_ij = 1 / (1 + |y_i -
y_j|^2) and Z = sum_{k != l} w_kl; the exaggeration schedule of Sec. 1.2 and
Sec. 4; the gains / momentum update the paper takes over from t-SNE; and the
KL divergence of Sec. 1.1 at the final embedding.

On a tiny input with a fine interpolation grid the oracle's interpolated run
must follow this exact run. With the gains frozen (gain_inc = 0, gain_dec = 1)
the update is continuous in the gradient and the two runs agree to about
1e-4; with the adaptive gains a sign test on a near-zero coordinate can flip
between the two, so that case is compared loosely. The same comparisons
against a run whose schedule is read one iteration late, or whose final KL
takes Z from the embedding before the last step, must fail by far more than
the tolerances."""
import numpy as np
import pytest


def tiny_problem(N=40, seed=3):
    """Three Gaussian clusters in 5-d; P from a 6-nearest-neighbour Gaussian
    kernel, row-normalised, symmetrised, summing to 1 (stored in FP32 as the
    oracle takes it). Y0 ~ N(0, 1e-4)."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(scale=4.0, size=(3, 5))
    X = centres[rng.integers(0, 3, size=N)] + rng.normal(size=(N, 5))
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    A = np.zeros((N, N))
    for i in range(N):
        nb = [j for j in np.argsort(d2[i]) if j != i][:6]
        A[i, nb] = np.exp(-d2[i, nb] / np.median(d2[i, nb]))
    A = A / A.sum(1, keepdims=True)
    P = (A + A.T) / (2 * N)
    rp = np.zeros(N + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(N):
        nz = np.nonzero(P[i])[0]
        cols.extend(nz)
        vals.extend(P[i, nz])
        rp[i + 1] = len(cols)
    col = np.asarray(cols, dtype=np.int32)
    val = np.asarray(vals, dtype=np.float32)
    Pd = np.zeros((N, N))
    for i in range(N):
        Pd[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]].astype(np.float64)
    Y0 = rng.normal(scale=1e-2, size=(N, 2))
    return (rp, col, val), Pd, Y0


def kernel(Y):
    diff = Y[:, None, :] - Y[None, :, :]
    w = 1.0 / (1.0 + (diff ** 2).sum(-1))
    np.fill_diagonal(w, 0.0)
    return diff, w, w.sum()


def exact_grad(Y, Pd, alpha):
    diff, w, Z = kernel(Y)
    return 4.0 * (((alpha * Pd - w / Z) * w)[:, :, None] * diff).sum(1)


def exact_kl(Y, Pd, Z=None):
    _, w, Zy = kernel(Y)
    q = w / (Zy if Z is None else Z)
    m = Pd > 0
    return float((Pd[m] * np.log(Pd[m] / q[m])).sum())


def plain_tsne(Y0, Pd, sc, lag=0, n_iter=None):
    """The run as the paper states it; lag > 0 reads the schedule late."""
    Y = Y0.copy()
    uY = np.zeros_like(Y)
    g = np.ones_like(Y)
    for it in range(sc.n_iter if n_iter is None else n_iter):
        t = max(it - lag, 0)
        if t < sc.early_iters:
            a = sc.early_alpha
        elif sc.late_iters > 0 and t >= sc.n_iter - sc.late_iters:
            a = sc.late_alpha
        else:
            a = 1.0
        mu = sc.momentum_early if t < sc.mom_switch_iter else sc.momentum_late
        dY = exact_grad(Y, Pd, a)
        g = np.where(np.sign(dY) != np.sign(uY), g + sc.gain_inc, g * sc.gain_dec)
        g = np.maximum(g, sc.min_gain)
        uY = mu * uY - sc.lr * g * dY
        Y = Y + uY
    return Y


def schedule(orc, **kw):
    # every phase of the schedule within 60 iterations: early exaggeration 4
    # for 20, momentum switch at 30, late exaggeration 2 over the last 10
    return orc.Schedule(n_iter=60, early_iters=20, late_iters=10, mom_switch_iter=30,
                        early_alpha=4.0, late_alpha=2.0, **kw)


# 60 intervals of p = 3 nodes per dimension: the interpolated gradient is
# within about 1e-4 of the exact one at the widths these runs reach
OPTS = dict(n_int_fixed=60)


@pytest.fixture(scope="module")
def frozen(orc):
    P, Pd, Y0 = tiny_problem()
    sc = schedule(orc, lr=5.0, gain_inc=0.0, gain_dec=1.0)
    Y_orc, kl_orc = orc.run(Y0, P, sc, orc.InterpOptions(**OPTS))
    return Pd, Y0, sc, Y_orc, kl_orc


def test_run_follows_the_exact_tsne(frozen):
    Pd, Y0, sc, Y_orc, kl_orc = frozen
    Y = plain_tsne(Y0, Pd, sc)
    assert np.linalg.norm(Y_orc - Y) / np.linalg.norm(Y) < 5e-4
    kl = exact_kl(Y, Pd)
    assert abs(kl_orc - kl) <= 1e-4 * kl
    assert kl < 0.5 * exact_kl(Y0, Pd)  # the run did optimise


def test_a_schedule_read_late_is_seen(frozen):
    Pd, Y0, sc, Y_orc, _ = frozen
    Y_late = plain_tsne(Y0, Pd, sc, lag=1)
    assert np.linalg.norm(Y_orc - Y_late) / np.linalg.norm(Y_late) > 1e-2


def test_final_kl_takes_z_of_the_final_embedding(frozen):
    Pd, Y0, sc, Y_orc, kl_orc = frozen
    Y = plain_tsne(Y0, Pd, sc)
    Y_prev = plain_tsne(Y0, Pd, sc, n_iter=sc.n_iter - 1)
    _, _, Z_prev = kernel(Y_prev)
    stale = exact_kl(Y, Pd, Z=Z_prev)
    assert abs(stale - kl_orc) > 1e-2 * kl_orc


def test_run_with_adaptive_gains_tracks_the_exact_tsne(orc):
    P, Pd, Y0 = tiny_problem()
    sc = schedule(orc, lr=2.0)
    Y_orc, kl_orc = orc.run(Y0, P, sc, orc.InterpOptions(**OPTS))
    Y = plain_tsne(Y0, Pd, sc)
    assert np.linalg.norm(Y_orc - Y) / np.linalg.norm(Y) < 1e-2
    kl = exact_kl(Y, Pd)
    assert abs(kl_orc - kl) <= 2e-3 * kl
