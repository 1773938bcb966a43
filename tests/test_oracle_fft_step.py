"""Pins of the oracle's FFT (against numpy.fft and the DFT definition) and of
its optimizer (special cases of the update rule; exaggeration schedule,
Sec. 1.2 and Sec. 4)."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024])
def test_fft_matches_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    np.testing.assert_allclose(orc.fft(x), np.fft.fft(x), rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(orc.fft(x, inverse=True) / n, np.fft.ifft(x), rtol=0, atol=1e-13 * max(1, n))


def test_fft_is_the_dft():
    import oracle
    n = 16
    x = np.random.default_rng(1).normal(size=n) + 0j
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    np.testing.assert_allclose(oracle.fft(x), F @ x, atol=1e-12)


def test_fft_rejects_non_power_of_two(orc):
    with pytest.raises(RuntimeError):
        orc.fft(np.ones(12))


def test_alpha_schedule(orc):
    sc = orc.Schedule(n_iter=1000, early_iters=250, late_iters=250, early_alpha=12, late_alpha=4)
    assert [orc.alpha_at(sc, i) for i in (0, 249, 250, 749, 750, 999)] == [12, 12, 1, 1, 4, 4]
    assert orc.alpha_at(orc.Schedule(late_iters=0), 999) == 1.0


def test_step_plain_descent_and_gains(orc):
    sc = orc.Schedule(lr=200.0)
    Y = np.array([[1.0, -2.0]])
    dY = np.array([[0.5, -0.25]])
    uY = np.zeros((1, 2))
    g = np.ones((1, 2))
    orc.step(Y, uY, g, dY, sc, 0)
    # sign(uY)=0 differs from sign(dY): gain 1 + 0.2; uY = -lr * 1.2 * dY
    np.testing.assert_allclose(g, [[1.2, 1.2]])
    np.testing.assert_allclose(uY, [[-120.0, 60.0]])
    np.testing.assert_allclose(Y, [[-119.0, 58.0]])
    # same sign as uY now (uY = -120 < 0 and dY < 0): gain * 0.8; momentum 0.5 before 250
    dY2 = np.array([[-1.0, 1.0]])
    orc.step(Y, uY, g, dY2, sc, 1)
    np.testing.assert_allclose(g, [[0.96, 0.96]])
    np.testing.assert_allclose(uY, [[0.5 * -120 + 200 * 0.96, 0.5 * 60 - 200 * 0.96]])
    # the floor on the gains, and momentum 0.8 from iteration 250
    g[:] = 0.011
    uY[:] = [[1.0, 1.0]]
    dY3 = np.array([[1.0, 1.0]])
    orc.step(Y, uY, g, dY3, sc, 300)
    np.testing.assert_allclose(g, [[0.01, 0.01]])
    np.testing.assert_allclose(uY, [[0.8 - 2.0, 0.8 - 2.0]])


def test_run_decreases_kl(orc):
    """A short run on clustered data lowers KL far below its value at Y0."""
    from paper_1712_09005_gb300 import inputs
    X = inputs.mixture(N=300, n_clusters=3, seed=5)
    P = inputs.affinities(X, 10.0, device="cpu").as_tuple()
    Y0 = inputs.initial_embedding(300, 2, seed=5).astype(np.float64)
    ex0 = orc.exact_gradient(Y0, P)
    kl0 = orc.kl(Y0, P, ex0["Z"])
    # lr scaled to the small N (lr = 200 suits N in the thousands and up)
    sc = orc.Schedule(n_iter=150, early_iters=50, mom_switch_iter=50, lr=25.0)
    Y, kl = orc.run(Y0, P, sc, orc.InterpOptions(n_min=20))
    assert kl < 0.6 * kl0
    assert np.isfinite(Y).all()
