"""Pins of the oracle's exact gradient, Z and KL (Sec. 1.1, Sec. 1.2).

None of these re-types the oracle's formula: the gradient is checked against
central finite differences of the KL cost, Z and the two-point case against
hand-derived closed forms (tests/golden/closed_forms.json), and both against
invariants the mathematics fixes (zero net force, translation invariance).
"""
import json
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def dense_P(N, rng):
    """A random symmetric P with zero diagonal summing to 1, as CSR."""
    A = rng.random((N, N))
    A = A + A.T
    np.fill_diagonal(A, 0.0)
    A /= A.sum()
    rows, cols = np.nonzero(A)
    rp = np.zeros(N + 1, dtype=np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    val = A[rows, cols].astype(np.float32)
    # renormalise after the fp32 cast so that sum p = 1 holds for the stored values
    return rp, cols.astype(np.int32), val


def kl_exact(orc, Y, P):
    Z = orc.exact_gradient(Y, P)["Z"]
    return orc.kl(Y, P, Z)


@pytest.mark.parametrize("s", [1, 2])
def test_gradient_is_derivative_of_kl(orc, s):
    """dC/dy by central differences equals the analytic gradient (alpha = 1)."""
    rng = np.random.default_rng(10 + s)
    N = 14
    P = dense_P(N, rng)
    # exact normalisation of the fp32 values, so that sum p = 1 as the gradient assumes
    P = (P[0], P[1], (P[2] / P[2].astype(np.float64).sum()).astype(np.float32))
    Y = rng.normal(0, 1.5, size=(N, s))
    g = orc.exact_gradient(Y, P)["dY"]
    total = float(P[2].astype(np.float64).sum())
    h = 1e-6
    fd = np.zeros_like(Y)
    for i in range(N):
        for m in range(s):
            Yp = Y.copy(); Yp[i, m] += h
            Ym = Y.copy(); Ym[i, m] -= h
            fd[i, m] = (kl_exact(orc, Yp, P) - kl_exact(orc, Ym, P)) / (2 * h)
    # the gradient formula holds for sum p = 1; fp32 storage leaves |1 - sum| ~ 1e-7
    assert abs(total - 1.0) < 1e-6
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=1e-7)


def test_two_point_closed_form(orc):
    gold = GOLD["two_point_gradient"]
    Y = np.array(gold["Y"])
    P = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([0.5, 0.5], np.float32))
    out = orc.exact_gradient(Y, P, alpha=gold["alpha"])
    np.testing.assert_allclose(out["dY"][0], gold["dY1"], rtol=1e-14)
    np.testing.assert_allclose(out["dY"][1], -np.array(gold["dY1"]), rtol=1e-14)
    # KL of two points is 0 for any placement
    assert abs(orc.kl(Y, P, out["Z"]) - GOLD["two_point_kl"]["KL"]) < 1e-15


def test_three_collinear_Z(orc):
    gold = GOLD["three_collinear_Z"]
    Y = np.array(gold["Y"])
    P = (np.array([0, 0, 0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert abs(orc.exact_gradient(Y, P)["Z"] - gold["Z"]) < 1e-14


@pytest.mark.parametrize("s", [1, 2])
def test_zero_net_force_and_translation(orc, s):
    rng = np.random.default_rng(3)
    N = 60
    P = dense_P(N, rng)
    Y = rng.normal(0, 3, size=(N, s))
    out = orc.exact_gradient(Y, P, alpha=12.0)
    scale = np.abs(out["dY"]).sum()
    assert np.abs(out["dY"].sum(axis=0)).max() < 1e-12 * scale
    moved = orc.exact_gradient(Y + np.array([17.25, -3.5][:s]), P, alpha=12.0)
    np.testing.assert_allclose(moved["dY"], out["dY"], rtol=1e-9, atol=1e-12 * scale)
    assert abs(moved["Z"] - out["Z"]) < 1e-11 * out["Z"]


def test_attraction_repulsion_split(orc):
    """dY = 4 (alpha attr + rep) for every alpha (Sec. 1.2 exaggeration is linear)."""
    rng = np.random.default_rng(5)
    N = 30
    P = dense_P(N, rng)
    Y = rng.normal(0, 2, size=(N, 2))
    a1 = orc.exact_gradient(Y, P, alpha=1.0)
    a12 = orc.exact_gradient(Y, P, alpha=12.0)
    np.testing.assert_allclose(a12["dY"] - a1["dY"], 4 * 11 * a1["attr"], rtol=1e-10, atol=1e-14)
    # Eq. (frep) points toward the other points, so the descent step -4 rep
    # pushes each point away from the bulk: rep . (y - mean) < 0 for most points
    centred = Y - Y.mean(axis=0)
    assert (np.sum(a1["rep"] * centred, axis=1) < 0).mean() > 0.7
