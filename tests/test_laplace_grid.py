"""The library's minimax Laplace grid (host entry point ltgw_laplace_grid),
checked against the function it approximates: 1/X on [a, b]."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2307_04508_gb300 import build, ltgw
    build.build()
    ltgw.load()
    return ltgw


def _err_curve(x, w, a, b, n=40000):
    X = np.exp(np.linspace(np.log(a), np.log(b), n))
    return X, (1.0 / X - np.exp(-np.outer(X, x)) @ w) * a


@pytest.mark.parametrize("k", [4, 6, 8, 10])
def test_reported_error_is_the_measured_one(L, k):
    a, b = 0.07, 1.4e4
    x, w, err = L.laplace_grid(k, a, b)
    assert np.all(x > 0) and np.all(w > 0) and np.all(np.diff(x) > 0)
    _, r = _err_curve(x, w, a, b)
    assert abs(np.abs(r).max() - err) <= 1e-3 * err


@pytest.mark.parametrize("k", [4, 6, 8])
def test_equioscillation(L, k):
    # minimax: the error alternates 2k+1 times with (nearly) equal magnitude
    a, b = 0.5, 1e4
    x, w, err = L.laplace_grid(k, a, b)
    X, r = _err_curve(x, w, a, b)
    sg = np.sign(r)
    runs, start = [], 0
    for i in range(1, len(r) + 1):
        if i == len(r) or sg[i] != sg[start]:
            runs.append(np.abs(r[start:i]).max())
            start = i
    assert len(runs) >= 2 * k + 1
    big = sorted(runs)[-(2 * k + 1):]
    assert min(big) > 0.97 * max(big)


def test_error_falls_with_points_and_beats_trapezoid(L):
    a, b = 0.07, 1e4
    errs = [L.laplace_grid(k, a, b)[2] for k in (4, 6, 8, 10, 14)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    # best trapezoid rule in log(tau) with 8 points, over a parameter scan
    best = 1e9
    X = np.exp(np.linspace(np.log(a), np.log(b), 4000))
    for h in np.linspace(0.3, 4, 40):
        for t0 in np.linspace(-np.log(b) - 4, 2, 60):
            t = t0 + h * np.arange(8)
            r = (1 / X - np.exp(-np.outer(X, np.exp(t))) @ (h * np.exp(t))) * a
            best = min(best, np.abs(r).max())
    assert errs[2] < 0.2 * best


def test_scaling_to_the_interval(L):
    # the grid for [s a, s b] is the grid for [a, b] with x/s and w/s
    x1, w1, e1 = L.laplace_grid(6, 0.3, 3e3)
    x2, w2, e2 = L.laplace_grid(6, 0.6, 6e3)
    assert np.allclose(x2, x1 / 2, rtol=1e-6) and np.allclose(w2, w1 / 2, rtol=1e-6)
    assert abs(e1 - e2) < 1e-6 * e1
