"""Oracle pins for the direct-sampling statistics of Sec. 3: the drag
autocorrelation and correlation time (caption of Fig. pdf_drag) and the
waiting-time return time r(a).  Checked on hand-counted series and on a
stationary AR(1) series (the OU process sampled at a fixed step), whose
autocorrelation rho^tau and per-step upcrossing probability P(X < a <= Y)
(bivariate normal) are known exactly."""
import numpy as np
import pytest


def test_autocorrelation_small_cases(orc):
    c, tc = orc.autocorrelation(np.array([1.0, -1.0, 1.0, -1.0, 1.0, -1.0]), 2)
    assert c[0] == 1.0 and abs(c[1] + 1.0) < 1e-15 and abs(c[2] - 1.0) < 1e-15 and tc == 1
    # a slow sine: C(tau) ~ cos(omega tau); zero near a quarter period
    t = np.arange(20000)
    c, tc = orc.autocorrelation(np.sin(2 * np.pi * t / 400.0), 150)
    assert abs(tc - 100) <= 1
    assert np.allclose(c[:50], np.cos(2 * np.pi * np.arange(50) / 400.0), atol=1e-2)
    # the correlation of the fluctuations: a constant offset changes nothing
    c2, tc2 = orc.autocorrelation(np.array([1.0, -1.0, 1.0, -1.0, 1.0, -1.0]) + 7.0, 2)
    assert np.allclose(c2, [1.0, -1.0, 1.0], atol=1e-14) and tc2 == 1


def ar1(rng, rho, n, length):
    x = np.zeros((n, length))
    x[:, 0] = rng.standard_normal(n)
    s = np.sqrt(1 - rho * rho)
    for t in range(1, length):
        x[:, t] = rho * x[:, t - 1] + s * rng.standard_normal(n)
    return x


def test_autocorrelation_of_ar1(orc):
    rng = np.random.default_rng(1)
    rho = 0.9
    x = ar1(rng, rho, 16, 20000)
    c, tc = orc.autocorrelation(x, 40)
    assert np.allclose(c, rho ** np.arange(41), atol=0.02)
    assert tc == -1 or tc > 30


def test_return_times_hand_counted(orc):
    d = np.array([[0, 2, 0, 0, 3, 3, 0, 2, 0, 0, 0, 5]], dtype=float)
    ev, r = orc.return_times(d, [1.0, 2.5, 10.0], gap=0)
    assert list(ev) == [4, 2, 0] and r[0] == 12 / 4 and r[1] == 12 / 2 and np.isinf(r[2])
    # gap 2: the up-crossing at t = 4 follows t = 1 by 3 > 2 (a new event); at
    # t = 7 it follows t = 5 by 2 (the same fluctuation)
    ev, _ = orc.return_times(d, [1.0], gap=2)
    assert ev[0] == 3
    # a series that starts above the level: no up-crossing at t = 0
    ev, _ = orc.return_times(np.array([5.0, 5.0, 0.0, 5.0]), [1.0], gap=0)
    assert ev[0] == 1


def test_return_time_of_ar1_matches_the_upcrossing_probability(orc):
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(2)
    rho, n, length = 0.8, 32, 20000
    x = ar1(rng, rho, n, length)
    levels = [0.5, 1.5]
    ev, r = orc.return_times(x, levels, gap=0)
    for a, e, rr in zip(levels, ev, r):
        cov = [[1.0, rho], [rho, 1.0]]
        p_below_both = multivariate_normal(mean=[0, 0], cov=cov).cdf([a, a])
        from scipy.stats import norm
        p_up = norm.cdf(a) - p_below_both          # P(X < a, Y >= a)
        expected = n * (length - 1) * p_up
        assert abs(e - expected) < 4 * np.sqrt(expected), (a, e, expected)
        assert abs(rr * p_up - 1) < 0.05
