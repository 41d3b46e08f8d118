"""Pins of the oracle's estimator helpers (oracle/__init__.py): the GKTL
exponent's window sum (eq. Weight), the time-averaged drag and its maximum
(eq. def_time_averaged_drag), the GKTL probability and return-time estimator
(App. C.2, eq. Biased_Path_Approximation inverted), with and without a
potential in the exponents, and the generalised AMS estimator (App. B.1).

Each is tied to something other than itself: hand-computed short series, a
second implementation in the C oracle, the closed form of a Poisson process,
and brute-force direct sampling of the Ornstein-Uhlenbeck process of App. B.2
with numpy's own generator."""
import numpy as np
import pytest

DT, STEPS_PER_PERIOD, PERIODS, WINDOW = 0.05, 10, 20, 40  # T_a = 10, tau = 0.5, T = 2
LEVELS = np.array([1.25, 1.5, 1.75])


def ou_direct_window_max(n, n_steps, window, dt, seed, chunk=20000):
    """max over t in [T, T_a] of the trailing mean of x over `window` steps, for
    n independent stationary OU paths (x_{m+1} = a x_m + sqrt((1 - a^2)/2) xi,
    numpy's generator; brute force, independent of the oracle's code)"""
    a = np.exp(-dt)
    sig = np.sqrt((1 - a * a) / 2)
    rng = np.random.default_rng(seed)
    out = []
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        x = np.sqrt(0.5) * rng.standard_normal(m)
        cum = np.zeros((m, n_steps + 1))
        for s in range(n_steps):
            x = a * x + sig * rng.standard_normal(m)
            cum[:, s + 1] = cum[:, s] + x
        out.append(np.max((cum[:, window:] - cum[:, :-window]) / window, axis=1))
    return np.concatenate(out)


@pytest.fixture(scope="module")
def direct():
    """P(max F_T >= a) from 2e5 direct OU paths of the GKTL set-up, with its
    binomial standard error"""
    mx = ou_direct_window_max(200000, PERIODS * STEPS_PER_PERIOD, WINDOW, DT, 2024)
    p = np.array([(mx >= a).mean() for a in LEVELS])
    return p, np.sqrt(p * (1 - p) / mx.size)


# ---------------------------------------------------------------- window sums and time averages
def test_window_sum_hand_computed(orc):
    """eq. (Weight): s_n = k sum of the drag over steps t0 < t <= t1; drag[n, t-1]
    is the drag after step t"""
    d = np.array([[1.0, 2.0, 3.0, 4.0, 5.0], [-1.0, 0.5, 0.25, 8.0, 16.0]])
    assert np.array_equal(orc.window_sum(d, 1, 3, 2.0), [2.0 * (2 + 3), 2.0 * (0.5 + 0.25)])
    assert np.array_equal(orc.window_sum(d, 0, 5, 1.0), [15.0, 23.75])
    assert np.array_equal(orc.window_sum(d, 4, 5, -1.0), [-5.0, -16.0])  # only the last step
    assert np.array_equal(orc.window_sum(d, 2, 2, 3.0), [0.0, 0.0])  # empty window


def test_trailing_mean_max_hand_computed(orc):
    """eq. (def_time_averaged_drag): F_T(t) = (1/T) sum_{s=t-T+1}^{t} D(s), maximised
    over t in [t_begin + T, t_end]; a spike in the first step (before t_begin)
    and one in the last step catch a window shifted either way"""
    d = np.array([[8.0, 0.0, 0.0, 0.0, 0.0, 4.0]])
    assert orc.trailing_mean_max(d, 2, 6, t_begin=1)[0] == 2.0  # (0 + 4)/2; the 8 lies before t_begin
    assert orc.trailing_mean_max(d, 2, 6)[0] == 4.0  # (8 + 0)/2 from t_begin = 0
    assert orc.trailing_mean_max(d, 2, 5, t_begin=1)[0] == 0.0  # the 4 comes after t_end
    assert orc.trailing_mean_max(d, 1, 6)[0] == 8.0  # T = 1: the series itself
    assert orc.trailing_mean_max(d, 6, 6)[0] == 2.0  # one window: the whole series
    assert orc.trailing_mean_max(d, 3, 4, t_begin=2)[0] == -np.inf  # no window fits
    e = np.array([[1.0, 3.0, -2.0, 5.0], [0.0, 0.0, 6.0, 0.0]])
    assert np.array_equal(orc.trailing_mean_max(e, 2, 4), [2.0, 3.0])  # means (2, 0.5, 1.5) and (0, 3, 3)


def test_trailing_mean_max_matches_the_c_oracle(orc):
    """the C oracle's own window loop over the final GKTL histories (a second
    implementation) gives the same maxima"""
    o = orc.ou_gktl(64, 6, 10, DT, 0.8, 3, window_steps=15, full=True)
    assert np.allclose(orc.trailing_mean_max(o["hist"][:, 1:], 15), o["max_mean"], rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- return time
def test_return_time_of_a_poisson_process(orc):
    """App. C.2: for events at rate 1/r in time, the probability of at least
    one in T_a - T is P = 1 - e^{-(T_a - T)/r}, and r(a) = -(T_a - T)/ln(1 - P)
    returns r exactly; simulated exponential waiting times agree within their
    standard error"""
    t_a, t = 50.0, 10.0
    for r in (10.0, 40.0, 1e6):
        p = 1.0 - np.exp(-(t_a - t) / r)
        assert abs(orc.return_time(np.array([p]), t_a, t)[0] - r) < 1e-9 * r
    rng = np.random.default_rng(5)
    r = 60.0
    first = rng.exponential(r, 200000)  # time of the first event of each experiment
    p = (first <= t_a - t).mean()
    se = np.sqrt(p * (1 - p) / first.size)
    lo, hi = orc.return_time(np.array([p + 3 * se, p - 3 * se]), t_a, t)
    assert lo < r < hi
    assert np.isinf(orc.return_time(np.array([0.0]), t_a, t)[0])


# ---------------------------------------------------------------- GKTL estimator
def gktl_replicas(orc, k, kappa, reps, n=1024):
    """App. C.2 estimator over independent GKTL runs on the OU process; the
    maxima come from the final histories through trailing_mean_max.  Returns
    (mean, standard error) with the potential's correction and without it."""
    ps, raw = [], []
    for r in range(reps):
        o = orc.ou_gktl(n, PERIODS, STEPS_PER_PERIOD, DT, k, 500 + r, kappa=kappa, full=True)
        maxima = orc.trailing_mean_max(o["hist"][:, 1:], WINDOW)
        integ = DT * o["hist"][:, 1:].sum(axis=1)
        assert np.allclose(integ, o["integrals"], rtol=1e-12, atol=1e-12)
        ps.append(orc.gktl_probability(o["log_z"], k, o["integrals"], maxima, LEVELS, o["correction"]))
        raw.append(orc.gktl_probability(o["log_z"], k, o["integrals"], maxima, LEVELS))
    ps, raw = np.array(ps), np.array(raw)
    return ((ps.mean(axis=0), ps.std(axis=0, ddof=1) / np.sqrt(reps)),
            (raw.mean(axis=0), raw.std(axis=0, ddof=1) / np.sqrt(reps)))


def agree(est, se, direct, bias=0.1):
    """within 3 combined standard errors plus the O(1/N) bias of GKTL (a
    fraction of the probability)"""
    p_dir, se_dir = direct
    return np.abs(est - p_dir) < 3 * np.sqrt(se ** 2 + se_dir ** 2) + bias * p_dir


@pytest.mark.parametrize("k", [0.5, 1.0])
def test_gktl_estimator_matches_direct_sampling(orc, direct, k):
    """P(max F_T >= a) from GKTL tilted by e^{k int x} (N = 1024, T_a = 10,
    cloning every 0.5, T = 2) against 2e5 direct paths, at levels down to
    P = 5e-3 where the tilt matters; the estimator with the exponent's sign
    flipped is far off"""
    (est, se), _ = gktl_replicas(orc, k, 0.0, 24)
    assert np.all(agree(est, se, direct)), (est, se, direct[0])
    o = orc.ou_gktl(1024, PERIODS, STEPS_PER_PERIOD, DT, k, 77, full=True)
    maxima = orc.trailing_mean_max(o["hist"][:, 1:], WINDOW)
    flipped = orc.gktl_probability(o["log_z"], -k, o["integrals"], maxima, LEVELS)
    assert np.all(flipped > 10 * direct[0])


def test_gktl_with_potential_matches_direct_sampling(orc, direct):
    """The learned score's role in GKTL: a potential kappa (V(x_{t_i}) -
    V(x_{t_{i-1}})), V = x, added to every exponent; with each final trajectory
    weighted by e^{-kappa (V(T_a) - V(0))} the estimate still matches direct
    sampling, and without that correction it does not"""
    (est, se), (raw, raw_se) = gktl_replicas(orc, 0.5, 1.0, 24)
    assert np.all(agree(est, se, direct)), (est, se, direct[0])
    assert np.all(~agree(raw, raw_se, direct)), (raw, raw_se, direct[0])


def test_gktl_potential_bookkeeping(orc):
    """kappa = 0 leaves the run untouched; the correction is kappa times the
    final x minus the start of the same genealogy (the first element of each
    final history); the per-period log R add up to log Z"""
    a = orc.ou_gktl(128, 5, 10, DT, 0.7, 9, full=True)
    b = orc.ou_gktl(128, 5, 10, DT, 0.7, 9, kappa=0.0, full=True)
    assert a["log_z"] == b["log_z"] and np.array_equal(a["hist"], b["hist"])
    assert np.all(a["correction"] == 0.0)
    c = orc.ou_gktl(128, 5, 10, DT, 0.7, 9, kappa=1.5, full=True)
    assert np.allclose(c["correction"], 1.5 * (c["hist"][:, -1] - c["hist"][:, 0]), rtol=0, atol=1e-15)
    assert abs(c["log_r"].sum() - c["log_z"]) < 1e-13
    assert not np.array_equal(c["hist"], a["hist"])  # the potential changes the selection


# ---------------------------------------------------------------- AMS estimator
def test_ams_probability_hand_computed(orc):
    """generalised AMS: prod_j (1 - |K_j|/N) times the fraction of the final
    maxima at or above the level: two iterations killing one of four, two of
    four maxima >= 1.5 -> (3/4)^2 / 2"""
    lw = 2 * np.log1p(-1 / 4)
    q = np.array([0.1, 2.0, 3.0, 1.0])
    assert abs(orc.ams_probability(lw, q, 1.5) - 9 / 32) < 1e-15
    assert abs(orc.ams_probability(lw, q, 2.0) - 9 / 32) < 1e-15  # a maximum equal to the level counts
    assert orc.ams_probability(lw, q, 3.5) == 0.0
    assert orc.ams_probability(0.0, q, -1.0) == 1.0


def test_ams_estimator_with_another_score_matches_direct_sampling(orc):
    """App. B.1 with a score that is not the event's observable (as the learned
    score is): the trailing mean of x over 10 steps seen every 5 steps drives
    the kills and branches, the event is max x >= a.  The estimator on the
    returned weights, maxima and killed records equals the C oracle's own, and
    its mean over 40 runs (N = 32, T_a = 5, 60 iterations) matches 2e5 direct
    paths; the final ensemble alone (killed trajectories left out) falls short
    at a = 1.5"""
    n_steps, levels = 100, [1.5, 2.0]
    pd = orc.ou_direct_max(200000, n_steps, DT, 7, levels)
    for a, p_dir in zip(levels, pd):
        ps, finals = [], []
        for s in range(40):
            p, it, lw, mx, killed = orc.ou_ams_score(32, n_steps, DT, 5, 10, np.inf, a, 60, 3000 + s)
            assert it == 60 and len(killed[0]) >= 60
            assert orc.ams_probability(lw, mx, a, killed) == pytest.approx(p, rel=1e-13, abs=0)
            ps.append(p)
            finals.append(orc.ams_probability(lw, mx, a))
        ps, finals = np.array(ps), np.array(finals)
        se = np.sqrt(ps.var(ddof=1) / len(ps) + p_dir * (1 - p_dir) / 200000)
        assert abs(ps.mean() - p_dir) < 3 * se, (a, ps.mean(), p_dir, se)
        if a == levels[0]:  # 0.08 against 0.27: the events of killed trajectories are missing
            se_f = np.sqrt(finals.var(ddof=1) / len(finals) + p_dir * (1 - p_dir) / 200000)
            assert p_dir - finals.mean() > 3 * se_f, (a, finals.mean(), p_dir)


def test_ams_killed_records_with_the_event_as_score(orc):
    """With the event's observable as the score (score x at every step, stop at
    a), every killed trajectory lies below a: its records add nothing, and the
    estimate is the final ensemble's"""
    for s in range(5):
        p, it, lw, mx, killed = orc.ou_ams_score(32, 100, DT, 1, 1, 2.0, 2.0, 400, 50 + s)
        assert len(killed[0]) >= it and np.all(killed[1] < 2.0)
        assert p == orc.ams_probability(lw, mx, 2.0)
        assert p == orc.ou_ams(32, 100, DT, 2.0, 400, 50 + s)[0]
