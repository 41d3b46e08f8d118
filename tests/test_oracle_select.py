"""Pins of the oracle's GKTL and AMS selection rules and of both algorithms on
the Ornstein-Uhlenbeck process of App. B.2, against closed forms and brute
force."""
import numpy as np
import pytest

from tests import seeded_inputs as si


def counts(parent, n):
    return np.bincount(parent, minlength=n)


# ---------------------------------------------------------------- GKTL weights
def test_weights_sum_to_n_and_normaliser(orc):
    """eq. (Weight): W_n = e^{s_n}/R, R = (1/N) sum e^{s_n}, sum W = N."""
    s = si.log_weights(64, 1, spread=3.0)
    W, logR = orc.gktl_weights(s)
    assert abs(W.sum() - 64) < 1e-12
    assert abs(logR - np.log(np.mean(np.exp(s)))) < 1e-13
    assert np.allclose(W, np.exp(s) / np.mean(np.exp(s)), rtol=1e-13)
    # shifting every exponent shifts log R only
    W2, logR2 = orc.gktl_weights(s + 700.0)
    assert np.allclose(W2, W, rtol=1e-13) and abs(logR2 - logR - 700.0) < 1e-10


def test_k_zero_is_direct_sampling(orc):
    """k = 0 (no bias): every weight is one and every trajectory keeps its slot."""
    W, logR = orc.gktl_weights(np.zeros(37))
    assert np.all(W == 1.0) and logR == 0.0
    for it in range(20):
        assert np.array_equal(orc.gktl_select(W, 5, it), np.arange(37))


def test_integer_weights_are_copied_exactly(orc):
    """Integer weights have no residual: exactly W_n copies, extras fill the
    emptied slots in ascending order."""
    W = np.array([2.0, 0.0, 1.0, 0.0, 3.0, 1.0, 0.0, 1.0])
    p = orc.gktl_select(W, 1, 0)
    assert list(p) == [0, 0, 2, 4, 4, 5, 4, 7]


@pytest.mark.parametrize("n,spread,draws", [(4, 0.8, 40000), (32, 0.7, 8000)])
def test_selection_mean_copies_equal_weights(orc, n, spread, draws):
    """eq. (Weight): trajectory n is continued W_n times on average while the
    ensemble stays at N (brute force; 4 standard errors)."""
    W = si.normalised_weights(n, 4, spread=spread)
    acc = np.zeros(n)
    acc2 = np.zeros(n)
    for it in range(draws):
        p = orc.gktl_select(W, 2024, it)
        c = counts(p, n)
        assert c.sum() == n
        # minimal-variance copy numbers: floor(W) or floor(W) + 1
        assert np.all((c - np.floor(W) >= 0) & (c - np.floor(W) <= 1))
        for i in np.nonzero(c)[0]:
            assert p[i] == i  # a surviving trajectory keeps its slot
        acc += c
        acc2 += c * c
    mean = acc / draws
    se = np.sqrt(np.maximum(acc2 / draws - mean ** 2, 1e-12) / draws)
    assert np.all(np.abs(mean - W) < 4 * se + 1e-12), (mean, W, se)


def test_selection_rejects_weights_not_summing_to_n(orc):
    with pytest.raises(ValueError):
        orc.gktl_select(np.array([1.0, 1.5, 1.0]), 0, 0)


def test_selection_rejects_bad_weights(orc):
    with pytest.raises(ValueError):
        orc.gktl_select(np.array([1.0, np.nan, 1.0]), 0, 0)
    with pytest.raises(ValueError):
        orc.gktl_weights(np.array([0.0, np.inf]))


# ---------------------------------------------------------------- AMS selection
def test_ams_kills_minimum_and_draws_survivors(orc):
    Q = si.scores(32, 3)
    killed, surv, z = orc.ams_select(Q, 9, 1)
    assert z == Q.min()
    assert list(killed) == [int(np.argmin(Q))]
    assert surv[0] != killed[0] and 0 <= surv[0] < 32


def test_ams_ties_all_killed(orc):
    Q = si.scores(40, 5, n_ties=3)
    killed, surv, z = orc.ams_select(Q, 1, 4)
    assert len(killed) == 3 and np.all(Q[killed] == z)
    assert np.all(Q[surv] > z)
    Qe = np.full(6, 2.5)
    killed, surv, z = orc.ams_select(Qe, 1, 1)
    assert len(killed) == 6 and len(surv) == 0


def test_ams_survivor_uniform(orc):
    """Survivor drawn uniformly among the N - |K| others (chi-square, 20000 draws)."""
    Q = np.arange(8, dtype=float)
    hits = np.zeros(8)
    n = 20000
    for it in range(n):
        _, surv, _ = orc.ams_select(Q, 77, it)
        hits[surv[0]] += 1
    assert hits[0] == 0
    exp = n / 7
    chi2 = ((hits[1:] - exp) ** 2 / exp).sum()
    assert chi2 < 22.5  # 6 dof, p = 0.001


# ---------------------------------------------------------------- OU process
def var_time_integral(M, dt):
    """Variance of dt * sum_{m=1}^M x_m for the stationary AR(1) with
    x_{m+1} = a x_m + noise, a = e^{-dt}, Var x = 1/2:
    dt^2 (1/2) [M + 2 sum_{j=1}^{M-1} (M - j) a^j]."""
    a = np.exp(-dt)
    j = np.arange(1, M)
    return dt * dt * 0.5 * (M + 2.0 * np.sum((M - j) * a ** j))


def test_ou_time_integral_variance_continuum_limit():
    """The discrete variance tends to T - 1 + e^{-T} (App. B.2 process, tau_c = 1)."""
    T = 10.0
    for dt in (0.01, 0.001):
        M = int(round(T / dt))
        assert abs(var_time_integral(M, dt) - (T - 1 + np.exp(-T))) < 2 * dt * T


@pytest.mark.parametrize("k", [0.5, 1.0, 2.0])
def test_ou_gktl_normaliser_matches_scgf(orc, k):
    """App. C.1, eq. (mean_field): Z = prod R_i estimates E_0[exp(k int A)], which
    for the Gaussian OU integral is exp(k^2 Var/2) (T_a = 10, tau = 0.5, N = 1024,
    20 replicas; 3 standard errors plus the O(1/N) bias of the estimator)."""
    dt, P, periods = 0.05, 10, 20
    V = var_time_integral(P * periods, dt)
    zs, means = [], []
    for r in range(20):
        logZ, fi, _ = orc.ou_gktl(1024, periods, P, dt, k, 100 + r)
        zs.append(logZ)
        means.append(fi.mean())
    zs = np.array(zs)
    se = zs.std(ddof=1) / np.sqrt(len(zs))
    exact = k * k * V / 2
    assert abs(zs.mean() - exact) < 3 * se + 0.01 * exact
    # tilted mean of the time integral is k Var (Gaussian)
    means = np.array(means)
    se_m = means.std(ddof=1) / np.sqrt(len(means))
    assert abs(means.mean() - k * V) < 3 * se_m + 0.05 * k * V


def test_ou_gktl_k0_is_unbiased(orc):
    logZ, fi, _ = orc.ou_gktl(256, 10, 10, 0.05, 0.0, 3)
    assert logZ == 0.0


def test_ou_ams_matches_direct_sampling(orc):
    """App. B.2: AMS with score x on N = 32 trajectories of duration T_a = 5
    estimates P(max x >= a); 50 runs against 2e5 direct trajectories."""
    levels = [1.5, 2.0, 2.5]
    direct = orc.ou_direct_max(200000, 100, 0.05, 7, levels)
    for a, pd in zip(levels, direct):
        ps = np.array([orc.ou_ams(32, 100, 0.05, a, 2000, 1000 + s)[0] for s in range(50)])
        se = np.sqrt(ps.var(ddof=1) / len(ps) + pd * (1 - pd) / 200000)
        assert abs(ps.mean() - pd) < 3 * se, (a, ps.mean(), pd, se)
