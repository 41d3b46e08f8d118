"""GPU GKTL and AMS drivers and their estimators, through the C ABI: the
drivers equal the composition of the documented calls, k = 0 reduces GKTL to
direct sampling, the estimator kernels match the oracle's FP64 formulas, and
the AMS run keeps its invariants."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SMALL = dict(nx=64, ny=24, obstacle=(12, 9, 6, 6), tau=0.6, gx=1e-5)


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


def make(L, n, seed, **kw):
    cfg = L.config(**dict(SMALL, **kw))
    return L.lbm_ensemble_create(cfg, n, seed, torch.cuda.current_stream()), cfg


def pops(L, e, cfg, n):
    return np.stack([L.lbm_ensemble_get_populations(e, c, cfg.nx, cfg.ny) for c in range(n)])


def zeros(n, dtype=torch.float64):
    return torch.zeros(n, dtype=dtype, device="cuda")

def window_max(d, window, t_end=None):
    """largest mean of `window` consecutive drag values of each row, windows
    ending at steps window .. t_end: a check of the drivers' own bookkeeping on
    their own drag history (the oracle's time averages are compared on seeded
    series elsewhere)"""
    d = np.asarray(d, dtype=np.float64)
    t_end = d.shape[1] if t_end is None else t_end
    c = np.concatenate([np.zeros((d.shape[0], 1)), np.cumsum(d[:, :t_end], axis=1)], axis=1)
    return np.max((c[:, window:] - c[:, :-window]) / window, axis=1)



def test_gktl_k0_is_direct_sampling(L, orc):
    n, period, periods = 16, 20, 5
    e, cfg = make(L, n, 3, max_steps=200, n_snapshots=2)
    try:
        logR, parent = zeros(periods), zeros(periods * n, torch.int32)
        integ, maxima = zeros(n), zeros(n)
        L.lbm_gktl_run(e, period, periods, 0.0, 0.0, 9, 30, logR, parent, integ, maxima)
        assert torch.all(logR == 0)
        assert np.array_equal(parent.cpu().numpy().reshape(periods, n), np.tile(np.arange(n), (periods, 1)))
        d = np.zeros((n, period * periods))
        L.lbm_ensemble_drag(e, 0, period * periods, d)
        assert np.allclose(integ.cpu().numpy(), d.sum(axis=1), rtol=1e-12, atol=1e-15)
        assert np.allclose(maxima.cpu().numpy(), window_max(d, 30), rtol=1e-11, atol=1e-14)
        # with k = 0 the estimator is the plain fraction of trajectories above a
        levels = torch.tensor(np.quantile(maxima.cpu().numpy(), [0.1, 0.5, 0.9]), device="cuda")
        p = zeros(3)
        L.gktl_probability(0.0, logR, integ, maxima, levels, 100.0, 30.0, p)
        frac = [(maxima.cpu().numpy() >= a).mean() for a in levels.cpu().numpy()]
        assert np.allclose(p.cpu().numpy(), frac, rtol=1e-14)
    finally:
        L.lbm_ensemble_destroy(e)


def test_gktl_run_equals_its_composition(L):
    """lbm_gktl_run is exactly step + window_sum + gktl_weights + gktl_select +
    clone per period, with iter = period index."""
    n, period, periods, k, eps, seed = 12, 15, 4, 40.0, 0.002, 5
    e1, cfg = make(L, n, 7, max_steps=100, n_snapshots=3)
    e2, _ = make(L, n, 7, max_steps=100, n_snapshots=3)
    try:
        stream = torch.cuda.current_stream()
        for e in (e1, e2):
            L.lbm_ensemble_step(e, 10)
            L.lbm_ensemble_set_snapshots(e, [1, 4, 7])
        logR, parent = zeros(periods), zeros(periods * n, torch.int32)
        L.lbm_gktl_run(e1, period, periods, k, eps, seed, 0, logR, parent)
        s, W, lr = zeros(n), zeros(n), zeros(periods)
        par = zeros(periods * n, torch.int32)
        st = zeros(1, torch.int32)
        for i in range(periods):
            t0 = 10 + i * period
            L.lbm_ensemble_step(e2, period)
            L.lbm_ensemble_window_sum(e2, t0, t0 + period, k, s)
            L.gktl_weights(s, W, lr[i:i + 1], stream)
            L.gktl_select(W, seed, i, par[i * n:(i + 1) * n], st, stream)
            L.lbm_ensemble_clone(e2, par[i * n:(i + 1) * n], eps, seed, i)
        torch.cuda.synchronize()
        assert torch.equal(logR, lr) and torch.equal(parent, par)
        assert np.array_equal(pops(L, e1, cfg, n), pops(L, e2, cfg, n))
        assert (parent.cpu().numpy().reshape(periods, n) != np.arange(n)).any()  # cloning happened
    finally:
        L.lbm_ensemble_destroy(e1)
        L.lbm_ensemble_destroy(e2)


def test_gktl_probability_matches_oracle(L, orc):
    rng = np.random.default_rng(11)
    n, periods = 300, 7
    logR = rng.normal(0.1, 0.05, periods)
    integ = rng.normal(0.0, 2.0, n)
    maxima = rng.normal(0.0, 1.0, n)
    levels = np.array([-1.0, 0.0, 0.5, 1.5, 2.5, 10.0])
    k = 0.7
    p, r = zeros(len(levels)), zeros(len(levels))
    L.gktl_probability(k, torch.tensor(logR, device="cuda"), torch.tensor(integ, device="cuda"),
                       torch.tensor(maxima, device="cuda"), torch.tensor(levels, device="cuda"), 50.0, 10.0, p, r)
    p_ref = orc.gktl_probability(logR.sum(), k, integ, maxima, levels)
    assert np.allclose(p.cpu().numpy(), p_ref, rtol=1e-13, atol=0)
    with np.errstate(invalid="ignore"):
        r_ref = orc.return_time(p_ref, 50.0, 10.0)  # P >= 1 (synthetic weights) has no return time
    got = r.cpu().numpy()
    assert np.allclose(got, r_ref, rtol=1e-12, equal_nan=True)
    assert np.isinf(got[-1]) and got[-1] > 0  # P = 0 above every maximum


def test_gktl_probability_with_potential_on_an_oracle_run(L, orc):
    """App. C.2 with a potential in the exponents: the estimator kernel, given
    the per-period log R, integrals, window maxima and corrections of an oracle
    GKTL run on the OU process (k = 0.5, kappa = 1, V = x), equals the
    oracle's estimator (pinned against brute-force sampling on the CPU)"""
    o = orc.ou_gktl(1024, 20, 10, 0.05, 0.5, 501, kappa=1.0, full=True)
    maxima = orc.trailing_mean_max(o["hist"][:, 1:], 40)
    levels = np.array([0.5, 1.0, 1.25, 1.5, 1.75, 5.0])
    dev = {k: torch.tensor(v, device="cuda") for k, v in
           dict(logR=o["log_r"], integ=o["integrals"], maxima=maxima, corr=o["correction"], levels=levels).items()}
    p, r = zeros(len(levels)), zeros(len(levels))
    L.gktl_probability(0.5, dev["logR"], dev["integ"], dev["maxima"], dev["levels"], 10.0, 2.0, p, r,
                       correction_dev=dev["corr"])
    p_ref = orc.gktl_probability(o["log_z"], 0.5, o["integrals"], maxima, levels, o["correction"])
    assert np.allclose(p.cpu().numpy(), p_ref, rtol=1e-12, atol=0)
    assert np.allclose(r.cpu().numpy()[:-1], orc.return_time(p_ref, 10.0, 2.0)[:-1], rtol=1e-12)
    p_raw = zeros(len(levels))  # without the correction the kernel gives the oracle's uncorrected sum
    L.gktl_probability(0.5, dev["logR"], dev["integ"], dev["maxima"], dev["levels"], 10.0, 2.0, p_raw)
    assert np.allclose(p_raw.cpu().numpy(), orc.gktl_probability(o["log_z"], 0.5, o["integrals"], maxima, levels),
                       rtol=1e-12, atol=0)


def test_ams_probability_with_killed_records_on_an_oracle_run(L, orc):
    """Generalised AMS with a score other than the event (App. B.1): the
    estimator kernel, given the final maxima and the killed records of an
    oracle AMS run on the OU process, equals the oracle's estimator"""
    p_orc, it, lw, mx, (rl, rm) = orc.ou_ams_score(32, 100, 0.05, 5, 10, np.inf, 1.5, 60, 3007)
    levels = np.array([0.5, 1.0, 1.5, 2.0, 2.5])
    p = zeros(len(levels))
    L.ams_probability(lw, torch.tensor(mx, device="cuda"), torch.tensor(levels, device="cuda"), p,
                      records=(torch.tensor(rl, device="cuda"), torch.tensor(rm, device="cuda")))
    ref = [orc.ams_probability(lw, mx, a, (rl, rm)) for a in levels]
    assert np.allclose(p.cpu().numpy(), ref, rtol=1e-13, atol=0)
    assert abs(p.cpu().numpy()[2] - p_orc) <= 1e-13 * p_orc


def test_ams_run_invariants(L, orc):
    n, t_a, window, J = 8, 240, 40, 12
    e, cfg = make(L, n, 21, max_steps=t_a, ckpt_stride=30, n_snapshots=2)
    try:
        L.lbm_ensemble_set_snapshots(e, [0, 1])
        Q = zeros(n)
        it, lw, levels, kills, (rec_lw, rec_mx) = L.lbm_ams_run(e, t_a, window, J, float("inf"), 0.002, 13, Q,
                                                               with_kills=True, with_records=True)
        assert it == J
        # with the drag as score a killed trajectory's event maximum is its level
        assert np.array_equal(rec_mx, np.repeat(levels, kills))
        assert np.all(np.diff(levels) > 0)  # every kill removes the minimum: the level rises
        q = Q.cpu().numpy()
        assert np.all(q > levels[-1])
        # weight of the estimator: one factor (1 - |K_j|/N) per iteration; branched
        # copies of one survivor can share its maximum, so |K_j| >= 1
        assert np.all(kills >= 1) and np.all(kills < n)
        assert abs(lw - sum(np.log1p(-k / n) for k in kills)) < 1e-13
        d = np.zeros((n, t_a))
        L.lbm_ensemble_drag(e, 0, t_a, d)
        assert np.allclose(q, window_max(d, window, t_a), rtol=1e-11, atol=1e-14)
        assert list(L.lbm_ensemble_time(e, n)) == [t_a] * n
        p = zeros(2)
        lv = torch.tensor([levels[-1], q.max()], device="cuda")
        L.ams_probability(lw, Q, lv, p)
        ref = [orc.ams_probability(lw, q, a) for a in lv.cpu().numpy()]
        assert np.allclose(p.cpu().numpy(), ref, rtol=1e-14)
        # above the last killed level the killed records add nothing
        L.ams_probability(lw, Q, lv, p, records=(torch.tensor(rec_lw, device="cuda"),
                                                 torch.tensor(rec_mx, device="cuda")))
        assert np.allclose(p.cpu().numpy()[1:], ref[1:], rtol=1e-14)
        assert p.cpu().numpy()[0] > ref[0]  # at the last killed level its trajectories count
    finally:
        L.lbm_ensemble_destroy(e)


def test_ams_on_the_instantaneous_drag(L, orc):
    """AMS with the instantaneous drag as the score (window = 1: the trailing
    mean of one step is D(t) itself), the second AMS workload of the paper
    (Sec. 4.1): the levels rise, every final maximum is the maximum of the
    trajectory's drag series, the estimator weight is the product of the
    survival fractions, and the branched histories replay bitwise."""
    n, t_a, J = 8, 200, 10
    runs = []
    for _ in range(2):
        e, cfg = make(L, n, 31, max_steps=t_a, ckpt_stride=25, n_snapshots=2)
        try:
            L.lbm_ensemble_set_snapshots(e, [0, 1])
            Q = zeros(n)
            it, lw, levels, kills = L.lbm_ams_run(e, t_a, 1, J, float("inf"), 0.002, 17, Q, with_kills=True)
            d = np.zeros((n, t_a))
            L.lbm_ensemble_drag(e, 0, t_a, d)
            runs.append((it, lw, levels, kills, Q.cpu().numpy(), d))
        finally:
            L.lbm_ensemble_destroy(e)
    it, lw, levels, kills, q, d = runs[0]
    assert 1 <= it <= J and np.all(np.diff(levels) > 0)
    assert np.array_equal(q, d.max(axis=1))  # window 1: the score is D(t)
    assert np.all(q > levels[-1]) or np.all(q == q[0])
    assert abs(lw - sum(np.log1p(-k / n) for k in kills)) < 1e-13
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_ams_run_is_deterministic_and_stops_at_level(L):
    n, t_a, window = 6, 120, 20
    runs = []
    for _ in range(2):
        e, cfg = make(L, n, 4, max_steps=t_a, ckpt_stride=20, n_snapshots=1)
        try:
            L.lbm_ensemble_set_snapshots(e, [2])
            Q = zeros(n)
            it, lw, levels = L.lbm_ams_run(e, t_a, window, 8, float("inf"), 0.002, 3, Q)
            runs.append((it, lw, levels, Q.cpu().numpy(), pops(L, e, cfg, n)))
        finally:
            L.lbm_ensemble_destroy(e)
    assert runs[0][0] == runs[1][0] and runs[0][1] == runs[1][1]
    assert np.array_equal(runs[0][2], runs[1][2]) and np.array_equal(runs[0][3], runs[1][3])
    assert np.array_equal(runs[0][4], runs[1][4])
    # a level below every score stops before the first kill
    e, cfg = make(L, n, 4, max_steps=t_a, ckpt_stride=20)
    try:
        Q = zeros(n)
        it, lw, _ = L.lbm_ams_run(e, t_a, window, 8, -1e30, 0.0, 3, Q)
        assert it == 0 and lw == 0.0
    finally:
        L.lbm_ensemble_destroy(e)


def test_driver_argument_errors(L):
    e, cfg = make(L, 4, 1, max_steps=50)
    try:
        Q = zeros(4)
        with pytest.raises(L.LbmError):  # no checkpoints
            L.lbm_ams_run(e, 40, 10, 2, float("inf"), 0.0, 1, Q)
        with pytest.raises(L.LbmError):  # beyond max_steps
            L.lbm_gktl_run(e, 20, 3, 1.0, 0.0, 1, 0, zeros(3), zeros(12, torch.int32))
        with pytest.raises(L.LbmError):  # perturbation without a snapshot bank
            L.lbm_gktl_run(e, 10, 2, 1.0, 0.002, 1, 0, zeros(2), zeros(8, torch.int32))
    finally:
        L.lbm_ensemble_destroy(e)
