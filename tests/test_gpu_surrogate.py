"""The learned score inside the method, on the GPU: the checkpoint score
series, AMS with the learned score, GKTL with the learned potential, the
training data recorder, and what the trained network gains over the plain
drag-based score."""
import numpy as np
import pytest
import torch

from tests import seeded_inputs as si

pytestmark = pytest.mark.gpu

NX, NY, F = 128, 32, 4
KW = dict(nx=NX, ny=NY, obstacle=(28, 12, 8, 8), tau=0.6, gx=1e-5)


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


def ensemble(L, n, seed, **kw):
    cfg = L.config(**dict(KW, **kw))
    return L.lbm_ensemble_create(cfg, n, seed, torch.cuda.current_stream()), cfg


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



@pytest.fixture()
def model(L):
    m = L.cnn_create(NY // F, NX // F, 16, 3)
    yield m
    L.cnn_destroy(m)


def fields(L, e, clones):
    x = torch.zeros((len(clones), NY // F, NX // F, 8), dtype=torch.bfloat16, device="cuda")
    L.lbm_ensemble_fields(e, clones, F, 100.0, 50.0, x, NX, NY)
    return x


def test_checkpoint_scores_are_the_network_on_the_state(L, model):
    n, C = 5, 20
    e, cfg = ensemble(L, n, 1, max_steps=100, ckpt_stride=C)
    try:
        L.lbm_ensemble_attach_score(e, model, F, 100.0, 50.0)
        L.lbm_ensemble_step(e, 60)
        hist = L.lbm_ensemble_score_history(e, n, 100 // C + 1)
        assert np.all(np.isnan(hist[:, 0])) and np.all(np.isfinite(hist[:, 1:4])) and np.all(np.isnan(hist[:, 4:]))
        pred = torch.zeros(n, dtype=torch.float32, device="cuda")
        L.cnn_predict(model, fields(L, e, list(range(n))), pred)
        assert np.array_equal(hist[:, 3], pred.cpu().numpy().astype(np.float64))
        now = zeros(n)
        L.lbm_ensemble_evaluate_score(e, now)
        assert np.array_equal(now.cpu().numpy(), hist[:, 3])
        with pytest.raises(L.LbmError):  # input size must be the downsampled channel
            L.lbm_ensemble_attach_score(e, model, 2, 100.0, 50.0)
    finally:
        L.lbm_ensemble_destroy(e)


def test_ams_with_learned_score(L, model):
    """score_kind 1: the killed level rises, branches restore a checkpoint of the
    survivor exactly (shared score history up to the branch), the run is
    deterministic, and the event maxima are still taken on the drag."""
    n, C, t_a, J = 8, 20, 200, 10
    results = []
    for _ in range(2):
        e, cfg = ensemble(L, n, 9, max_steps=t_a, ckpt_stride=C, n_snapshots=2)
        try:
            L.lbm_ensemble_attach_score(e, model, F, 100.0, 50.0)
            L.lbm_ensemble_set_snapshots(e, [0, 1])
            Q = zeros(n)
            it, lw, levels, kills = L.lbm_ams_run(e, t_a, 40, J, float("inf"), 0.002, 5, Q, with_kills=True,
                                                   score_kind=1)
            hist = L.lbm_ensemble_score_history(e, n, t_a // C + 1)
            results.append((it, lw, levels, Q.cpu().numpy(), hist))
        finally:
            L.lbm_ensemble_destroy(e)
    it, lw, levels, q, hist = results[0]
    assert 1 <= it <= J and np.all(np.diff(levels) > 0)
    assert np.allclose(q, hist.max(axis=1), rtol=0, atol=0)
    assert np.all(q > levels[-1])
    if it < J:
        # every branch copies its survivor's score series up to the branch, so
        # the ensemble can collapse onto one maximum (the AMS failure mode the
        # paper reports for the drag score): then all scores tie and AMS stops
        assert np.all(q == q[0])
    assert abs(lw - sum(np.log1p(-k / n) for k in kills)) < 1e-13
    for a, b in zip(results[0], results[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_ams_with_learned_score_records_the_killed_trajectories(L, orc, model):
    """With the learned score the killed trajectories can hold the event
    (their drag maximum) though their score was the lowest, so the generalised
    AMS estimator counts them: the record of each trajectory killed at the last
    iteration J is the time-averaged drag maximum that a run stopped after J - 1
    iterations (deterministic) shows for the clones of minimum learned score"""
    n, C, t_a, J, window = 8, 20, 200, 6, 40
    out = {}
    for iters in (J, J - 1):
        e, cfg = ensemble(L, n, 9, max_steps=t_a, ckpt_stride=C, n_snapshots=2)
        try:
            L.lbm_ensemble_attach_score(e, model, F, 100.0, 50.0)
            L.lbm_ensemble_set_snapshots(e, [0, 1])
            Q = zeros(n)
            res = L.lbm_ams_run(e, t_a, window, iters, float("inf"), 0.002, 5, Q, with_kills=True, score_kind=1,
                                with_records=True)
            d = np.zeros((n, t_a))
            L.lbm_ensemble_drag(e, 0, t_a, d)
            out[iters] = (res, Q.cpu().numpy(), d)
        finally:
            L.lbm_ensemble_destroy(e)
    (it, lw, levels, kills, (rec_lw, rec_mx)), _, _ = out[J]
    assert it == J and len(rec_mx) == kills.sum()
    (it1, lw1, _, kills1, (rec_lw1, rec_mx1)), q_learned, drag = out[J - 1]
    assert np.array_equal(rec_mx[:len(rec_mx1)], rec_mx1) and np.array_equal(rec_lw[:len(rec_lw1)], rec_lw1)
    killed = np.nonzero(q_learned == q_learned.min())[0]
    assert len(killed) == kills[-1]
    ev = window_max(drag, window, t_a)
    assert np.allclose(rec_mx[len(rec_mx1):], ev[killed], rtol=1e-11, atol=1e-14)
    assert np.allclose(rec_lw[len(rec_lw1):], lw1, rtol=0, atol=1e-15)


def test_gktl_with_learned_potential(L, model):
    n, period, periods = 12, 20, 4
    # kappa = 0 with a score attached is the plain run, bit for bit
    outs = []
    for attach in (False, True):
        e, cfg = ensemble(L, n, 2, max_steps=100, n_snapshots=2)
        try:
            if attach:
                L.lbm_ensemble_attach_score(e, model, F, 100.0, 50.0)
            L.lbm_ensemble_set_snapshots(e, [0, 1])
            logR, parent = zeros(periods), zeros(periods * n, torch.int32)
            L.lbm_gktl_run(e, period, periods, 200.0, 0.002, 4, 0, logR, parent)
            outs.append((logR.cpu().numpy(), parent.cpu().numpy()))
        finally:
            L.lbm_ensemble_destroy(e)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    # kappa != 0: the correction is kappa (V(end) - V(start of the ancestor));
    # exact copies (eps = 0) so that the final states are the scored ones
    e, cfg = ensemble(L, n, 2, max_steps=100)
    try:
        L.lbm_ensemble_attach_score(e, model, F, 100.0, 50.0)
        v_start = zeros(n)
        L.lbm_ensemble_evaluate_score(e, v_start)
        logR, parent = zeros(periods), zeros(periods * n, torch.int32)
        corr = zeros(n)
        kappa = 0.7
        L.lbm_gktl_run(e, period, periods, 200.0, 0.0, 4, 0, logR, parent, kappa=kappa, correction_dev=corr)
        v_end = zeros(n)
        L.lbm_ensemble_evaluate_score(e, v_end)
        v0 = v_end.cpu().numpy() - corr.cpu().numpy() / kappa
        # trace each final slot back through the genealogy to its ancestor at t0
        par = parent.cpu().numpy().reshape(periods, n)
        anc = np.arange(n)
        for i in range(periods - 1, -1, -1):
            anc = par[i][anc]
        assert np.allclose(v0, v_start.cpu().numpy()[anc], rtol=1e-12, atol=1e-12)
        assert np.all(np.isfinite(logR.cpu().numpy()))
    finally:
        L.lbm_ensemble_destroy(e)


def test_gktl_with_learned_potential_matches_oracle(L, orc):
    """App. C.1 with the learned potential against an oracle composition of the
    same steps: the oracle runs every clone (FP64 LBM), scores each state with
    the FP64 network on its own block means (activations rounded to BF16 as the
    GPU stores them), adds kappa (V(t_i) - V(t_{i-1})) to k sum D, weights,
    resamples, and carries V(t_i) and the ancestor's V(0) along the
    genealogy.  Seeded network parameters on both sides; eps = 0.  The
    parents agree exactly, log R and the correction kappa (V(T_a) - V(0)) to
    the network's BF16 precision."""
    from oracle import cnn

    def bf16_round(a):
        return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)

    n, period, periods, k, kappa, sel_seed, seed = 6, 20, 3, 200.0, 0.7, 4, 2
    m = L.cnn_create(NY // F, NX // F, 16, 3)
    p = si.cnn_params(31)
    L.cnn_set_params(m, p)
    pq = p.astype(np.float64)
    off, _ = cnn.offsets()
    pq[:off[4]] = bf16_round(pq[:off[4]])  # the GPU multiplies BF16 copies of the conv weights
    e, cfg = ensemble(L, n, seed, max_steps=period * periods)
    try:
        L.lbm_ensemble_attach_score(e, m, F, 100.0, 50.0)
        logR, parent, corr = zeros(periods), zeros(periods * n, torch.int32), zeros(n)
        L.lbm_gktl_run(e, period, periods, k, 0.0, sel_seed, 0, logR, parent, kappa=kappa, correction_dev=corr)
        got_logR, got_parent, got_corr = logR.cpu().numpy(), parent.cpu().numpy().reshape(periods, n), corr.cpu().numpy()
    finally:
        L.lbm_ensemble_destroy(e)
        L.cnn_destroy(m)
    oc = orc.cfg(NX, NY, obstacle=KW["obstacle"], tau=KW["tau"], gx=KW["gx"])

    def V(f):
        x = bf16_round(cnn.fields(oc, f, F, 100.0, 50.0))[None]
        return float(cnn.forward(pq, x, store=bf16_round)[0][0])
    f = [orc.init(oc, seed, c, 0.01) for c in range(n)]
    v0 = np.array([V(fc) for fc in f])
    vprev = v0.copy()
    ref_logR, ref_parent, v_scale = [], [], np.abs(v0).max()
    for i in range(periods):
        runs = [orc.run(oc, fc, period) for fc in f]
        f = [r[0] for r in runs]
        vnow = np.array([V(fc) for fc in f])
        v_scale = max(v_scale, np.abs(vnow).max())
        s_ = np.array([k * r[1].sum() for r in runs]) + kappa * (vnow - vprev)
        W, lr = orc.gktl_weights(s_)
        par = orc.gktl_select(W, sel_seed, i)
        ref_logR.append(lr)
        ref_parent.append(par)
        f = [f[q].copy() for q in par]
        v0, vprev = v0[par], vnow[par]
    ref_corr = kappa * (vprev - v0)
    assert np.array_equal(got_parent, np.array(ref_parent))
    assert (got_parent != np.arange(n)).any()  # the selection cloned
    tol = 2e-2 * kappa * v_scale  # the network's BF16 precision, carried into s
    assert np.abs(got_logR - np.array(ref_logR)).max() <= tol
    assert np.abs(got_corr - ref_corr).max() <= tol


def test_dataset_labels_are_future_drag_means(L):
    n, n_snaps, every, horizon = 6, 4, 15, 25
    e, cfg = ensemble(L, n, 3, max_steps=200)
    try:
        L.lbm_ensemble_step(e, 10)
        first = fields(L, e, list(range(n)))
        x = torch.zeros((n_snaps * n, NY // F, NX // F, 8), dtype=torch.bfloat16, device="cuda")
        y = torch.zeros(n_snaps * n, dtype=torch.float32, device="cuda")
        mu, sd = L.lbm_surrogate_dataset(e, n_snaps, every, horizon, F, 100.0, 50.0, x, y, n, NX, NY)
        assert torch.equal(x[:n], first)
        d = np.zeros((n, 10 + (n_snaps - 1) * every + horizon))
        L.lbm_ensemble_drag(e, 0, d.shape[1], d)
        want = np.array([[d[c, 10 + i * every:10 + i * every + horizon].mean() for c in range(n)]
                         for i in range(n_snaps)]).ravel()
        got = y.cpu().numpy().astype(np.float64) * sd + mu
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
        assert abs(y.mean().item()) < 1e-5 and abs(y.std(unbiased=False).item() - 1) < 1e-4
    finally:
        L.lbm_ensemble_destroy(e)


def test_trained_score_beats_the_drag_score(L):
    """What the network gains: trained on ensemble trajectories, it predicts the
    time-averaged drag over the next 100 steps from the flow fields better (R^2
    on held-out clones) than the plain drag-based score, the time-averaged drag
    over the last 100 steps."""
    n, n_snaps, every, horizon, t0 = 64, 24, 25, 100, 100
    e, cfg = ensemble(L, n, 11, max_steps=t0 + (n_snaps - 1) * every + horizon, init_amp=0.02)
    m = L.cnn_create(NY // F, NX // F, 32, 5)
    try:
        L.lbm_ensemble_step(e, t0)
        x = torch.zeros((n_snaps * n, NY // F, NX // F, 8), dtype=torch.bfloat16, device="cuda")
        y = torch.zeros(n_snaps * n, dtype=torch.float32, device="cuda")
        mu, sd = L.lbm_surrogate_dataset(e, n_snaps, every, horizon, F, 100.0, 50.0, x, y, n, NX, NY)
        d = np.zeros((n, cfg.max_steps))
        L.lbm_ensemble_drag(e, 0, cfg.max_steps, d)
        clone = np.tile(np.arange(n), n_snaps)
        snap = np.repeat(np.arange(n_snaps), n)
        train = clone < 48
        xt, yt = x[torch.tensor(train)].contiguous(), y[torch.tensor(train)].contiguous()
        losses = L.cnn_fit(m, xt, yt, 32, 30, 2e-3, 7)
        assert losses[-1] < 0.5 * losses[0]
        pred = torch.zeros(len(y), dtype=torch.float32, device="cuda")
        L.cnn_predict(m, x, pred)
        test = ~train
        yv = y.cpu().numpy()[test]
        pv = pred.cpu().numpy()[test]
        # drag score: trailing mean of the past horizon, normalised like the labels
        past = np.array([d[c, t0 + s * every - horizon:t0 + s * every].mean() for c, s in zip(clone, snap)])
        base = ((past - mu) / sd)[test]
        a, b = np.polyfit(base, yv, 1)  # best affine use of the drag score

        def r2(p):
            return 1 - np.mean((yv - p) ** 2) / np.var(yv)
        print(f"R^2 network {r2(pv):.3f}, drag score {r2(a * base + b):.3f}")
        assert r2(pv) > r2(a * base + b)
    finally:
        L.cnn_destroy(m)
        L.lbm_ensemble_destroy(e)
