"""Direct-sampling statistics on the GPU (Sec. 3) against the oracle on the
same drag series (a seeded synthetic series written into the ensemble's
history, so that both sides read one input): the pooled autocorrelation and
correlation time (FP64 sums in another order: 1e-10 relative) and the
waiting-time return times (event counts are integers: exact)."""
import numpy as np
import pytest
import torch

from tests import seeded_inputs as si

pytestmark = pytest.mark.gpu

KW = dict(nx=200, ny=37, obstacle=(50, 14, 9, 7), tau=0.53, gx=3e-5, max_steps=900, init_amp=0.05)


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


@pytest.fixture(scope="module")
def run(L):
    n, steps = 6, 900
    cfg = L.config(**KW)
    e = L.lbm_ensemble_create(cfg, n, 4, torch.cuda.current_stream())
    L.lbm_ensemble_step(e, steps)
    d = si.drag_series(n, steps, 4, rho=0.95)
    L.lbm_ensemble_set_drag(e, 0, steps, d)
    back = np.zeros((n, steps))
    L.lbm_ensemble_drag(e, 0, steps, back)
    assert np.array_equal(back, d)
    yield e, d
    L.lbm_ensemble_destroy(e)


def test_autocorrelation_matches_oracle(L, orc, run):
    e, d = run
    t0, t1, lag = 300, 900, 250
    c = torch.zeros(lag + 1, dtype=torch.float64, device="cuda")
    tc = L.lbm_drag_autocorrelation(e, t0, t1, lag, c)
    ref, ref_tc = orc.autocorrelation(d[:, t0:t1], lag)
    got = c.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)
    assert tc == ref_tc or abs(ref[ref_tc]) < 1e-10


@pytest.mark.parametrize("gap", [0, 7])
def test_return_times_match_oracle(L, orc, run, gap):
    e, d = run
    t0, t1 = 300, 900
    x = d[:, t0:t1]
    levels = np.quantile(x, [0.5, 0.8, 0.95, 0.999]).tolist() + [x.max() + 1.0]
    ev, r = L.lbm_drag_return_times(e, t0, t1, torch.tensor(levels, dtype=torch.float64, device="cuda"), gap)
    ref_ev, ref_r = orc.return_times(x, levels, gap)
    assert np.array_equal(ev, ref_ev)
    assert np.array_equal(np.isinf(r), np.isinf(ref_r))
    assert np.allclose(r[np.isfinite(r)], ref_r[np.isfinite(ref_r)], rtol=1e-15)


def test_statistics_argument_errors(L, run):
    e, _ = run
    c = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LbmError):  # beyond the steps the clones have taken
        L.lbm_drag_autocorrelation(e, 0, 901, 5, c)
    with pytest.raises(L.LbmError):  # lag as long as the window
        L.lbm_drag_autocorrelation(e, 100, 105, 5, c)
    with pytest.raises(L.LbmError):
        L.lbm_drag_return_times(e, 0, 100, torch.zeros(2, dtype=torch.float64, device="cuda"), -1)
