"""GPU observables of the square (forebody and base pressures of eq.
drag_approx, mean wall shears of eq. avg_shear_def) and the in-place App. D
perturbation, against the FP64 oracle through the C ABI.  The observables of
every step are compared with the oracle's on its own states: pressures 1e-6
relative (sums of FP32 densities), shears 1e-3 of their largest magnitude
(the wall stencil amplifies the FP32 velocity error ninefold)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

RAGGED = dict(nx=200, ny=37, obstacle=(50, 14, 9, 7), tau=0.6, gx=2e-5, gy=-5e-6, max_steps=200, init_amp=0.02)
OPEN = dict(nx=203, ny=37, obstacle=(80, 14, 9, 7), tau=0.56, open_x=1, u_in=0.05, grid=(12, 4, 3, 4),
            sponge_len=30, sponge_tau=0.95, max_steps=200, init_amp=0.01, collision="cm")


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


class Ens:
    def __init__(self, L, n, seed=0, **kw):
        self.L, self.n = L, n
        self.cfg = L.config(**kw)
        self.h = L.lbm_ensemble_create(self.cfg, n, seed, torch.cuda.current_stream())

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.L.lbm_ensemble_destroy(self.h)

    def pops(self, c):
        return self.L.lbm_ensemble_get_populations(self.h, c, self.cfg.nx, self.cfg.ny)

    def obs(self, t0, t1):
        o = np.zeros((self.n, t1 - t0, 4))
        self.L.lbm_ensemble_observables(self.h, t0, t1, o)
        return o

    def drag(self, t0, t1):
        d = np.zeros((self.n, t1 - t0))
        self.L.lbm_ensemble_drag(self.h, t0, t1, d)
        return d


def ocfg(orc, kw):
    extra = {}
    if kw.get("open_x"):
        extra = dict(open_x=1, u_in=kw["u_in"], grid=kw["grid"], sponge_len=kw["sponge_len"],
                     sponge_tau=kw["sponge_tau"], collision=1 if kw.get("collision") == "cm" else 0)
    return orc.cfg(kw["nx"], kw["ny"], obstacle=kw["obstacle"], tau=kw["tau"], gx=kw.get("gx", 0.0),
                   gy=kw.get("gy", 0.0), **extra)


def oracle_series(orc, oc, seed, clone, amp, n):
    f = orc.init(oc, seed, clone, amp)
    out = []
    for _ in range(n):
        f, _, _ = orc.step(oc, f)
        out.append(orc.observables(oc, f))
    return np.array(out)


def check_series(got, ref):
    for k in (0, 1):
        assert np.abs(got[:, k] - ref[:, k]).max() < 1e-6 * np.abs(ref[:, k]).max(), k
    for k in (2, 3):
        assert np.abs(got[:, k] - ref[:, k]).max() < 1e-3 * np.abs(ref[:, k]).max(), k


@pytest.mark.parametrize("kw", [RAGGED, OPEN], ids=["periodic_forced", "open_cm"])
def test_observables_match_oracle(L, orc, kw):
    n_steps = 80
    oc = ocfg(orc, kw)
    with Ens(L, 2, seed=4, **kw) as e:
        L.lbm_ensemble_set_observables(e.h, True)
        L.lbm_ensemble_step(e.h, n_steps)
        got = e.obs(0, n_steps)
    for c in range(2):
        check_series(got[c], oracle_series(orc, oc, 4, c, kw["init_amp"], n_steps))


def test_observables_graphs_and_launches_agree_and_start_when_enabled(L):
    with Ens(L, 2, seed=1, **RAGGED) as a, Ens(L, 2, seed=1, **RAGGED) as b:
        L.lbm_ensemble_set_graphs(b.h, 0)
        for e in (a, b):
            L.lbm_ensemble_step(e.h, 10)  # not recorded
            L.lbm_ensemble_set_observables(e.h, True)
            L.lbm_ensemble_step(e.h, 30)
            L.lbm_ensemble_step(e.h, 30)
        oa, ob = a.obs(0, 70), b.obs(0, 70)
        assert np.array_equal(oa, ob)
        assert np.all(oa[:, :10] == 0.0) and np.all(oa[:, 10:, 0] > 0.0)
        # each face pressure is cs2 times the face's 7 rows of near-unit density
        assert np.abs(oa[:, 10:, :2] / (7 / 3) - 1).max() < 0.05


def test_observables_follow_clones(L):
    kw = dict(RAGGED, n_snapshots=2)
    with Ens(L, 3, seed=2, **kw) as e:
        L.lbm_ensemble_set_observables(e.h, True)
        L.lbm_ensemble_step(e.h, 25)
        before = e.obs(0, 25)
        L.lbm_ensemble_clone(e.h, torch.tensor([0, 0, 2], dtype=torch.int32, device="cuda"), 0.0, 1, 0)
        after = e.obs(0, 25)
        assert np.array_equal(after[1], before[0]) and np.array_equal(after[2], before[2])


def test_observables_errors(L):
    with Ens(L, 1, **dict(RAGGED, obstacle=(50, 1, 9, 7))) as e:  # one fluid row below the square
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_set_observables(e.h, True)
        with pytest.raises(L.LbmError):  # never enabled
            e.obs(0, 1)


@pytest.mark.parametrize("kw", [RAGGED, OPEN], ids=["periodic", "open"])
def test_perturb_in_place_matches_oracle(L, orc, kw):
    kw = dict(kw, n_snapshots=3)
    oc = ocfg(orc, kw)
    n = 4
    with Ens(L, n, seed=7, **kw) as e:
        L.lbm_ensemble_step(e.h, 20)
        L.lbm_ensemble_set_snapshots(e.h, [3, 0, 2])
        before = [e.pops(c) for c in range(n)]
        at20 = [orc.run(oc, orc.init(oc, 7, c, kw["init_amp"]), 20)[0] for c in range(n)]  # the oracle's own states
        snaps = np.stack([at20[3], at20[0], at20[2]])
        L.lbm_ensemble_perturb(e.h, [1, 3], 0.002, 99, 4)
        for c in (0, 2):
            assert np.array_equal(e.pops(c), before[c])
        for c in (1, 3):
            ref = orc.perturb(oc, at20[c], snaps, orc.perturb_alphas(99, 4, c, 3), 0.002)
            got = e.pops(c)
            assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-6
            assert np.abs(got - before[c]).max() > 1e-6
            m_ref, _, _ = orc.moments(oc, at20[c])
            m_got, _, _ = orc.moments(oc, got)
            assert abs(m_got - m_ref) / m_ref < 1e-6
        L.lbm_ensemble_perturb(e.h, [0], 0.0, 1, 1)  # eps = 0: nothing
        assert np.array_equal(e.pops(0), before[0])
        for bad in ([4], [1, 1], [-1]):
            with pytest.raises(L.LbmError):
                L.lbm_ensemble_perturb(e.h, bad, 0.002, 1, 1)
