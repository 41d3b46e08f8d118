"""GPU open channel (Sec. 2: parabolic equilibrium inlet, entrance grid of bars,
sponge, regularized outlet at unit density) against the FP64 oracle through
the C ABI: a ragged channel (nx not a multiple of 8) with square, grid and
sponge under both collisions, every open-channel step variant (each against
the oracle and all bitwise alike), 16-bit storage, graph replay, the App. D
perturbation with the grid's solid cells, the paper's 513 x 129 geometry, and
argument checks.  Tolerances as for the periodic channel: populations 1e-5
and drag 1e-4 relative (FP32 arithmetic against FP64)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

POP_TOL, DRAG_TOL = 1e-5, 1e-4
RATES = dict(omega_bulk=1.3, omega_3=0.9, omega_4=1.7)
# ragged: nx = 203; square at x 80..88; grid bars of 3 rows every 7 at x 12..15;
# sponge over the last 30 columns up to tau 0.95
OPEN = dict(nx=203, ny=37, obstacle=(80, 14, 9, 7), tau=0.56, open_x=1, u_in=0.05, grid=(12, 4, 3, 4),
            sponge_len=30, sponge_tau=0.95, max_steps=400, init_amp=0.01)
# the channel of Sec. 2: 513 x 129, R = 16 at the centre, bars of R/2 every R
# from x = R, R/2 thick; Re_grid = 1200 on u_c = 0.05 and R/2; sponge of 8R
PAPER = dict(nx=513, ny=129, obstacle=(248, 56, 16, 16), tau=0.5 + 3 * 0.05 * 8 / 1200, open_x=1, u_in=0.05,
             grid=(16, 8, 8, 8), sponge_len=128, sponge_tau=1.0, collision="cm", max_steps=200, init_amp=0.0)


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

    def drag(self, t0, t1):
        d = np.zeros((self.n, t1 - t0))
        self.L.lbm_ensemble_drag(self.h, t0, t1, d)
        return d


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel_pop(a, b):
    """largest relative error of any single population (the populations are
    positive): |f_gpu - f_oracle| <= tol |f_oracle| element by element"""
    return (np.abs(a - b) / np.abs(b)).max()


def ocfg(orc, kw):
    coll = kw.get("collision", "bgk")
    rates = {k: kw[k] for k in ("omega_bulk", "omega_3", "omega_4") if k in kw}
    return orc.cfg(kw["nx"], kw["ny"], obstacle=kw.get("obstacle", (0, 0, 0, 0)), tau=kw["tau"],
                   collision=1 if coll == "cm" else 0, open_x=1, u_in=kw["u_in"], grid=kw.get("grid", (0, 0, 0, 0)),
                   sponge_len=kw.get("sponge_len", 0), sponge_tau=kw.get("sponge_tau", 1.0), **rates)


def open_variants(L, storage):
    """indices of the step variants with an open-channel instantiation"""
    out = []
    for v in range(L.lbm_step_variant_count()):
        st, vec, warps = L.lbm_step_variant_info(v)
        if st != L.STORAGE[storage] or L.lbm_step_variant_kind(v) != 0:
            continue
        with Ens(L, 1, **dict(OPEN, storage=storage, max_steps=2)) as e:
            try:
                L.lbm_ensemble_set_variant(e.h, v)
            except L.LbmError:
                continue
        out.append(v)
    return out


@pytest.mark.parametrize("coll", ["bgk", "cm"])
def test_open_channel_matches_oracle(L, orc, coll):
    kw = dict(OPEN, collision=coll, **(RATES if coll == "cm" else {}))
    oc = ocfg(orc, kw)
    with Ens(L, 2, seed=4, **kw) as e:
        for c in range(2):
            assert np.abs(e.pops(c) - orc.init(oc, 4, c, 0.01)).max() < 1e-7
        L.lbm_ensemble_step(e.h, 200)
        d = e.drag(0, 200)
        for c in range(2):
            f_ref, d_ref = orc.run(oc, orc.init(oc, 4, c, 0.01), 200)
            assert rel_pop(e.pops(c), f_ref) < POP_TOL, c
            assert rel(d[c], d_ref) < DRAG_TOL, c


def test_every_open_variant_matches_oracle_and_each_other(L, orc):
    kw = dict(OPEN, max_steps=80)
    oc = ocfg(orc, kw)
    ref = [orc.run(oc, orc.init(oc, 9, c, 0.01), 60) for c in range(2)]
    vs = open_variants(L, "fp32")
    assert len(vs) >= 3
    first = None
    for v in vs:
        with Ens(L, 2, seed=9, **kw) as e:
            L.lbm_ensemble_set_variant(e.h, v)
            L.lbm_ensemble_step(e.h, 60)
            got = [e.pops(c) for c in range(2)]
            d = e.drag(0, 60)
        for c in range(2):
            assert rel_pop(got[c], ref[c][0]) < POP_TOL, (v, c)
            assert rel(d[c], ref[c][1]) < DRAG_TOL, (v, c)
        if first is None:
            first = got
        else:
            for a, b in zip(got, first):
                assert np.array_equal(a, b), v


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_open_channel_16bit_storage(L, orc, storage):
    """shifted 16-bit storage against FP64: the stored g = f - w carries 11
    (FP16) or 8 (BF16) significant bits, so the error is bounded relative to
    the largest |g| (3e-3 and 2e-2 over 200 steps, as for the periodic
    channel), and every 16-bit variant agrees bitwise"""
    kw = dict(OPEN, storage=storage, shift_exp=4 if storage == "fp16" else 0)
    oc = ocfg(orc, kw)
    f_ref, d_ref = orc.run(oc, orc.init(oc, 2, 0, 0.01), 200)
    g_ref = f_ref - orc.feq(1.0, 0.0, 0.0)[:, None, None]
    tol = 3e-3 if storage == "fp16" else 2e-2
    first = None
    for v in open_variants(L, storage):
        with Ens(L, 1, seed=2, **kw) as e:
            L.lbm_ensemble_set_variant(e.h, v)
            L.lbm_ensemble_step(e.h, 200)
            f = e.pops(0)
            assert np.all(np.isfinite(e.drag(0, 200)))
        assert np.abs(f - f_ref).max() / np.abs(g_ref).max() < tol, v
        if first is None:
            first = f
        else:
            assert np.array_equal(f, first), v


def test_open_graph_replay_equals_launches(L):
    kw = dict(OPEN, max_steps=120)
    with Ens(L, 2, seed=1, **kw) as a, Ens(L, 2, seed=1, **kw) as b:
        L.lbm_ensemble_set_graphs(b.h, 0)
        for _ in range(3):  # repeated chunks replay the cached graph
            L.lbm_ensemble_step(a.h, 33)
            L.lbm_ensemble_step(b.h, 33)
        for c in range(2):
            assert np.array_equal(a.pops(c), b.pops(c))
        assert np.array_equal(a.drag(0, 99), b.drag(0, 99))


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_open_state_does_not_depend_on_the_chunking(L, storage):
    """Within a chunk of steps the outlet column is not stored: each step pulls
    the outlet computed from the previous step's velocities, and the column is
    written after the chunk's last step.  So 150 steps in one call, in 150
    calls of one step, and in calls of 7, 50 and 93 steps give the same
    populations (the outlet column included) and drag, bit for bit"""
    kw = dict(OPEN, max_steps=150, storage=storage, collision="cm")
    with Ens(L, 2, seed=5, **kw) as a, Ens(L, 2, seed=5, **kw) as b, Ens(L, 2, seed=5, **kw) as c:
        L.lbm_ensemble_step(a.h, 150)
        for _ in range(150):
            L.lbm_ensemble_step(b.h, 1)
        for k in (7, 50, 93):
            L.lbm_ensemble_step(c.h, k)
        for i in range(2):
            fa = a.pops(i)
            assert np.array_equal(fa, b.pops(i)) and np.array_equal(fa, c.pops(i))
            assert np.isfinite(fa).all()
        assert np.array_equal(a.drag(0, 150), b.drag(0, 150)) and np.array_equal(a.drag(0, 150), c.drag(0, 150))


def test_open_single_clone_steps_match_ensemble(L):
    """the small-list variant (one clone: an AMS branch) gives the same states"""
    kw = dict(OPEN, max_steps=60)
    with Ens(L, 3, seed=6, **kw) as a, Ens(L, 3, seed=6, **kw) as b:
        L.lbm_ensemble_step(a.h, 40)
        for c in range(3):
            L.lbm_ensemble_step_clones(b.h, 40, [c])
        for c in range(3):
            assert np.array_equal(a.pops(c), b.pops(c))


def test_open_perturbation_keeps_grid_at_rest(L, orc):
    """App. D on an open channel: the grid's cells are solid, left at rest,
    and outside the fluid mass that the perturbation preserves"""
    kw = dict(OPEN, n_snapshots=2, max_steps=100)
    oc = ocfg(orc, kw)
    solid = orc.solid_mask(oc)
    assert solid[:, 12:16].any()
    n = 4
    with Ens(L, n, seed=3, **kw) as e:
        L.lbm_ensemble_step(e.h, 30)
        L.lbm_ensemble_set_snapshots(e.h, [1, 2])
        before = [e.pops(c) for c in range(n)]
        parent = torch.tensor([0, 0, 2, 2], dtype=torch.int32, device="cuda")
        L.lbm_ensemble_clone(e.h, parent, 1e-3, 77, 1)
        after = [e.pops(c) for c in range(n)]
        w = orc.feq(1.0, 0.0, 0.0)
        for c in range(n):
            assert np.abs(after[c][:, solid] - w[:, None]).max() < 1e-7
        mass0 = before[0][:, ~solid].sum()
        assert abs(after[1][:, ~solid].sum() - mass0) < 1e-9 * mass0 * 100
        assert np.abs(after[1] - before[0]).max() > 1e-6  # perturbed


def test_paper_channel_matches_oracle(L, orc):
    """513 x 129 with the square, the grid of bars and the sponge, central
    moments at tau = 0.501, 100 steps from rest on the inlet profile"""
    oc = ocfg(orc, PAPER)
    f_ref, d_ref = orc.run(oc, orc.init(oc, 0, 0, 0.0), 100)
    with Ens(L, 1, seed=0, **PAPER) as e:
        L.lbm_ensemble_step(e.h, 100)
        assert rel_pop(e.pops(0), f_ref) < POP_TOL
        assert rel(e.drag(0, 100)[0], d_ref) < DRAG_TOL


def test_open_argument_errors(L):
    bad = [dict(gx=1e-5), dict(sponge_tau=1.2), dict(sponge_len=0, tau=1.1), dict(grid=(0, 4, 3, 4)),
           dict(grid=(190, 12, 3, 4)), dict(obstacle=(196, 14, 5, 5)), dict(open_x=2), dict(u_in=0.4),
           dict(ny=2, obstacle=(0, 0, 0, 0), grid=(0, 0, 0, 0)), dict(grid=(12, 4, 0, 4))]
    for b in bad:
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_create(L.config(**dict(OPEN, **b)), 1, 0, torch.cuda.current_stream())
    periodic = dict(nx=64, ny=16, tau=0.6, max_steps=4)
    for b in (dict(grid=(4, 2, 2, 2)), dict(sponge_len=8)):
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_create(L.config(**periodic, **b), 1, 0, torch.cuda.current_stream())
    with pytest.raises(L.LbmError):  # nx = 203 is only valid for an open channel
        L.lbm_ensemble_create(L.config(**dict(OPEN, open_x=0, grid=(0, 0, 0, 0), sponge_len=0)), 1, 0,
                              torch.cuda.current_stream())
    with Ens(L, 1, **dict(OPEN, max_steps=4)) as e:  # row-staged variants have no open instantiation
        for v in range(L.lbm_step_variant_count()):
            if L.lbm_step_variant_kind(v) == 1 and L.lbm_step_variant_info(v)[0] == 0:
                with pytest.raises(L.LbmError):
                    L.lbm_ensemble_set_variant(e.h, v)
    n, nx, ny = 1, 208, 37
    cfg = L.config(**dict(OPEN, nx=nx))
    pitch = L.noalloc_pitch(nx)
    a = torch.zeros((n, 9, ny, pitch), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LbmError):
        L.lbm_step_noalloc(cfg, n, a, torch.zeros_like(a), torch.zeros(n, dtype=torch.float64, device="cuda"),
                           torch.cuda.current_stream())


def test_open_branch_replays_bitwise(L):
    """AMS branching on the open channel: with eps = 0 the branch is the source
    trajectory bit for bit (state, drag and the square's observables); with a
    perturbation it departs from the source after t_b"""
    kw = dict(OPEN, collision="cm", max_steps=160, ckpt_stride=25, n_snapshots=2)
    with Ens(L, 3, seed=6, **kw) as e:
        L.lbm_ensemble_set_observables(e.h, True)
        L.lbm_ensemble_step(e.h, 120)
        L.lbm_ensemble_branch(e.h, 1, 2, 87, 0.0, 3, 1)
        assert list(L.lbm_ensemble_time(e.h, 3)) == [120, 87, 120]
        L.lbm_ensemble_step_clones(e.h, 33, [1])
        assert np.array_equal(e.pops(1), e.pops(2))
        d = e.drag(0, 120)
        assert np.array_equal(d[1], d[2])
        o = np.zeros((3, 120, 4))
        L.lbm_ensemble_observables(e.h, 0, 120, o)
        assert np.array_equal(o[1], o[2])
        L.lbm_ensemble_set_snapshots(e.h, [0, 2])
        L.lbm_ensemble_branch(e.h, 1, 2, 50, 0.002, 3, 2)
        L.lbm_ensemble_step_clones(e.h, 70, [1])
        d = e.drag(0, 120)
        assert np.array_equal(d[1, :50], d[2, :50])
        assert not np.array_equal(d[1, 50:], d[2, 50:])


def test_open_gktl_and_ams_runs_are_deterministic(L):
    """the GKTL and AMS drivers on the open channel: finite estimator weights,
    rising AMS levels, and two runs from the same seeds agree bit for bit"""
    n, t_a = 8, 200
    kw = dict(OPEN, collision="cm", max_steps=t_a, ckpt_stride=25, n_snapshots=2)
    results = []
    for _ in range(2):
        with Ens(L, n, seed=11, **kw) as e:
            L.lbm_ensemble_set_snapshots(e.h, [0, 1])
            logR = torch.zeros(4, dtype=torch.float64, device="cuda")
            parent = torch.zeros((4, n), dtype=torch.int32, device="cuda")
            L.lbm_gktl_run(e.h, 25, 4, 5.0, 0.002, 9, 0, logR, parent)
            g = (logR.cpu().numpy(), parent.cpu().numpy(), e.drag(0, 100))
        with Ens(L, n, seed=12, **kw) as e:
            L.lbm_ensemble_set_snapshots(e.h, [0, 1])
            Q = torch.zeros(n, dtype=torch.float64, device="cuda")
            it, lw, levels = L.lbm_ams_run(e.h, t_a, 20, 6, float("inf"), 0.002, 13, Q)
            a = (it, lw, np.asarray(levels), Q.cpu().numpy())
        results.append((g, a))
    (g0, a0), (g1, a1) = results
    assert np.all(np.isfinite(g0[0])) and np.all((g0[1] >= 0) & (g0[1] < n))
    assert a0[0] == 6 and np.isfinite(a0[1]) and np.all(np.diff(a0[2]) > 0)
    for x, y in zip(g0, g1):
        assert np.array_equal(x, y)
    assert a0[0] == a1[0] and a0[1] == a1[1]
    assert np.array_equal(a0[2], a1[2]) and np.array_equal(a0[3], a1[3])
