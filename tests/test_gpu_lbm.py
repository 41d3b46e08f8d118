"""GPU parity of the fused lattice-Boltzmann step, drag, reductions, cloning
and branching against the FP64 oracle, through the C ABI.

Tolerances (FP32 arithmetic and storage): populations 1e-5 relative to their
largest value, drag series 1e-4 relative to its largest magnitude over the
first 200 steps.  Reduced-precision storage is compared against FP64 with
bounds derived from the 16-bit format (see each test)."""
import numpy as np
import pytest
import torch

from tests import seeded_inputs as si

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
DRAG_TOL = 1e-4


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    assert torch.cuda.is_available()
    return lbmrare


class Ens:
    """create/destroy around the C handle"""

    def __init__(self, L, n, seed=0, **kw):
        self.L = L
        self.kw = kw
        self.n = n
        self.cfg = L.config(**kw)
        self.stream = torch.cuda.current_stream()
        self.h = L.lbm_ensemble_create(self.cfg, n, seed, self.stream)

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


def oracle_cfg(orc, kw):
    return orc.cfg(kw["nx"], kw["ny"], obstacle=kw.get("obstacle", (0, 0, 0, 0)), tau=kw.get("tau", 0.6),
                   gx=kw.get("gx", 0.0), gy=kw.get("gy", 0.0))


CFG1 = dict(nx=256, ny=64, obstacle=si.channel(256, 64, 8, 64), tau=0.52, gx=1e-6, max_steps=2000)
RAGGED = dict(nx=200, ny=37, obstacle=(50, 14, 9, 7), tau=0.6, gx=2e-5, gy=-5e-6, max_steps=400)


def test_init_matches_oracle(L, orc):
    with Ens(L, 3, seed=5, **RAGGED, init_amp=0.02) as e:
        oc = oracle_cfg(orc, RAGGED)
        for c in range(3):
            ref = orc.init(oc, 5, c, 0.02)
            assert np.abs(e.pops(c) - ref).max() < 1e-7


@pytest.mark.parametrize("seed", [0, 1])
def test_cfg1_200_steps_match_oracle(L, orc, seed):
    """256 x 64 channel, 8 x 8 obstacle at (64, 32), tau 0.52, g 1e-6: FP32
    populations and drag over 200 steps against FP64."""
    with Ens(L, 1, seed=seed, **CFG1) as e:
        L.lbm_ensemble_step(e.h, 200)
        oc = oracle_cfg(orc, CFG1)
        f_ref, d_ref = orc.run(oc, orc.init(oc, seed, 0, 0.01), 200)
        assert rel_pop(e.pops(0), f_ref) < POP_TOL
        assert rel(e.drag(0, 200)[0], d_ref) < DRAG_TOL


def test_every_variant_on_ragged_grid(L, orc):
    """nx = 200 (not a multiple of the warp width in sites), ny = 37, obstacle
    away from the centre, force with both components: every compiled FP32
    variant against the oracle over 60 steps, several clones."""
    oc = oracle_cfg(orc, RAGGED)
    refs = [orc.run(oc, orc.init(oc, 9, c, 0.01), 60) for c in range(3)]
    n_var = L.lbm_step_variant_count()
    tried = 0
    for v in range(n_var):
        st, vec, warps = L.lbm_step_variant_info(v)
        if st != 0:
            continue
        with Ens(L, 3, seed=9, **RAGGED) as e:
            L.lbm_ensemble_set_variant(e.h, v)
            L.lbm_ensemble_step(e.h, 60)
            d = e.drag(0, 60)
            for c in range(3):
                assert rel_pop(e.pops(c), refs[c][0]) < POP_TOL, (vec, warps, c)
                assert rel(d[c], refs[c][1]) < DRAG_TOL, (vec, warps, c)
        tried += 1
    assert tried >= 3


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_every_variant_agrees_bitwise(L, storage):
    """All compiled variants of one storage format (register-staged row
    segments of every width, bulk-copy-staged whole rows) compute the same
    populations bit for bit (one collision routine, the same loads); the drag
    differs only by the grouping of its partial sums.  Small step calls (an AMS
    branch) may run another variant than the ensemble, so this is what makes a
    branch replay the source's path exactly."""
    kw = dict(RAGGED, max_steps=50, storage=storage)
    ref = None
    n_var = L.lbm_step_variant_count()
    for v in range(n_var):
        st, vec, warps = L.lbm_step_variant_info(v)
        if st != L.STORAGE[storage]:
            continue
        with Ens(L, 3, seed=9, **kw) as e:
            L.lbm_ensemble_set_variant(e.h, v)
            L.lbm_ensemble_step(e.h, 30)
            got = ([e.pops(c) for c in range(3)], e.drag(0, 30))
        if ref is None:
            ref = got
            continue
        for a, b in zip(got[0], ref[0]):
            assert np.array_equal(a, b), (vec, warps)
        assert np.abs(got[1] - ref[1]).max() <= 1e-5 * np.abs(ref[1]).max()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_temporal_blocking_on_one_branch(L, storage):
    """The temporally blocked variant (tiles in shared memory, up to three steps
    per launch, an odd number per launch) on a single clone of the AMS channel,
    the call it serves (one branch, 512 x 128): 267 steps in chunks cut by a
    checkpoint at 250 (launches of 3, then 1) give the populations of the
    register-staged variant bit for bit and its drag to FP32 rounding; the
    checkpoint it took at step 250 is the other's"""
    kw = dict(nx=512, ny=128, obstacle=(120, 56, 16, 16), tau=0.505, gx=1e-6, max_steps=300, ckpt_stride=250,
              storage=storage)
    st = L.STORAGE[storage]
    tb = [v for v in range(L.lbm_step_variant_count())
          if L.lbm_step_variant_kind(v) == 2 and L.lbm_step_variant_info(v)[0] == st]
    assert len(tb) == 1
    out = []
    for forced in (None, tb[0]):
        with Ens(L, 2, seed=4, **kw) as e:
            if forced is not None:
                L.lbm_ensemble_set_variant(e.h, forced)
            L.lbm_ensemble_step_clones(e.h, 267, [1])
            L.lbm_ensemble_branch(e.h, 0, 1, 250, 0.0, 1, 1)  # restores the checkpoint at 250
            d = np.zeros((2, 267))
            L.lbm_ensemble_drag(e.h, 0, 267, d)
            out.append((e.pops(1), e.pops(0), d[1]))
    (f_a, ck_a, d_a), (f_b, ck_b, d_b) = out
    assert np.array_equal(f_a, f_b) and np.array_equal(ck_a, ck_b)
    # the drag (about 0.05) is the sum of some 200 link momenta of order 0.2, in
    # FP32 partials grouped otherwise: differences of a few 1e-7
    assert np.abs(d_a - d_b).max() <= 5e-5 * np.abs(d_a).max()


def test_bounded_wait_runs_out_and_reports(L):
    """A device-side wait on an mbarrier that nothing completes gives up after
    its spin limit and reports LBM_ERR_TIMEOUT; the context remains usable."""
    assert L.lbm_selftest_bounded_wait(20000) == L.LBM_ERR_TIMEOUT
    with Ens(L, 1, **dict(RAGGED, max_steps=4)) as e:
        L.lbm_ensemble_step(e.h, 2)
        assert np.all(np.isfinite(e.drag(0, 2)))


def test_one_step_from_arbitrary_state(L, orc):
    """A single step from a non-equilibrium state loaded into the GPU."""
    kw = dict(nx=96, ny=20, obstacle=(30, 7, 5, 6), tau=0.8, gx=1e-4, gy=2e-5, max_steps=10)
    oc = oracle_cfg(orc, kw)
    rng = np.random.default_rng(3)
    f = orc.init(oc, 1, 0, 0.05) * (1 + 0.01 * rng.standard_normal((9, 20, 96)))
    f[:, orc.solid_mask(oc)] = orc.feq(1.0, 0.0, 0.0)[:, None]
    with Ens(L, 2, **kw) as e:
        L.lbm_ensemble_set_populations(e.h, 1, f)
        L.lbm_ensemble_step(e.h, 1)
        g, fo, _ = orc.step(oc, f)
        assert rel(e.pops(1), g) < 1e-6
        assert abs(e.drag(0, 1)[1, 0] - fo[0]) < 1e-5 * abs(fo[0]) + 1e-9


def test_no_obstacle_and_obstacle_on_wall(L, orc):
    for obst in [(0, 0, 0, 0), (20, 0, 6, 5)]:
        kw = dict(nx=64, ny=16, obstacle=obst, tau=0.7, gx=1e-5, max_steps=50)
        oc = oracle_cfg(orc, kw)
        with Ens(L, 1, seed=4, **kw) as e:
            L.lbm_ensemble_step(e.h, 40)
            f_ref, d_ref = orc.run(oc, orc.init(oc, 4, 0, 0.01), 40)
            assert rel_pop(e.pops(0), f_ref) < POP_TOL
            if obst[2]:
                assert rel(e.drag(0, 40)[0], d_ref) < DRAG_TOL
            else:
                assert np.all(e.drag(0, 40) == 0.0)


def test_minimum_width_channel(L, orc):
    kw = dict(nx=8, ny=4, tau=0.9, gx=1e-4, max_steps=30)
    oc = oracle_cfg(orc, kw)
    with Ens(L, 1, seed=2, **kw) as e:
        L.lbm_ensemble_step(e.h, 30)
        f_ref, _ = orc.run(oc, orc.init(oc, 2, 0, 0.01), 30)
        assert rel_pop(e.pops(0), f_ref) < POP_TOL


def test_mass_conserved_and_moments(L, orc):
    with Ens(L, 2, seed=1, **CFG1) as e:
        m0, px0, py0 = L.lbm_ensemble_moments(e.h, 2)
        oc = oracle_cfg(orc, CFG1)
        for c in range(2):
            mr, pxr, pyr = orc.moments(oc, orc.init(oc, 1, c, 0.01))
            assert abs(m0[c] - mr) < 1e-9 * mr
            assert abs(px0[c] - pxr) < 1e-6 and abs(py0[c] - pyr) < 1e-6
        L.lbm_ensemble_step(e.h, 1000)
        m1, _, _ = L.lbm_ensemble_moments(e.h, 2)
        # FP32 storage: each step rounds every population (2^-24 relative);
        # the mass performs a random walk far below this bound
        assert np.all(np.abs(m1 - m0) / m0 < 1e-5)


def test_window_sum_and_scores_match_oracle(L, orc):
    kw = dict(RAGGED, max_steps=300)
    with Ens(L, 4, seed=3, **kw) as e:
        L.lbm_ensemble_step(e.h, 300)
        d = si.drag_series(4, 300, 11)  # one seeded series for both sides
        L.lbm_ensemble_set_drag(e.h, 0, 300, d)
        with pytest.raises(L.LbmError):  # beyond the clones' time
            L.lbm_ensemble_set_drag(e.h, 0, 301, np.zeros((4, 301)))
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        L.lbm_ensemble_window_sum(e.h, 100, 250, 3.5, out)
        ref = orc.window_sum(d, 100, 250, 3.5)
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-15)
        for window, t_end in [(50, 300), (7, 123), (300, 300), (301, 300)]:
            q = torch.zeros(4, dtype=torch.float64, device="cuda")
            L.lbm_ensemble_scores(e.h, window, 0, t_end, q)
            ref = orc.trailing_mean_max(d, window, t_end)
            got = q.cpu().numpy()
            if window > t_end:
                assert np.all(np.isneginf(got))
            else:
                assert np.allclose(got, ref, rtol=1e-11, atol=1e-14)
        # first crossing of the last scores: brute force on the host series
        L.lbm_ensemble_scores(e.h, 20, 0, 300, None)
        means = np.array([[d[c, t - 20:t].mean() for t in range(20, 301)] for c in range(4)])
        for c in range(4):
            level = np.quantile(means[c], 0.8)
            t = L.lbm_ensemble_first_crossing(e.h, c, level)
            idx = np.nonzero(means[c] > level * (1 + 1e-12) + 1e-18)[0]
            assert t == 20 + idx[0] or abs(means[c][t - 20] - level) < 1e-12 * abs(level)
            assert L.lbm_ensemble_first_crossing(e.h, c, means[c].max() + 1.0) == -1


def test_subset_step_equals_full_step(L):
    kw = dict(RAGGED, max_steps=100)
    with Ens(L, 4, seed=8, **kw) as a, Ens(L, 4, seed=8, **kw) as b:
        L.lbm_ensemble_step(a.h, 30)
        for c in [2, 0]:
            L.lbm_ensemble_step_clones(b.h, 30, [c])
        for c in [0, 2]:
            assert np.array_equal(a.pops(c), b.pops(c))
        assert np.array_equal(a.drag(0, 30)[[0, 2]], b.drag(0, 30)[[0, 2]])
        assert list(L.lbm_ensemble_time(b.h, 4)) == [30, 0, 30, 0]


def test_graph_replay_equals_direct_launches(L):
    """Replayed step-chunk graphs do the same work as direct launches: the
    same populations and drag bit for bit, for whole-ensemble chunks, chunks
    cut by checkpoints, and subset steps whose clone list changes between
    replays of one cached graph."""
    kw = dict(RAGGED, max_steps=200, ckpt_stride=25)
    out = []
    for graphs in (False, True):
        with Ens(L, 4, seed=12, **kw) as e:
            L.lbm_ensemble_set_graphs(e.h, graphs)
            L.lbm_ensemble_step(e.h, 60)       # chunks 25, 25, 10
            L.lbm_ensemble_step(e.h, 15)       # 15
            for c in [3, 1, 0, 2]:             # one cached graph, four different lists
                L.lbm_ensemble_step_clones(e.h, 15, [c])
            L.lbm_ensemble_step(e.h, 50)
            out.append(([e.pops(c) for c in range(4)], e.drag(0, 140)))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[1][1])


def test_clone_exact_copy_and_perturbation(L, orc):
    kw = dict(RAGGED, max_steps=100, n_snapshots=3)
    oc = oracle_cfg(orc, kw)
    with Ens(L, 5, seed=2, **kw) as e:
        L.lbm_ensemble_step(e.h, 20)
        before = [e.pops(c) for c in range(5)]
        hist = e.drag(0, 20)
        parent = torch.tensor([0, 0, 2, 2, 4], dtype=torch.int32, device="cuda")
        L.lbm_ensemble_clone(e.h, parent, 0.0, 1, 0)
        assert np.array_equal(e.pops(1), before[0])
        assert np.array_equal(e.pops(3), before[2])
        assert np.array_equal(e.pops(4), before[4])
        h2 = e.drag(0, 20)
        assert np.array_equal(h2[1], hist[0]) and np.array_equal(h2[3], hist[2])
        # App. D perturbation with a snapshot bank of three states; the oracle
        # perturbs its own states of the same clones at step 20
        L.lbm_ensemble_set_snapshots(e.h, [4, 2, 0])
        at20 = {c: orc.run(oc, orc.init(oc, 2, c, 0.01), 20)[0] for c in (0, 2, 4)}
        snaps = np.stack([at20[4], at20[2], at20[0]])
        parent = torch.tensor([0, 4, 2, 3, 4], dtype=torch.int32, device="cuda")
        L.lbm_ensemble_clone(e.h, parent, 0.002, 77, 5)
        alpha = orc.perturb_alphas(77, 5, 1, 3)
        ref = orc.perturb(oc, at20[4], snaps, alpha, 0.002)
        got = e.pops(1)
        assert rel(got, ref) < 1e-6
        m_ref, _, _ = orc.moments(oc, at20[4])
        m_got, _, _ = orc.moments(oc, got)
        assert abs(m_got - m_ref) / m_ref < 1e-6
        assert np.array_equal(e.pops(3), before[2])  # kept its own slot (a copy of 2 since the first call)


def test_centred_perturbation_matches_oracle(L, orc):
    """the centred App. D coefficients (alpha_n - 1/2, lbm_ensemble_set_perturbation):
    a cloned slot equals the oracle's perturbation with the centred coefficients
    of the same counters, keeps the parent's mass, and differs from the printed
    form; switching back restores the printed form"""
    kw = dict(RAGGED, max_steps=100, n_snapshots=3)
    oc = oracle_cfg(orc, kw)
    with Ens(L, 5, seed=2, **kw) as e:
        L.lbm_ensemble_step(e.h, 20)
        L.lbm_ensemble_set_snapshots(e.h, [4, 2, 0])
        at20 = {c: orc.run(oc, orc.init(oc, 2, c, 0.01), 20)[0] for c in (0, 2, 4)}
        snaps = np.stack([at20[4], at20[2], at20[0]])
        L.lbm_ensemble_set_perturbation(e.h, True)
        L.lbm_ensemble_clone(e.h, torch.tensor([0, 4, 2, 3, 4], dtype=torch.int32, device="cuda"), 0.002, 77, 5)
        ref = orc.perturb(oc, at20[4], snaps, orc.perturb_alphas(77, 5, 1, 3, centred=True), 0.002)
        printed = orc.perturb(oc, at20[4], snaps, orc.perturb_alphas(77, 5, 1, 3), 0.002)
        got = e.pops(1)
        assert rel(got, ref) < 1e-6
        assert rel(got, printed) > 5e-6
        assert abs(orc.moments(oc, got)[0] - orc.moments(oc, at20[4])[0]) / orc.moments(oc, at20[4])[0] < 1e-6
        L.lbm_ensemble_set_perturbation(e.h, False)
        L.lbm_ensemble_clone(e.h, torch.tensor([0, 1, 2, 4, 4], dtype=torch.int32, device="cuda"), 0.002, 77, 5)
        ref3 = orc.perturb(oc, at20[4], snaps, orc.perturb_alphas(77, 5, 3, 3), 0.002)
        assert rel(e.pops(3), ref3) < 1e-6
        assert L.lib().lbm_ensemble_set_perturbation(e.h, 2) == L.LBM_ERR_ARG


def test_step_timing_and_launch_count(L):
    """the tracing hooks: the library's launch counter grows with a step call,
    and with timing on, CUDA events around each step chunk on the ensemble's
    stream report a positive time and the number of timed steps, which reset
    clears"""
    with Ens(L, 2, seed=1, **dict(RAGGED, max_steps=100)) as e:
        n0 = L.lbm_launch_count()
        L.lbm_ensemble_step(e.h, 10)
        assert L.lbm_launch_count() - n0 >= 2  # fused steps and the drag finalisation
        assert L.lbm_ensemble_kernel_time(e.h) == (0.0, 0)  # timing is off by default
        L.lbm_ensemble_set_timing(e.h, True)
        L.lbm_ensemble_step(e.h, 30)
        ms, n = L.lbm_ensemble_kernel_time(e.h, reset=True)
        assert n == 30 and ms > 0.0
        assert L.lbm_ensemble_kernel_time(e.h) == (0.0, 0)


def test_clone_with_a_rejected_parent(L):
    """a parent index outside [0, N) (a rejected selection writes -1) leaves its
    slot unchanged while the other slots are cloned, and the next synchronising
    call reports LBM_ERR_NONFINITE (the rejection's cause)"""
    with Ens(L, 3, seed=3, **dict(RAGGED, max_steps=20)) as e:
        L.lbm_ensemble_step(e.h, 5)
        before = [e.pops(c) for c in range(3)]
        L.lbm_ensemble_clone(e.h, torch.tensor([0, 0, -1], dtype=torch.int32, device="cuda"), 0.0, 1, 0)
        after = [e.pops(c) for c in range(3)]
        assert np.array_equal(after[0], before[0]) and np.array_equal(after[1], before[0])
        assert np.array_equal(after[2], before[2])
        with pytest.raises(L.LbmError) as ei:
            e.drag(0, 5)
        assert ei.value.status == L.LBM_ERR_NONFINITE


def test_snapshot_bank_from_checkpoints(L, orc):
    """The App. D bank refilled from checkpointed states (the flow at the
    branching time) perturbs exactly like states taken live at that time."""
    kw = dict(RAGGED, max_steps=100, ckpt_stride=20, n_snapshots=2)
    oc = oracle_cfg(orc, kw)
    with Ens(L, 4, seed=3, **kw) as e:
        L.lbm_ensemble_step(e.h, 65)
        L.lbm_ensemble_set_snapshots_from_checkpoint(e.h, [3, 1], 2)
        before = e.pops(2)
        parent = torch.tensor([0, 1, 0, 3], dtype=torch.int32, device="cuda")
        L.lbm_ensemble_clone(e.h, parent, 0.002, 5, 9)
        alpha = orc.perturb_alphas(5, 9, 2, 2)
        # the oracle's own states: the bank at step 40, the parent at step 65
        at40 = {c: orc.run(oc, orc.init(oc, 3, c, 0.01), 40)[0] for c in (1, 3)}
        parent0 = orc.run(oc, orc.init(oc, 3, 0, 0.01), 65)[0]
        ref = orc.perturb(oc, parent0, np.stack([at40[3], at40[1]]), alpha, 0.002)
        assert rel(e.pops(2), ref) < 1e-6
        assert not np.array_equal(e.pops(2), before)
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_set_snapshots_from_checkpoint(e.h, [0], 99)


def test_branch_replays_bitwise(L):
    """AMS branching restores the last checkpoint and replays: with eps = 0 the
    branch is the source trajectory, state and drag, bit for bit."""
    kw = dict(RAGGED, max_steps=200, ckpt_stride=25, n_snapshots=2)
    with Ens(L, 3, seed=6, **kw) as e:
        L.lbm_ensemble_step(e.h, 120)
        src_state = None
        L.lbm_ensemble_branch(e.h, 1, 2, 87, 0.0, 3, 1)
        assert list(L.lbm_ensemble_time(e.h, 3)) == [120, 87, 120]
        L.lbm_ensemble_step_clones(e.h, 33, [1])
        assert np.array_equal(e.pops(1), e.pops(2))
        d = e.drag(0, 120)
        assert np.array_equal(d[1], d[2])
        # with a perturbation the branch departs from the source after t_b
        L.lbm_ensemble_set_snapshots(e.h, [0, 2])
        L.lbm_ensemble_branch(e.h, 1, 2, 50, 0.002, 3, 2)
        L.lbm_ensemble_step_clones(e.h, 70, [1])
        d = e.drag(0, 120)
        assert np.array_equal(d[1, :50], d[2, :50])
        assert not np.array_equal(d[1, 50:], d[2, 50:])


def test_branch_replays_across_step_variants(L):
    """An ensemble large enough to step with the wide variant, a branch that
    replays one clone (a small step call, another variant): the replayed
    state is the source's bit for bit, the drag history up to the branch time
    is the source's exactly, and later drag values agree to FP32 rounding
    (their per-warp FP32 partials are grouped differently)."""
    kw = dict(nx=1024, ny=128, obstacle=(250, 56, 16, 16), tau=0.6, gx=2e-5, max_steps=120, ckpt_stride=25)
    with Ens(L, 3, seed=9, **kw) as e:
        L.lbm_ensemble_step(e.h, 80)
        L.lbm_ensemble_branch(e.h, 1, 2, 63, 0.0, 3, 1)
        L.lbm_ensemble_step_clones(e.h, 17, [1])
        assert np.array_equal(e.pops(1), e.pops(2))
        d = e.drag(0, 80)
        assert np.array_equal(d[1, :63], d[2, :63])
        # FP32 partials summed in another grouping: the drag cancels link momenta
        # ten times larger, so FP32 rounding moves it by a few 1e-7
        assert np.abs(d[1, 63:] - d[2, 63:]).max() <= 5e-5 * np.abs(d[2]).max()


def test_perturbed_branch_matches_oracle(L, orc):
    """App. B.1's branch with App. D's perturbation against the oracle: the
    source's state at t_b (the oracle runs the source from its seeded start),
    perturbed with the bank of states at t = 120 and the weights of counter
    (4, iter, dst, n), then 150 further steps; the branch's state and its drag
    after t_b match element by element at the FP32 tolerances, and its drag up
    to t_b is the source's"""
    kw = dict(RAGGED, max_steps=300, ckpt_stride=25, n_snapshots=2)
    oc = oracle_cfg(orc, kw)
    t_b, seed, it, eps, after = 63, 11, 4, 0.05, 150  # eps above App. D's 0.002 so that it shows
    with Ens(L, 3, seed=8, **kw) as e:
        L.lbm_ensemble_step(e.h, 120)
        L.lbm_ensemble_set_snapshots(e.h, [0, 2])
        L.lbm_ensemble_branch(e.h, 1, 2, t_b, eps, seed, it)
        L.lbm_ensemble_step_clones(e.h, after, [1])
        got = e.pops(1)
        d = np.zeros((3, t_b + after))
        L.lbm_ensemble_drag(e.h, 0, t_b + after, d)
    snaps = np.stack([orc.run(oc, orc.init(oc, 8, c, 0.01), 120)[0] for c in (0, 2)])
    f_src, d_src = orc.run(oc, orc.init(oc, 8, 2, 0.01), t_b)
    f_b = orc.perturb(oc, f_src, snaps, orc.perturb_alphas(seed, it, 1, 2), eps)
    f_ref, d_ref = orc.run(oc, f_b, after)
    assert rel_pop(got, f_ref) < POP_TOL
    assert rel(d[1, t_b:], d_ref) < DRAG_TOL
    assert rel(d[1, :t_b], d_src) < DRAG_TOL
    # the perturbation is not negligible at these tolerances
    f_plain, _ = orc.run(oc, f_src, after)
    assert rel_pop(f_plain, f_ref) > 20 * POP_TOL


def test_nonfinite_state_is_reported(L):
    kw = dict(nx=64, ny=16, obstacle=(20, 5, 6, 6), tau=0.6, max_steps=20)
    with Ens(L, 2, **kw) as e:
        f = e.pops(0)
        f[3, 5, 18] = np.inf
        with pytest.raises(L.LbmError) as ei:
            L.lbm_ensemble_set_populations(e.h, 0, f)
        assert ei.value.status == L.LBM_ERR_NONFINITE
        # finite in FP32 but the density of the node next to the obstacle
        # overflows at the next collision: the drag becomes NaN
        f = e.pops(0)
        f[:, 6, 19] = 3e38
        L.lbm_ensemble_set_populations(e.h, 0, f)
        L.lbm_ensemble_step(e.h, 10)
        with pytest.raises(L.LbmError) as ei:
            e.drag(0, 10)
        assert ei.value.status == L.LBM_ERR_NONFINITE


def test_argument_errors(L):
    with Ens(L, 2, **dict(RAGGED, max_steps=10)) as e:
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_step(e.h, 11)
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_step_clones(e.h, 1, [0, 0])
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_step_clones(e.h, 1, [2])
        L.lbm_ensemble_step_clones(e.h, 2, [1])
        with pytest.raises(L.LbmError) as ei:
            L.lbm_ensemble_step(e.h, 1)
        assert ei.value.status == L.LBM_ERR_STATE
        with pytest.raises(L.LbmError):
            e.drag(0, 5)


def test_ams_workload_full_size_sampled_parity(L, orc):
    """The AMS workload's launch shape: 256 trajectories of 512 x 128 with a
    16 x 16 obstacle at x = 128, tau 0.505, autotuned as the bench runs it;
    three sampled trajectories against the oracle over 20 steps."""
    kw = dict(nx=512, ny=128, obstacle=si.channel(512, 128, 16), tau=0.505, gx=1e-6, max_steps=40)
    with Ens(L, 256, seed=21, **kw) as e:
        L.lbm_ensemble_autotune(e.h)
        L.lbm_ensemble_step(e.h, 20)
        d = e.drag(0, 20)
        oc = oracle_cfg(orc, kw)
        for c in (0, 137, 255):
            f_ref, d_ref = orc.run(oc, orc.init(oc, 21, c, 0.01), 20)
            assert rel_pop(e.pops(c), f_ref) < POP_TOL
            assert rel(d[c], d_ref) < DRAG_TOL


@pytest.mark.parametrize("storage,tol", [("fp16", 3e-3), ("bf16", 3e-2)])
def test_precision_workload_full_size_sampled_parity(L, orc, storage, tol):
    """The precision workload's launch shape: 16 clones of 2048 x 512 with a
    64 x 64 obstacle at x = 512, shifted 16-bit storage, autotuned as the bench
    runs it (the row-staged kernel); two sampled clones against the FP64
    oracle over 20 steps, relative to the largest |f - w| as for CFG1."""
    kw = dict(nx=2048, ny=512, obstacle=si.channel(2048, 512, 64), tau=0.505, gx=1e-6, max_steps=40)
    with Ens(L, 16, seed=31, storage=storage, **kw) as e:
        L.lbm_ensemble_autotune(e.h)
        L.lbm_ensemble_step(e.h, 20)
        assert np.all(np.isfinite(e.drag(0, 20)))
        oc = oracle_cfg(orc, kw)
        w = orc.feq(1.0, 0.0, 0.0)[:, None, None]
        for c in (0, 15):
            f_ref, _ = orc.run(oc, orc.init(oc, 31, c, 0.01), 20)
            assert np.abs(e.pops(c) - f_ref).max() / np.abs(f_ref - w).max() < tol, c


def test_zero_steps_and_size_limits(L):
    """zero-step calls change nothing; a history filled to max_steps takes no
    further step; creation rejects, before any allocation, clone counts outside
    [1, 65535], a clone of 2^31 or more values (9 x 32768 x 8192) and lattices
    below the minimum"""
    with Ens(L, 2, **dict(RAGGED, max_steps=10)) as e:
        before = [e.pops(c) for c in range(2)]
        L.lbm_ensemble_step(e.h, 0)
        L.lbm_ensemble_step_clones(e.h, 0, [1])
        for c in range(2):
            assert np.array_equal(e.pops(c), before[c])
        L.lbm_ensemble_step(e.h, 10)
        assert np.all(np.isfinite(e.drag(0, 10)))
        with pytest.raises(L.LbmError):
            L.lbm_ensemble_step(e.h, 1)
    stream = torch.cuda.current_stream()
    big = dict(RAGGED, nx=32768, ny=8192, obstacle=(100, 100, 8, 8))
    for kw, n in [(RAGGED, 0), (RAGGED, 65536), (big, 1), (dict(RAGGED, nx=4, obstacle=(0, 0, 0, 0)), 1),
                  (dict(RAGGED, ny=1, obstacle=(0, 0, 0, 0)), 1)]:
        with pytest.raises(L.LbmError) as ei:
            L.lbm_ensemble_create(L.config(**kw), n, 0, stream)
        assert ei.value.status == L.LBM_ERR_ARG


@pytest.mark.parametrize("storage,tol", [("fp16", 3e-3), ("bf16", 3e-2)])
def test_reduced_precision_storage(L, orc, storage, tol):
    """Shifted 16-bit storage: g = f - w in FP16 (11-bit significand) or BF16
    (8-bit); populations after 200 steps stay within tol of the FP64 oracle
    relative to the largest |f - w| of the flow."""
    with Ens(L, 1, seed=0, storage=storage, **CFG1) as e:
        L.lbm_ensemble_step(e.h, 200)
        oc = oracle_cfg(orc, CFG1)
        f_ref, d_ref = orc.run(oc, orc.init(oc, 0, 0, 0.01), 200)
        w = orc.feq(1.0, 0.0, 0.0)[:, None, None]
        g_ref = f_ref - w
        err = np.abs(e.pops(0) - f_ref).max() / np.abs(g_ref).max()
        assert err < tol
        assert np.all(np.isfinite(e.drag(0, 200)))


def test_full_size_sampled_parity(L, orc):
    """The GKTL workload's launch shape: 64 clones of 1024 x 256 with a 32 x 32
    obstacle at x = 256, tau 0.505; two sampled clones against the oracle
    over 20 steps."""
    kw = dict(nx=1024, ny=256, obstacle=si.channel(1024, 256, 32, 256), tau=0.505, gx=1e-6, max_steps=40)
    with Ens(L, 64, seed=12, **kw) as e:
        L.lbm_ensemble_autotune(e.h)
        L.lbm_ensemble_step(e.h, 20)
        d = e.drag(0, 20)
        oc = oracle_cfg(orc, kw)
        for c in (0, 63):
            f_ref, d_ref = orc.run(oc, orc.init(oc, 12, c, 0.01), 20)
            assert rel_pop(e.pops(c), f_ref) < POP_TOL
            assert rel(d[c], d_ref) < DRAG_TOL
