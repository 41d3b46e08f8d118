"""Long-run parity beyond the predictability horizon: the drag statistics of
the GPU in FP32, shifted FP16 and shifted BF16 storage against the FP64 oracle
on the same seeds, in a chaotic flow.

Flow: the open channel of Sec. 2 at a quarter of its length - 129 x 33, a
square of side R = 8 at the centre, the entrance grid of R/2 bars every R
from x = R, a sponge over the last 32 columns up to tau = 1, central moments,
tau = 0.5015, u_c = 0.08 (drag correlation time about 340 steps).  In this
flow a relative change of 1e-6 in one population grows to the size of the
drag's fluctuations within about 4000 steps (measured on the GPU), so FP32
and FP64 trajectories of one seed separate there, and past it only their
statistics can agree (the element-wise comparisons of the other tests cover
the first 200 steps).  The size is set by the oracle's cost: its central-
moment collision inverts a 9 x 9 matrix at every node.

Statistics: drag samples pooled over 32 trajectories and steps
[4000, 8000).  Bounds:
  - mean and standard deviation within 2%, or within three standard errors
    of their two-sample difference where sampling noise is larger than 2%
    (standard errors from the spread of per-trajectory values);
  - Kolmogorov-Smirnov distance below 1.5 times the median distance between
    two halves of the oracle's own trajectories over 20 random splits (the
    null of one law, at half the sample size);
  - the upper tail: the fraction of GPU samples above the oracle's 99th and
    99.9th percentiles within three spreads of that fraction (from the
    difference between oracle halves) plus a fifth of it."""
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CH = dict(nx=129, ny=33, obstacle=(60, 12, 8, 8), tau=0.5015, open_x=1, u_in=0.08, grid=(8, 4, 4, 4),
          sponge_len=32, sponge_tau=1.0)
N_TRAJ, STEPS, T0, SEED = 32, 8000, 4000, 21


def oracle_drag(clone):
    """one oracle trajectory (seeded start of the given clone), its drag series"""
    import oracle
    kw = dict(CH)
    c = oracle.cfg(kw.pop("nx"), kw.pop("ny"), obstacle=kw.pop("obstacle"), collision=1, **kw)
    _, d = oracle.run(c, oracle.init(c, SEED, clone, 0.01), STEPS)
    return d


@pytest.fixture(scope="module")
def oracle_runs():
    cores = len(os.sched_getaffinity(0))
    with mp.get_context("spawn").Pool(min(cores, N_TRAJ)) as pool:
        return np.stack(pool.map(oracle_drag, range(N_TRAJ)))


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


def gpu_drag(L, storage):
    cfg = L.config(**CH, collision="cm", storage=storage, max_steps=STEPS, init_amp=0.01)
    e = L.lbm_ensemble_create(cfg, N_TRAJ, SEED, torch.cuda.current_stream())
    try:
        L.lbm_ensemble_step(e, STEPS)
        d = np.zeros((N_TRAJ, STEPS))
        L.lbm_ensemble_drag(e, 0, STEPS, d)
    finally:
        L.lbm_ensemble_destroy(e)
    return d


def ks(a, b):
    """two-sample Kolmogorov-Smirnov distance"""
    a, b = np.sort(a.ravel()), np.sort(b.ravel())
    x = np.concatenate([a, b])
    return np.abs(np.searchsorted(a, x, side="right") / a.size - np.searchsorted(b, x, side="right") / b.size).max()


def two_sample_se(per_a, per_b):
    return np.sqrt(per_a.var(ddof=1) / per_a.size + per_b.var(ddof=1) / per_b.size)


def test_trajectories_separate(L, oracle_runs):
    """the horizon is chaotic: the FP32 trajectories have left their FP64
    counterparts by the statistics window's end"""
    g = gpu_drag(L, "fp32")
    o = oracle_runs
    sig = o[:, T0:].std()
    early = np.abs(g[:, :200] - o[:, :200]).max() / np.abs(o[:, :200]).max()
    late = np.abs(g[:, -1000:] - o[:, -1000:]).max(axis=1) / sig
    assert early < 1e-4
    assert np.median(late) > 0.5, late


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_drag_statistics_match_oracle(L, oracle_runs, storage):
    g = gpu_drag(L, storage)[:, T0:]
    o = oracle_runs[:, T0:]
    assert np.all(np.isfinite(g))
    rng = np.random.default_rng(0)
    # mean and standard deviation
    for stat in (np.mean, np.std):
        gs, os_ = stat(g), stat(o)
        per_g, per_o = stat(g, axis=1), stat(o, axis=1)
        tol = max(0.02 * abs(os_), 3 * two_sample_se(per_g, per_o))
        print(f"{storage} {stat.__name__}: gpu {gs:.6g} oracle {os_:.6g} rel {abs(gs - os_) / abs(os_):.4f} "
              f"tol {tol / abs(os_):.4f}")
        assert abs(gs - os_) <= tol
    # the law: KS distance against the null of two oracle halves
    null = []
    for _ in range(20):
        p = rng.permutation(N_TRAJ)
        null.append(ks(o[p[:N_TRAJ // 2]], o[p[N_TRAJ // 2:]]))
    d = ks(g, o)
    print(f"{storage} KS {d:.4f} null median {np.median(null):.4f}")
    assert d < 1.5 * np.median(null)
    # the upper tail: exceedances of the oracle's quantiles; the spread of the
    # difference between two oracle halves (16 against 16 trajectories) is
    # sqrt(2) times that of 32 against 32
    for q in (0.99, 0.999):
        a = np.quantile(o, q)
        frac = (g > a).mean()
        diffs = []
        for _ in range(20):
            p = rng.permutation(N_TRAJ)
            diffs.append((o[p[:N_TRAJ // 2]] > a).mean() - (o[p[N_TRAJ // 2:]] > a).mean())
        spread = np.std(diffs) / np.sqrt(2)
        print(f"{storage} tail {q}: gpu {frac:.5f} oracle {1 - q:.5f} spread {spread:.5f}")
        assert abs(frac - (1 - q)) <= 3 * spread + 0.2 * (1 - q)


def test_storage_formats_within_two_percent_of_fp32(L):
    """Shifted FP16 and BF16 storage against FP32 on 2048 trajectories of the
    same seeds (three standard errors of the mean and standard deviation are
    about 1%, so a 2% bound is resolved): mean and standard deviation within
    2%, KS distance below 0.01, and the upper tail kept - the exceedances of
    FP32's 99th and 99.9th percentiles within three sampling spreads plus a
    tenth of the tail.  The spread is that of the difference between two
    independent ensembles of this size, from random halves of the FP32
    trajectories (past the horizon the 16-bit trajectories are independent
    samples of their law): the drag decorrelates in about 340 steps, so the
    99.9th percentile rests on a few tens of independent exceedances and is
    known to about 15% (measured at the 99.9th: FP16 -9% and -10%, BF16 -15%
    and -29% on two builds whose trajectories differ in their last bits)."""
    n = 2048
    runs = {}
    for st in ("fp32", "fp16", "bf16"):
        cfg = L.config(**CH, collision="cm", storage=st, max_steps=STEPS, init_amp=0.01)
        e = L.lbm_ensemble_create(cfg, n, SEED, torch.cuda.current_stream())
        try:
            L.lbm_ensemble_step(e, STEPS)
            d = np.zeros((n, STEPS))
            L.lbm_ensemble_drag(e, 0, STEPS, d)
        finally:
            L.lbm_ensemble_destroy(e)
        runs[st] = d[:, T0:]
    ref = runs["fp32"]
    rng = np.random.default_rng(1)
    for st in ("fp16", "bf16"):
        g = runs[st]
        assert np.all(np.isfinite(g))
        for stat in (np.mean, np.std):
            dev = (stat(g) - stat(ref)) / abs(stat(ref))
            print(f"{st} {stat.__name__} {dev:+.4f}")
            assert abs(dev) <= 0.02
        assert ks(g, ref) < 0.01
        for q in (0.99, 0.999):
            a = np.quantile(ref, q)
            frac = (g > a).mean()
            diffs = []
            for _ in range(20):
                p = rng.permutation(n)
                diffs.append((ref[p[:n // 2]] > a).mean() - (ref[p[n // 2:]] > a).mean())
            spread = np.std(diffs) / np.sqrt(2)  # two ensembles of n / 2 differ by sqrt(2) times two of n
            print(f"{st} exceedance of the FP32 {q} quantile {frac:.5f} spread {spread:.5f}")
            assert abs(frac - (1 - q)) <= 3 * spread + 0.1 * (1 - q)
