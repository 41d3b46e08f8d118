"""Host helpers of bench.py on the CPU: the two-sample KS distance of the
perturbation check, the pooled correlation time (FFT lagged sums against the
direct sums, and the quarter period of a sine), the lookup of the recorded
DRAM traffic by kernel label, and the arithmetic of the estimate benches (the
binomial error of a direct frequency and the time to a target error, against
simulation; the generalized-AMS estimate of one run, by hand)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ks_distance_against_definition():
    rng = np.random.default_rng(0)
    a, b = rng.normal(0, 1, 300), rng.normal(0.3, 1.2, 200)
    grid = np.concatenate([a, b])
    brute = max(abs((a <= g).mean() - (b <= g).mean()) for g in grid)
    assert abs(bench.ks_distance(a, b) - brute) < 1e-15
    assert bench.ks_distance(a, a) == 0.0
    assert bench.ks_distance(np.zeros(5), np.ones(5)) == 1.0


def test_pooled_tau_c_matches_direct_sums():
    rng = np.random.default_rng(1)
    x = np.zeros((3, 2000))
    e = rng.standard_normal((3, 2000))
    for t in range(1, 2000):
        x[:, t] = 0.95 * x[:, t - 1] + e[:, t]
    xc = x - x.mean()
    var = (xc * xc).mean()
    direct = next(lag for lag in range(1, 1000) if (xc[:, :-lag] * xc[:, lag:]).mean() / var <= 0.0)
    assert bench.pooled_tau_c(x, 999) == direct
    # a sine of period 400 first reaches zero correlation at a quarter period
    s = np.sin(2 * np.pi * np.arange(8000) / 400)[None, :]
    assert abs(bench.pooled_tau_c(s, 1000) - 100) <= 1
    assert bench.pooled_tau_c(np.cumsum(np.ones((2, 50)), axis=1), 3) == -1


def test_traffic_records_are_keyed_without_warps():
    assert bench.traffic_key("step_kernel<fp32, vec=4, warps=8>") == "step_kernel<fp32, vec=4>"
    assert bench.traffic_key("step_kernel<fp32, vec=4, warps=4, open> + open_bc_kernel") == \
        "step_kernel<fp32, vec=4, open> + open_bc_kernel"
    for (workload, key), rec in bench.NCU_TRAFFIC.items():
        assert "warps=" not in key
        assert 0 < rec["bytes_per_site"] < 80
        assert len(bench.kernel_sha(rec["files"])) == 16


def test_binomial_cv_matches_simulated_frequencies():
    rng = np.random.default_rng(2)
    p, n = 0.03, 400
    freqs = rng.binomial(n, p, size=20000) / n
    assert abs(freqs.std() / freqs.mean() / bench.binomial_cv(p, n) - 1) < 0.02
    assert bench.binomial_cv(0.0, 10) == float("inf") and bench.binomial_cv(1.0, 10) == float("inf")


def test_seconds_to_rel_error_from_averaged_runs():
    # a mean of m runs with per-run error cv has error cv / sqrt(m): 16 runs
    # of 2 s at cv = 0.8 reach 0.2
    assert abs(bench.seconds_to_rel_error(2.0, 0.8) - 32.0) < 1e-12
    rng = np.random.default_rng(3)
    runs = rng.exponential(1.0, size=(20000, 25))  # cv 1 per run, 25 runs -> 0.2
    means = runs.mean(axis=1)
    assert abs(means.std() / means.mean() - 0.2) < 0.01
    assert abs(bench.seconds_to_rel_error(1.0, 1.0) - 25.0) < 1e-12


def test_ams_estimate_on_a_hand_computed_run():
    # N = 4, two iterations killing one each: weight (3/4)^2; 2 of 4 final maxima
    # at or above the level (one exactly at it)
    lw = 2 * np.log(1 - 1 / 4)
    assert abs(bench.ams_estimate(lw, [0.5, 0.7, 0.9, 0.7], 0.7) - 0.5625 * 0.75) < 1e-15
    assert abs(bench.ams_estimate(lw, [0.5, 0.6, 0.9, 0.7], 0.7) - 0.5625 * 0.5) < 1e-15
    assert bench.ams_estimate(0.0, [0.1, 0.2], 0.3) == 0.0


def test_solid_cells_of_the_workloads():
    import argparse
    gktl = bench.workload(argparse.Namespace(workload="gktl", clones=None))
    assert bench.solid_cells(gktl) == 32 * 32
    # open channel: the 16 x 16 square and 8 bars of 8 rows (rows 8-15, 24-31,
    # ..., 120-127 of 129) over the grid's 8 columns
    opn = bench.workload(argparse.Namespace(workload="open", clones=None))
    assert bench.solid_cells(opn) == 16 * 16 + 8 * 64


def test_cpu_baseline_record_of_the_gpu_arm():
    """the CPU-baseline object of the GPU arm's line: the oracle on two host
    processes over the bounded sample"""
    import argparse
    w = bench.workload(argparse.Namespace(workload="gktl", clones=None))
    cb = bench.cpu_baseline(w, 2)
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["unit"] == "GLUPS"
    assert 0 < cb["per_core"] <= 1.2 * cb["value"] and "1024x256" in cb["sample"]


def test_open_workload_is_the_paper_channel():
    """the open-channel workload takes its numbers from Sec. 2
    (tests/golden/paper_channel_sec2.txt); tau follows from Re_grid on the
    bar size R/2 and the lattice viscosity nu = (tau - 1/2)/3 of App. A"""
    import argparse
    g = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_channel_sec2.txt")) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = (s.strip() for s in line.split("="))
                g[k] = float(v)
    w = bench.workload(argparse.Namespace(workload="open", clones=None))
    assert (w["nx"], w["ny"], w["side"]) == (g["nx"], g["ny"], g["R"])
    x0, y0, sx, sy = w["obst"]
    assert (sx, sy) == (g["R"], g["R"])
    assert abs((x0 + sx / 2) - w["nx"] / 2) <= 0.5 and abs((y0 + sy / 2) - w["ny"] / 2) <= 0.5  # centred
    _, _, bar, gap = bench.OPEN_GRID
    assert (bar, gap) == (g["grid_bar"], g["grid_spacing"])
    assert bench.OPEN_UC == g["u_centre"]
    nu = g["u_centre"] * (g["R"] / 2) / g["Re_grid"]
    assert abs(bench.OPEN_TAU - (0.5 + 3 * nu)) < 1e-15


def test_perturbation_parameters_are_the_papers():
    """every bench workload perturbs with App. D's epsilon and snapshot count
    (tests/golden/perturbation_app_d.txt)"""
    g = {}
    with open(os.path.join(ROOT, "tests", "golden", "perturbation_app_d.txt")) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = (s.strip() for s in line.split("="))
                g[k] = float(v)
    assert bench.EPS == g["epsilon"] and bench.N_SNAP == g["N_s"]
