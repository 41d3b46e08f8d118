"""Host helpers of bench.py on the CPU: the two-sample KS distance of the
perturbation check, the pooled correlation time (FFT lagged sums against the
direct sums, and the quarter period of a sine), and the lookup of the recorded
DRAM traffic by kernel label."""
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
