"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: it only draws numbers
(weights, scores, populations) from numpy generators with fixed seeds, so the
same inputs can be fed to both implementations.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def log_weights(n: int, seed: int, spread: float = 1.0) -> np.ndarray:
    """GKTL exponents s_n = k * integral, Gaussian with the given spread."""
    return rng(seed).normal(0.0, spread, size=n)


def normalised_weights(n: int, seed: int, spread: float = 1.0) -> np.ndarray:
    """Positive weights scaled so that they sum to n (the selection input)."""
    s = log_weights(n, seed, spread)
    e = np.exp(s - s.max())
    return n * e / e.sum()


def scores(n: int, seed: int, n_ties: int = 0) -> np.ndarray:
    """AMS maximum scores; n_ties > 0 makes that many entries share the minimum."""
    q = rng(seed).normal(0.0, 1.0, size=n)
    if n_ties > 1:
        idx = rng(seed + 1).choice(n, size=n_ties, replace=False)
        q[idx] = q.min() - 1.0
    return q


def channel(nx: int, ny: int, side: int, cx: int | None = None):
    """Square obstacle of the given side centred on the channel's mid-height at x = cx
    (default nx/4): solid cells [cx - side/2, cx + side/2) x [ny/2 - side/2, ny/2 + side/2)."""
    if cx is None:
        cx = nx // 4
    if side <= 0:
        return (0, 0, 0, 0)
    return (cx - side // 2, ny // 2 - side // 2, side, side)


def cnn_params(seed: int) -> np.ndarray:
    """A parameter vector of the learned-score network in its documented flat
    layout (FP32 values): for conv layer l (input channels 8, then 32) a
    [32][80] or [32][304] block, 9 * C_in tap weights drawn uniformly within
    the He bound sqrt(6 / (9 * C_in)), then a bias drawn in [-0.1, 0.1], then
    zero padding; then 32 head weights within 1/sqrt(32) and a zero head bias."""
    g = rng(seed)
    out = []
    for cin, kpad in ((8, 80), (32, 304), (32, 304), (32, 304)):
        block = np.zeros((32, kpad))
        a = np.sqrt(6.0 / (9 * cin))
        block[:, :9 * cin] = g.uniform(-a, a, (32, 9 * cin))
        block[:, 9 * cin] = g.uniform(-0.1, 0.1, 32)
        out.append(block.ravel())
    out.append(g.uniform(-1, 1, 32) / np.sqrt(32.0))
    out.append(np.zeros(1))
    return np.concatenate(out).astype(np.float32)


def drag_series(n: int, steps: int, seed: int, mean: float = 1e-3, sd: float = 2e-3, rho: float = 0.9) -> np.ndarray:
    """n independent synthetic drag series [n, steps]: a stationary Gaussian
    AR(1) sequence with the given mean, standard deviation and lag-1
    correlation (the structure the statistics read: fluctuations, a
    correlation time, excursions above levels)"""
    g = rng(seed)
    x = np.zeros((n, steps))
    x[:, 0] = g.normal(0.0, 1.0, n)
    e = g.normal(0.0, np.sqrt(1.0 - rho * rho), (n, steps))
    for t in range(1, steps):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return mean + sd * x
