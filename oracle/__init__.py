"""Oracle: plain, slow, single-threaded FP64 CPU implementation of the method.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
(``paper_2005_09323_gb300``) never imports this package, and this package never
imports the product: they share no code.

The C sources (``oracle/*.c``) follow the paper's appendices step by step; see
the header comment of each file for the passage it restates.  This module only
compiles them (``build()``) and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["philox.c", "lbm.c", "select.c", "ou.c"]


def compile_sources(src_dir: str, out: str, extra=()) -> str:
    """gcc, -O2, IEEE FP64 (no contraction into fused multiply-adds, so x86 and
    Arm hosts round alike) of the oracle's C sources found in src_dir into
    the shared library out, with the extra compiler arguments given"""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *extra,
           *[os.path.join(src_dir, s) for s in _SOURCES], "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``oracle/liboracle.so``."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO):
        so_m = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_m for s in srcs):
            return _SO
    return compile_sources(_HERE, _SO)


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_SO)
    return _lib


@contextlib.contextmanager
def using(path: str):
    """Within the block every wrapper of this module calls the library at path
    (a build of modified sources: the mutation tests plant one mistake each)
    instead of liboracle.so."""
    global _lib
    saved = lib()
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = saved


def _load(path: str):
    L = C.CDLL(path)
    d, i32, i64, u64, p = C.c_double, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p
    L.orc_philox4x64.argtypes = [p, p, p]
    L.orc_u01.argtypes = [u64]; L.orc_u01.restype = d
    L.orc_below.argtypes = [u64, u64]; L.orc_below.restype = u64
    L.orc_feq.argtypes = [d, d, d, p]
    L.orc_guo.argtypes = [d, d, d, d, p]
    L.orc_init.argtypes = [p, u64, i32, d, p]
    L.orc_step.argtypes = [p, p, p, p, p]
    L.orc_run.argtypes = [p, p, p, i32, p]
    L.orc_moments.argtypes = [p, p, p, p, p]
    L.orc_macro.argtypes = [p, p, p, p, p]
    L.orc_is_solid.argtypes = [p, C.c_int, C.c_int]; L.orc_is_solid.restype = C.c_int
    L.orc_cm_collide.argtypes = [p, d, d, p, p, p, p]
    L.orc_tau_at.argtypes = [p, C.c_int]; L.orc_tau_at.restype = d
    L.orc_inlet_u.argtypes = [p, C.c_int]; L.orc_inlet_u.restype = d
    L.orc_observables.argtypes = [p, p, p]; L.orc_observables.restype = C.c_int
    L.orc_perturb_alphas.argtypes = [u64, u64, i32, i32, p]
    L.orc_perturb.argtypes = [p, p, i32, p, p, d, p]
    L.orc_gktl_weights.argtypes = [i32, p, p, p]; L.orc_gktl_weights.restype = C.c_int
    L.orc_gktl_select.argtypes = [i32, p, u64, u64, p]; L.orc_gktl_select.restype = C.c_int
    L.orc_ams_select.argtypes = [i32, p, u64, u64, p, p, p, p]; L.orc_ams_select.restype = C.c_int
    L.orc_ou_noise.argtypes = [u64, u64, u64, u64]; L.orc_ou_noise.restype = d
    L.orc_ou_gktl.argtypes = [i32, i32, i32, d, d, d, u64, p, i32, p, p, p, p]; L.orc_ou_gktl.restype = d
    L.orc_ou_direct_max.argtypes = [i64, i32, d, u64, i32, p, p]
    L.orc_ou_ams.argtypes = [i32, i32, d, d, i32, u64, p]; L.orc_ou_ams.restype = d
    L.orc_ou_ams_score.argtypes = [i32, i32, d, i32, i32, d, d, i32, u64, p, p, p, i32, p, p, p]
    L.orc_ou_ams_score.restype = d
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Cfg(C.Structure):
    """Mirror of ``orc_cfg``: channel nx x ny, solid cells [ox0,ox0+ow) x [oy0,oy0+oh)."""
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("ox0", C.c_int32), ("oy0", C.c_int32),
                ("ow", C.c_int32), ("oh", C.c_int32), ("tau", C.c_double), ("gx", C.c_double),
                ("gy", C.c_double), ("collision", C.c_int32), ("omega_bulk", C.c_double),
                ("omega_3", C.c_double), ("omega_4", C.c_double), ("open_x", C.c_int32), ("u_in", C.c_double),
                ("grid_x0", C.c_int32), ("grid_w", C.c_int32), ("grid_bar", C.c_int32), ("grid_gap", C.c_int32),
                ("sponge_len", C.c_int32), ("sponge_tau", C.c_double)]


def cfg(nx, ny, obstacle=(0, 0, 0, 0), tau=0.6, gx=0.0, gy=0.0, collision=0, omega_bulk=1.0, omega_3=1.0,
        omega_4=1.0, open_x=0, u_in=0.0, grid=(0, 0, 0, 0), sponge_len=0, sponge_tau=1.0) -> Cfg:
    """collision 0: BGK; 1: central-moment MRT (shear at 1/tau, the other
    rates as given).  open_x = 1: inlet/outlet channel with centreline inlet
    velocity u_in, entrance grid (x0, width, bar, gap) and sponge."""
    ox0, oy0, ow, oh = obstacle
    gx0, gw, gbar, ggap = grid
    return Cfg(nx, ny, ox0, oy0, ow, oh, tau, gx, gy, collision, omega_bulk, omega_3, omega_4, open_x, u_in,
               gx0, gw, gbar, ggap, sponge_len, sponge_tau)


# ---------------------------------------------------------------- rng
def philox4x64(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    o = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(x: int) -> float:
    return lib().orc_u01(int(x))


def below(x: int, m: int) -> int:
    return lib().orc_below(int(x), int(m))


# ---------------------------------------------------------------- lbm
def feq(rho, ux, uy):
    o = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _ptr(o))
    return o


def guo(ux, uy, gx, gy):
    o = np.zeros(9)
    lib().orc_guo(ux, uy, gx, gy, _ptr(o))
    return o


def cm_collide(f, ux, uy, feq9, S9, rates):
    """central-moment collision of one node (orc_cm_collide)"""
    f = np.ascontiguousarray(f, dtype=np.float64)
    a = np.ascontiguousarray(feq9, dtype=np.float64)
    b = np.ascontiguousarray(S9, dtype=np.float64)
    r = np.ascontiguousarray(rates, dtype=np.float64)
    o = np.zeros(9)
    lib().orc_cm_collide(_ptr(f), ux, uy, _ptr(a), _ptr(b), _ptr(r), _ptr(o))
    return o


def init(c: Cfg, seed: int, clone: int, amp: float) -> np.ndarray:
    f = np.zeros((9, c.ny, c.nx))
    lib().orc_init(C.byref(c), seed, clone, amp, _ptr(f))
    return f


def step(c: Cfg, f: np.ndarray):
    """One step; returns (f_new, force_on_obstacle[2], force_on_walls[2])."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    fo = np.zeros(2)
    fw = np.zeros(2)
    lib().orc_step(C.byref(c), _ptr(f), _ptr(out), _ptr(fo), _ptr(fw))
    return out, fo, fw


def run(c: Cfg, f: np.ndarray, n: int):
    """n steps; returns (f_final, drag[n]) with drag[t] the x-force after step t+1."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    scratch = np.empty_like(f)
    drag = np.zeros(max(n, 1))
    lib().orc_run(C.byref(c), _ptr(f), _ptr(scratch), n, _ptr(drag))
    return f, drag[:n]


def moments(c: Cfg, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    m, px, py = C.c_double(), C.c_double(), C.c_double()
    lib().orc_moments(C.byref(c), _ptr(f), C.byref(m), C.byref(px), C.byref(py))
    return m.value, px.value, py.value


def macro(c: Cfg, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros((c.ny, c.nx)); ux = np.zeros_like(rho); uy = np.zeros_like(rho)
    lib().orc_macro(C.byref(c), _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def observables(c: Cfg, f: np.ndarray) -> np.ndarray:
    """[p_fb, p_base, gamma_top, gamma_bottom] of a post-collision state (Sec. 2.1
    eq. drag_approx, Sec. 3.2 eq. avg_shear_def)"""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(4)
    if lib().orc_observables(C.byref(c), _ptr(f), _ptr(out)) != 0:
        raise ValueError("observables need a square with two fluid rows above and below and a column beside it")
    return out


def solid_mask(c: Cfg) -> np.ndarray:
    """solid cells: the square and, in an open channel, the entrance grid"""
    m = np.zeros((c.ny, c.nx), dtype=bool)
    for y in range(c.ny):
        for x in range(c.nx):
            m[y, x] = bool(lib().orc_is_solid(C.byref(c), x, y))
    return m


def perturb_alphas(seed, it, slot, n_s, centred=False):
    """App. D coefficients alpha_n, uniform in [0, 1) from the counter
    (4, iter, slot, n); centred=True subtracts 1/2 (the centred reading of the
    perturbation: the same random combination of snapshots with no mean pull
    towards them)"""
    a = np.zeros(n_s)
    lib().orc_perturb_alphas(seed, it, slot, n_s, _ptr(a))
    return a - 0.5 if centred else a


def perturb(c: Cfg, f, snaps, alpha, eps):
    f = np.ascontiguousarray(f, dtype=np.float64)
    snaps = np.ascontiguousarray(snaps, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    out = np.empty_like(f)
    lib().orc_perturb(C.byref(c), _ptr(f), int(len(alpha)), _ptr(snaps), _ptr(alpha), eps, _ptr(out))
    return out


# ---------------------------------------------------------------- selection
def gktl_weights(s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    W = np.zeros_like(s)
    logR = C.c_double()
    rc = lib().orc_gktl_weights(len(s), _ptr(s), _ptr(W), C.byref(logR))
    if rc != 0:
        raise ValueError(f"orc_gktl_weights: status {rc}")
    return W, logR.value


def gktl_select(W, seed, it):
    W = np.ascontiguousarray(W, dtype=np.float64)
    parent = np.zeros(len(W), dtype=np.int32)
    rc = lib().orc_gktl_select(len(W), _ptr(W), seed, it, _ptr(parent))
    if rc != 0:
        raise ValueError(f"orc_gktl_select: status {rc}")
    return parent


def ams_select(Q, seed, it):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = len(Q)
    killed = np.zeros(n, dtype=np.int32)
    surv = np.zeros(n, dtype=np.int32)
    nk = C.c_int32()
    z = C.c_double()
    rc = lib().orc_ams_select(n, _ptr(Q), seed, it, _ptr(killed), C.byref(nk), _ptr(surv), C.byref(z))
    if rc != 0:
        raise ValueError(f"orc_ams_select: status {rc}")
    k = nk.value
    return killed[:k].copy(), (surv[:k].copy() if k < n else np.zeros(0, np.int32)), z.value


# ---------------------------------------------------------------- OU test process
def ou_gktl(n, n_periods, steps_per_period, dt, k, seed, window_steps=0, kappa=0.0, full=False):
    """GKTL on the OU process (orc_ou_gktl).  Returns (log Z, final integrals,
    final max of the window mean or None); with full=True a dict that adds the
    final histories [N][M + 1], the potential's corrections
    kappa (V(x_{T_a}) - V(x_0)) and log R of each cloning step."""
    M = n_periods * steps_per_period
    fi = np.zeros(n)
    mm = np.zeros(n)
    hist = np.zeros((n, M + 1)) if full else None
    corr = np.zeros(n)
    logR = np.zeros(n_periods)
    logZ = lib().orc_ou_gktl(n, n_periods, steps_per_period, dt, k, kappa, seed, _ptr(fi), window_steps,
                             _ptr(mm) if window_steps > 0 else None, _ptr(hist) if full else None, _ptr(corr),
                             _ptr(logR))
    if full:
        return dict(log_z=logZ, integrals=fi, max_mean=(mm if window_steps > 0 else None), hist=hist,
                    correction=corr, log_r=logR)
    return logZ, fi, (mm if window_steps > 0 else None)


def ou_direct_max(n, n_steps, dt, seed, levels):
    levels = np.ascontiguousarray(levels, dtype=np.float64)
    frac = np.zeros_like(levels)
    lib().orc_ou_direct_max(n, n_steps, dt, seed, len(levels), _ptr(levels), _ptr(frac))
    return frac


def ou_ams(n, n_steps, dt, a, j_max, seed):
    it = C.c_int32()
    p = lib().orc_ou_ams(n, n_steps, dt, a, j_max, seed, C.byref(it))
    return p, it.value


def ou_ams_score(n, n_steps, dt, stride, score_window, score_level, a, j_max, seed):
    """AMS on the OU process with a trailing-mean score seen every stride steps
    (orc_ou_ams_score).  Returns (estimate, iterations, log weight, event
    maxima[N], killed records (log weight before the kill, event maximum))."""
    it = C.c_int32()
    lw = C.c_double()
    nr = C.c_int32()
    mx = np.zeros(n)
    cap = j_max * n
    rl, rm = np.zeros(max(cap, 1)), np.zeros(max(cap, 1))
    p = lib().orc_ou_ams_score(n, n_steps, dt, stride, score_window, score_level, a, j_max, seed, C.byref(it),
                               C.byref(lw), _ptr(mx), cap, C.byref(nr), _ptr(rl), _ptr(rm))
    return p, it.value, lw.value, mx, (rl[:nr.value].copy(), rm[:nr.value].copy())


# ---------------------------------------------------------------- observables & estimators
def window_sum(drag: np.ndarray, t0: int, t1: int, k: float) -> np.ndarray:
    """GKTL exponent of eq. (Weight): k times the time integral of the drag over
    steps t0 < t <= t1 (dt = 1 lattice step), per trajectory.  drag[n, t-1] is the
    drag after step t."""
    return k * np.sum(np.asarray(drag, dtype=np.float64)[:, t0:t1], axis=1)


def trailing_mean_max(drag: np.ndarray, window: int, t_end: int | None = None, t_begin: int = 0) -> np.ndarray:
    """max over t in [t_begin + window, t_end] of (1/window) sum_{s=t-window+1}^{t} drag(s):
    the time-averaged drag F_T of eq. (def_time_averaged_drag) with T = window
    steps, maximised along each trajectory that starts at t_begin (AMS score
    maximum Q_n; GKTL event amplitude).  -inf when t_end < t_begin + window.
    drag[n, t-1] is the drag after step t."""
    d = np.asarray(drag, dtype=np.float64)
    if t_end is None:
        t_end = d.shape[1]
    out = np.full(d.shape[0], -np.inf)
    if t_end < t_begin + window:
        return out
    # the window ending after step t holds drag[:, t - window:t]; t runs over
    # [t_begin + window, t_end], so the windows start at t_begin .. t_end - window
    windows = np.lib.stride_tricks.sliding_window_view(d[:, t_begin:t_end], window, axis=1)
    return np.max(np.sum(windows, axis=2) / window, axis=1)


def gktl_probability(log_z: float, k: float, integrals: np.ndarray, maxima: np.ndarray,
                     levels: np.ndarray, correction: np.ndarray | None = None) -> np.ndarray:
    """App. C.2: P(F_T >= a) ~ (1/N) sum_j Z e^{-k int_0^{T_a} A_j} 1{max F_T^(j) >= a},
    the biased path measure of eq. (Biased_Path_Approximation) inverted (the
    printed exponent's sign is read as the inversion requires).  With a
    potential in the exponents, correction[j] = kappa (V_j(T_a) - V_j(0)) of
    each final trajectory divides its weight by e^{correction[j]}."""
    integrals = np.asarray(integrals, dtype=np.float64)
    maxima = np.asarray(maxima, dtype=np.float64)
    corr = np.zeros_like(integrals) if correction is None else np.asarray(correction, dtype=np.float64)
    w = np.exp(log_z - k * integrals - corr)
    return np.array([np.sum(w * (maxima >= a)) / len(w) for a in np.atleast_1d(levels)])


def return_time(p: np.ndarray, t_a: float, t_window: float) -> np.ndarray:
    """App. C.2: r(a) = -(T_a - T) / ln(1 - P(F_T >= a))."""
    p = np.asarray(p, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return -(t_a - t_window) / np.log1p(-p)


def ams_probability(log_weight: float, maxima: np.ndarray, level: float, killed=None) -> float:
    """Generalised AMS estimator (Brehier, Lelievre & Rousset 2016) of the
    probability that the event maximum reaches the level: every trajectory the
    run has seen counts with its weight over N.  The final ensemble's weight is
    prod_j (1 - |K_j|/N) = e^{log_weight}; killed = (log weights before each
    kill, event maxima of the killed trajectories) adds those killed at
    iteration j with weight prod_{i<j} (1 - |K_i|/N).  With the event's own
    observable as the score no killed trajectory reaches a level above the
    last killed one, and the final ensemble alone gives the estimate."""
    maxima = np.asarray(maxima, dtype=np.float64)
    n = len(maxima)
    p = np.exp(log_weight) * np.sum(maxima >= level) / n
    if killed is not None:
        lw_k, mx_k = (np.asarray(a, dtype=np.float64) for a in killed)
        p += np.sum(np.exp(lw_k) * (mx_k >= level)) / n
    return float(p)


# ---------------------------------------------------------------- direct sampling (Sec. 3)
def autocorrelation(drag: np.ndarray, max_lag: int):
    """C(tau) = mean f~(t + tau) f~(t) / mean f~^2 of the drag fluctuations
    f~ = f - mean (caption of Fig. pdf_drag), pooled over the rows of drag
    [clones][steps] (independent trajectories; each lag averages the products
    available inside each row).  Returns (C[0..max_lag], tau_c) with tau_c the
    first lag where C <= 0 (C(tau_c) = 0 in the paper), -1 if none."""
    d = np.asarray(drag, dtype=np.float64)
    d = d.reshape(1, -1) if d.ndim == 1 else d
    n, length = d.shape
    mu = d.mean()
    x = d - mu
    var = np.mean(x * x)
    c = np.zeros(max_lag + 1)
    for tau in range(max_lag + 1):
        c[tau] = np.mean(x[:, tau:] * x[:, :length - tau]) / var
    below = np.nonzero(c <= 0.0)[0]
    return c, int(below[0]) if below.size else -1


def return_times(drag: np.ndarray, levels, gap: int):
    """Waiting-time return times of Sec. 3 from drag [clones][steps]: an
    event of level a starts where the series crosses from below a to >= a,
    unless it was >= a within the last `gap` steps (the same fluctuation);
    r(a) = observed steps / number of events, i.e. the mean waiting time
    between events.  Returns (events[len(levels)], r[len(levels)]), r = inf
    without events."""
    d = np.asarray(drag, dtype=np.float64)
    d = d.reshape(1, -1) if d.ndim == 1 else d
    n, length = d.shape
    events = np.zeros(len(levels), dtype=np.int64)
    for j, a in enumerate(levels):
        for row in d:
            last_above = None
            for t in range(length):
                if row[t] >= a:
                    if t > 0 and row[t - 1] < a and (last_above is None or t - last_above > gap):
                        events[j] += 1
                    last_above = t
    r = np.where(events > 0, n * length / np.maximum(events, 1), np.inf)
    return events, r
