"""ctypes binding of liblbmrare (include/lbmrare.h): argument marshalling only.

Every function keeps the C name and argument order.  Device pointers are
passed as torch CUDA tensors (checked for device, dtype and contiguity), host
arrays as numpy arrays; errors raise ``LbmError`` carrying the status and the
library's message.  The library must have been built (``build.build()``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBM_ERR_OOM, LBM_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
LBM_FP32, LBM_FP16_SHIFTED, LBM_BF16_SHIFTED = 0, 1, 2
STORAGE = {"fp32": LBM_FP32, "fp16": LBM_FP16_SHIFTED, "bf16": LBM_BF16_SHIFTED}
STORAGE_NAMES = tuple(STORAGE)

EXPORTS = [
    "lbm_last_error", "lbm_launch_count", "lbm_ensemble_create", "lbm_ensemble_destroy", "lbm_ensemble_step",
    "lbm_ensemble_step_clones", "lbm_ensemble_time", "lbm_ensemble_drag", "lbm_ensemble_window_sum", "lbm_ensemble_set_drag",
    "lbm_ensemble_scores", "lbm_ensemble_first_crossing", "lbm_ensemble_set_snapshots", "lbm_ensemble_clone",
    "lbm_ensemble_branch", "lbm_ensemble_moments", "lbm_ensemble_get_populations",
    "lbm_ensemble_set_populations", "lbm_ensemble_autotune", "lbm_ensemble_set_variant",
    "lbm_step_variant_info", "lbm_step_variant_count", "lbm_ensemble_set_timing", "lbm_ensemble_kernel_time",
    "lbm_ensemble_set_graphs", "lbm_step_variant_kind", "cnn_set_conv_path", "cnn_status", "cnn_tensor_core_paths",
    "lbm_drag_autocorrelation", "lbm_drag_return_times",
    "gktl_weights", "gktl_select", "ams_select", "lbm_step_noalloc",
    "lbm_gktl_run", "gktl_probability", "lbm_ams_run", "ams_probability",
    "cnn_create", "cnn_destroy", "cnn_param_count", "cnn_get_params", "cnn_set_params", "cnn_forward",
    "cnn_gradient", "cnn_get_gradient", "cnn_adam_step", "cnn_train_step", "lbm_ensemble_fields",
    "cnn_shape", "cnn_predict", "cnn_fit", "lbm_ensemble_attach_score", "lbm_ensemble_evaluate_score",
    "lbm_ensemble_score_history", "lbm_surrogate_dataset", "lbm_ensemble_set_snapshots_from_checkpoint",
    "lbm_selftest_bounded_wait", "lbm_ensemble_perturb", "lbm_ensemble_set_observables",
    "lbm_ensemble_observables", "lbm_ensemble_save", "lbm_ensemble_load",
    "lbm_ensemble_set_perturbation",
]


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lbmrare status {status}: {message}")
        self.status = status


class lbm_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("obs_x0", C.c_int32), ("obs_y0", C.c_int32),
                ("obs_w", C.c_int32), ("obs_h", C.c_int32), ("tau", C.c_double), ("gx", C.c_double),
                ("gy", C.c_double), ("storage", C.c_int32), ("shift_exp", C.c_int32), ("max_steps", C.c_int32),
                ("ckpt_stride", C.c_int32), ("n_snapshots", C.c_int32), ("init_amp", C.c_double),
                ("collision", C.c_int32), ("omega_bulk", C.c_double), ("omega_3", C.c_double),
                ("omega_4", C.c_double), ("open_x", C.c_int32), ("u_in", C.c_double), ("grid_x0", C.c_int32),
                ("grid_w", C.c_int32), ("grid_bar", C.c_int32), ("grid_gap", C.c_int32), ("sponge_len", C.c_int32),
                ("sponge_tau", C.c_double)]


class lbm_gktl_params(C.Structure):
    _fields_ = [("period", C.c_int32), ("n_periods", C.c_int32), ("k", C.c_double), ("eps", C.c_double),
                ("seed", C.c_uint64), ("window", C.c_int32), ("kappa", C.c_double),
                ("refresh_snapshots", C.c_int32)]


class lbm_ams_params(C.Structure):
    _fields_ = [("t_a", C.c_int32), ("window", C.c_int32), ("max_iter", C.c_int32), ("level", C.c_double),
                ("eps", C.c_double), ("seed", C.c_uint64), ("score_kind", C.c_int32),
                ("refresh_snapshots", C.c_int32)]


COLLISION = {"bgk": 0, "cm": 1}


def config(nx, ny, obstacle=(0, 0, 0, 0), tau=0.6, gx=0.0, gy=0.0, storage="fp32", shift_exp=0,
           max_steps=1000, ckpt_stride=0, n_snapshots=0, init_amp=0.01, collision="bgk", omega_bulk=1.0,
           omega_3=1.0, omega_4=1.0, open_x=0, u_in=0.0, grid=(0, 0, 0, 0), sponge_len=0,
           sponge_tau=1.0) -> lbm_config:
    """collision "bgk" or "cm" (central moments: shear at 1/tau, the bulk,
    third- and fourth-order central moments at omega_bulk, omega_3, omega_4);
    open_x = 1: open channel with centreline inlet velocity u_in, entrance
    grid (x0, width, bar, gap) and a sponge over the last sponge_len columns"""
    ox0, oy0, ow, oh = obstacle
    gx0, gw, gbar, ggap = grid
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    co = COLLISION[collision] if isinstance(collision, str) else int(collision)
    return lbm_config(nx, ny, ox0, oy0, ow, oh, tau, gx, gy, st, shift_exp, max_steps, ckpt_stride,
                      n_snapshots, init_amp, co, omega_bulk, omega_3, omega_4, open_x, u_in, gx0, gw, gbar, ggap,
                      sponge_len, sponge_tau)


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load liblbmrare.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with paper_2005_09323_gb300.build.build()")
        L = C.CDLL(_build.LIB)
        i32, i64, u64, d, p = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p
        sig = {
            "lbm_last_error": ([], C.c_char_p),
            "lbm_launch_count": ([], i64),
            "lbm_ensemble_create": ([p, i32, u64, p, p], C.c_int),
            "lbm_ensemble_destroy": ([p], C.c_int),
            "lbm_ensemble_step": ([p, i32], C.c_int),
            "lbm_ensemble_step_clones": ([p, i32, p, i32], C.c_int),
            "lbm_ensemble_time": ([p, p], C.c_int),
            "lbm_ensemble_drag": ([p, i32, i32, p, i32], C.c_int),
            "lbm_ensemble_window_sum": ([p, i32, i32, d, p], C.c_int),
            "lbm_ensemble_set_drag": ([p, i32, i32, p], C.c_int),
            "lbm_ensemble_scores": ([p, i32, i32, i32, p], C.c_int),
            "lbm_ensemble_first_crossing": ([p, i32, d, p], C.c_int),
            "lbm_ensemble_set_snapshots": ([p, i32, p], C.c_int),
            "lbm_ensemble_clone": ([p, p, d, u64, u64], C.c_int),
            "lbm_ensemble_branch": ([p, i32, i32, i32, d, u64, u64], C.c_int),
            "lbm_ensemble_moments": ([p, p, p, p], C.c_int),
            "lbm_ensemble_get_populations": ([p, i32, p], C.c_int),
            "lbm_ensemble_set_populations": ([p, i32, p], C.c_int),
            "lbm_ensemble_save": ([p, p, u64, p], C.c_int),
            "lbm_ensemble_load": ([p, p, u64], C.c_int),
            "lbm_ensemble_set_perturbation": ([p, i32], C.c_int),
            "lbm_ensemble_autotune": ([p, p], C.c_int),
            "lbm_ensemble_set_variant": ([p, i32], C.c_int),
            "lbm_step_variant_info": ([i32, p, p, p], C.c_int),
            "lbm_step_variant_count": ([], i32),
            "lbm_step_variant_kind": ([i32], i32),
            "lbm_ensemble_set_timing": ([p, i32], C.c_int),
            "lbm_ensemble_set_graphs": ([p, i32], C.c_int),
            "lbm_ensemble_kernel_time": ([p, p, p, i32], C.c_int),
            "gktl_weights": ([i32, p, p, p, p], C.c_int),
            "gktl_select": ([i32, p, u64, u64, p, p, p], C.c_int),
            "ams_select": ([i32, p, u64, u64, p, p, p, p, p], C.c_int),
            "lbm_step_noalloc": ([p, i32, p, p, p, p], C.c_int),
            "lbm_gktl_run": ([p, p, p, p, p, p, p], C.c_int),
            "gktl_probability": ([i32, d, p, i32, p, p, p, i32, p, d, d, p, p, p], C.c_int),
            "lbm_ams_run": ([p, p, p, p, p, p, p, p], C.c_int),
            "ams_probability": ([i32, d, p, i32, p, p, i32, p, p, p], C.c_int),
            "cnn_create": ([i32, i32, i32, u64, p], C.c_int),
            "cnn_destroy": ([p], C.c_int),
            "cnn_param_count": ([p], i64),
            "cnn_get_params": ([p, p], C.c_int),
            "cnn_set_params": ([p, p], C.c_int),
            "cnn_forward": ([p, p, i32, p, p], C.c_int),
            "cnn_gradient": ([p, p, p, i32, p, p], C.c_int),
            "cnn_get_gradient": ([p, p], C.c_int),
            "cnn_adam_step": ([p, C.c_float, C.c_float, C.c_float, C.c_float, p], C.c_int),
            "cnn_train_step": ([p, p, p, i32, C.c_float, p, p], C.c_int),
            "lbm_ensemble_fields": ([p, p, i32, i32, C.c_float, C.c_float, p], C.c_int),
            "cnn_shape": ([p, p, p, p], C.c_int),
            "cnn_set_conv_path": ([p, i32], C.c_int),
            "lbm_drag_autocorrelation": ([p, i32, i32, i32, p, p], C.c_int),
            "lbm_drag_return_times": ([p, i32, i32, i32, p, i32, p, p], C.c_int),
            "lbm_ensemble_perturb": ([p, i32, p, d, u64, u64], C.c_int),
            "lbm_ensemble_set_observables": ([p, i32], C.c_int),
            "lbm_ensemble_observables": ([p, i32, i32, p, i32], C.c_int),
            "cnn_status": ([p, p], C.c_int),
            "cnn_tensor_core_paths": ([p, i32, p, p], C.c_int),
            "cnn_predict": ([p, p, i64, p, p], C.c_int),
            "cnn_fit": ([p, p, p, i64, i32, i32, C.c_float, u64, p, p], C.c_int),
            "lbm_ensemble_attach_score": ([p, p, i32, C.c_float, C.c_float], C.c_int),
            "lbm_ensemble_evaluate_score": ([p, p], C.c_int),
            "lbm_ensemble_score_history": ([p, p], C.c_int),
            "lbm_surrogate_dataset": ([p, i32, i32, i32, i32, C.c_float, C.c_float, p, p, p, p], C.c_int),
            "lbm_ensemble_set_snapshots_from_checkpoint": ([p, i32, p, i32], C.c_int),
            "lbm_selftest_bounded_wait": ([i64, p, p], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != LBM_OK:
        raise LbmError(rc, lib().lbm_last_error().decode())


def _dev(t, dtype):
    """device pointer of a contiguous torch CUDA tensor of the given dtype (None -> NULL)"""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a torch CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _host(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def lbm_launch_count() -> int:
    return lib().lbm_launch_count()


# ---------------------------------------------------------------- ensemble
def lbm_ensemble_create(cfg: lbm_config, n_clones: int, seed: int, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().lbm_ensemble_create(C.byref(cfg), n_clones, seed, _stream(stream), C.byref(h)))
    return h


def lbm_ensemble_destroy(e):
    _check(lib().lbm_ensemble_destroy(e))


def lbm_ensemble_step(e, n_steps: int):
    _check(lib().lbm_ensemble_step(e, n_steps))


def lbm_ensemble_step_clones(e, n_steps: int, clones):
    a = np.ascontiguousarray(clones, dtype=np.int32)
    _check(lib().lbm_ensemble_step_clones(e, n_steps, _host(a), len(a)))


def lbm_ensemble_time(e, n: int) -> np.ndarray:
    t = np.zeros(n, dtype=np.int32)
    _check(lib().lbm_ensemble_time(e, _host(t)))
    return t


def lbm_ensemble_set_perturbation(e, centred: bool):
    """App. D coefficients: uniform in [0, 1) (False, as printed) or centred (True)"""
    _check(lib().lbm_ensemble_set_perturbation(e, 1 if centred else 0))


def lbm_ensemble_perturb(e, clones, eps: float, seed: int, it: int):
    a = np.ascontiguousarray(clones, dtype=np.int32)
    _check(lib().lbm_ensemble_perturb(e, len(a), _host(a), eps, seed, it))


def lbm_ensemble_set_observables(e, enable: bool):
    _check(lib().lbm_ensemble_set_observables(e, 1 if enable else 0))


def lbm_ensemble_observables(e, t0: int, t1: int, dst):
    """dst: numpy float64 [N, t1-t0, 4] (host, waits) or torch float64 CUDA tensor (enqueued):
    p_fb, p_base, gamma_top, gamma_bottom after each step."""
    if isinstance(dst, np.ndarray):
        if dst.dtype != np.float64 or not dst.flags.c_contiguous:
            raise TypeError("dst must be a contiguous float64 array")
        _check(lib().lbm_ensemble_observables(e, t0, t1, _host(dst), 0))
    else:
        import torch
        _check(lib().lbm_ensemble_observables(e, t0, t1, _dev(dst, torch.float64), 1))


def lbm_ensemble_drag(e, t0: int, t1: int, dst):
    """dst: numpy float64 [N, t1-t0] (host, waits) or torch float64 CUDA tensor (enqueued)."""
    if isinstance(dst, np.ndarray):
        if dst.dtype != np.float64 or not dst.flags.c_contiguous:
            raise TypeError("dst must be a contiguous float64 array")
        _check(lib().lbm_ensemble_drag(e, t0, t1, _host(dst), 0))
    else:
        import torch
        _check(lib().lbm_ensemble_drag(e, t0, t1, _dev(dst, torch.float64), 1))
    return dst


def lbm_ensemble_set_drag(e, t0: int, t1: int, src: np.ndarray):
    """overwrite the drag history of steps t0 < t <= t1 with src [N, t1 - t0] (waits)"""
    a = np.ascontiguousarray(src, dtype=np.float64)
    _check(lib().lbm_ensemble_set_drag(e, t0, t1, _host(a)))


def lbm_ensemble_window_sum(e, t0: int, t1: int, k: float, out_dev):
    import torch
    _check(lib().lbm_ensemble_window_sum(e, t0, t1, k, _dev(out_dev, torch.float64)))


def lbm_ensemble_scores(e, window: int, t_begin: int, t_end: int, out_dev=None):
    import torch
    _check(lib().lbm_ensemble_scores(e, window, t_begin, t_end, _dev(out_dev, torch.float64)))


def lbm_ensemble_first_crossing(e, clone: int, level: float) -> int:
    t = C.c_int32()
    _check(lib().lbm_ensemble_first_crossing(e, clone, level, C.byref(t)))
    return t.value


def lbm_ensemble_set_snapshots(e, clones):
    a = np.ascontiguousarray(clones, dtype=np.int32)
    _check(lib().lbm_ensemble_set_snapshots(e, len(a), _host(a)))


def lbm_ensemble_set_snapshots_from_checkpoint(e, clones, k: int):
    a = np.ascontiguousarray(clones, dtype=np.int32)
    _check(lib().lbm_ensemble_set_snapshots_from_checkpoint(e, len(a), _host(a), k))


def lbm_ensemble_clone(e, parent_dev, eps: float, seed: int, it: int):
    import torch
    _check(lib().lbm_ensemble_clone(e, _dev(parent_dev, torch.int32), eps, seed, it))


def lbm_ensemble_branch(e, dst: int, src: int, t_b: int, eps: float, seed: int, it: int):
    _check(lib().lbm_ensemble_branch(e, dst, src, t_b, eps, seed, it))


def lbm_ensemble_moments(e, n: int):
    m = np.zeros(n); px = np.zeros(n); py = np.zeros(n)
    _check(lib().lbm_ensemble_moments(e, _host(m), _host(px), _host(py)))
    return m, px, py


def lbm_ensemble_get_populations(e, clone: int, nx: int, ny: int) -> np.ndarray:
    f = np.zeros((9, ny, nx))
    _check(lib().lbm_ensemble_get_populations(e, clone, _host(f)))
    return f


def lbm_ensemble_set_populations(e, clone: int, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(lib().lbm_ensemble_set_populations(e, clone, _host(f)))


def lbm_ensemble_save(e) -> bytes:
    """The ensemble's run state as a byte string (lbm_ensemble_save)."""
    n = C.c_uint64(0)
    _check(lib().lbm_ensemble_save(e, None, 0, C.byref(n)))
    buf = C.create_string_buffer(max(n.value, 1))
    _check(lib().lbm_ensemble_save(e, buf, n.value, C.byref(n)))
    return buf.raw[:n.value]


def lbm_ensemble_load(e, state: bytes):
    """Overwrite the ensemble with a state from lbm_ensemble_save."""
    state = bytes(state)
    _check(lib().lbm_ensemble_load(e, state, len(state)))


def lbm_ensemble_autotune(e) -> int:
    v = C.c_int32()
    _check(lib().lbm_ensemble_autotune(e, C.byref(v)))
    return v.value


def lbm_ensemble_set_variant(e, variant: int):
    _check(lib().lbm_ensemble_set_variant(e, variant))


def lbm_step_variant_count() -> int:
    return lib().lbm_step_variant_count()


def lbm_step_variant_kind(variant: int) -> int:
    k = lib().lbm_step_variant_kind(variant)
    if k < 0:
        _check(k)
    return k


def lbm_step_variant_info(variant: int):
    s, v, w = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().lbm_step_variant_info(variant, C.byref(s), C.byref(v), C.byref(w)))
    return s.value, v.value, w.value


def lbm_ensemble_set_timing(e, enable: bool):
    _check(lib().lbm_ensemble_set_timing(e, int(bool(enable))))


def lbm_ensemble_set_graphs(e, enable: bool):
    _check(lib().lbm_ensemble_set_graphs(e, int(bool(enable))))


def lbm_selftest_bounded_wait(spins: int, stream=None) -> int:
    st = C.c_int32(0)
    _check(lib().lbm_selftest_bounded_wait(spins, _stream(stream), C.byref(st)))
    return st.value


def lbm_ensemble_kernel_time(e, reset: bool = False):
    ms = C.c_double()
    n = C.c_int64()
    _check(lib().lbm_ensemble_kernel_time(e, C.byref(ms), C.byref(n), int(bool(reset))))
    return ms.value, n.value


# ---------------------------------------------------------------- drivers
def lbm_gktl_run(e, period: int, n_periods: int, k: float, eps: float, seed: int, window: int,
                 logR_dev, parent_dev, integral_dev=None, maxima_dev=None, kappa: float = 0.0, correction_dev=None,
                 refresh_snapshots: bool = False):
    import torch
    prm = lbm_gktl_params(period, n_periods, k, eps, seed, window, kappa, int(refresh_snapshots))
    _check(lib().lbm_gktl_run(e, C.byref(prm), _dev(logR_dev, torch.float64), _dev(parent_dev, torch.int32),
                              _dev(integral_dev, torch.float64), _dev(maxima_dev, torch.float64),
                              _dev(correction_dev, torch.float64)))


def gktl_probability(k: float, logR_dev, integral_dev, maxima_dev, levels_dev, t_a: float, t_window: float,
                     p_dev, r_dev=None, stream=None, correction_dev=None):
    import torch
    _check(lib().gktl_probability(integral_dev.numel(), k, _dev(logR_dev, torch.float64), logR_dev.numel(),
                                  _dev(integral_dev, torch.float64), _dev(maxima_dev, torch.float64),
                                  _dev(correction_dev, torch.float64), levels_dev.numel(),
                                  _dev(levels_dev, torch.float64), t_a, t_window,
                                  _dev(p_dev, torch.float64), _dev(r_dev, torch.float64), _stream(stream)))


def lbm_ams_run(e, t_a: int, window: int, max_iter: int, level: float, eps: float, seed: int, Q_dev,
                with_kills: bool = False, score_kind: int = 0, refresh_snapshots: bool = False,
                with_records: bool = False):
    """returns (iterations, log_weight, levels z_1..z_iterations[, kills per
    iteration][, killed records (log weights before each kill, event maxima)])"""
    import torch
    prm = lbm_ams_params(t_a, window, max_iter, level, eps, seed, score_kind, int(refresh_snapshots))
    it = C.c_int32()
    lw = C.c_double()
    n = Q_dev.numel()
    levels = np.zeros(max(max_iter, 1))
    kills = np.zeros(max(max_iter, 1), dtype=np.int32)
    kmax = np.full(max(max_iter, 1) * n, np.nan) if with_records else None
    _check(lib().lbm_ams_run(e, C.byref(prm), C.byref(it), C.byref(lw), _dev(Q_dev, torch.float64), _host(levels),
                             _host(kills), _host(kmax) if with_records else None))
    out = (it.value, lw.value, levels[:it.value].copy())
    if with_kills:
        out = out + (kills[:it.value].copy(),)
    if with_records:
        rec_lw, rec_mx, w = [], [], 0.0
        for j in range(it.value):
            for i in range(kills[j]):
                rec_lw.append(w)
                rec_mx.append(kmax[j * n + i])
            w += np.log1p(-kills[j] / n)
        out = out + ((np.array(rec_lw), np.array(rec_mx)),)
    return out


def lbm_drag_autocorrelation(e, t0: int, t1: int, max_lag: int, c_dev):
    """C(tau) into c_dev (float64 CUDA tensor, max_lag + 1); returns tau_c"""
    import torch
    tc = C.c_int32()
    _check(lib().lbm_drag_autocorrelation(e, t0, t1, max_lag, _dev(c_dev, torch.float64), C.byref(tc)))
    return tc.value


def lbm_drag_return_times(e, t0: int, t1: int, levels_dev, gap: int):
    """returns (events[n_levels] int64, r[n_levels] float64) for the levels of levels_dev"""
    import torch
    n = levels_dev.numel()
    ev = np.zeros(n, dtype=np.int64)
    r = np.zeros(n)
    _check(lib().lbm_drag_return_times(e, t0, t1, n, _dev(levels_dev, torch.float64), gap, _host(ev), _host(r)))
    return ev, r


def ams_probability(log_weight: float, Q_dev, levels_dev, p_dev, records=None, stream=None):
    """records: None (final ensemble only) or (log weights, event maxima) of the
    killed trajectories, float64 CUDA tensors of one length"""
    import torch
    nr = 0 if records is None else records[0].numel()
    if records is not None and records[1].numel() != nr:
        raise TypeError("killed records: log weights and maxima differ in length")
    rl = None if records is None else _dev(records[0], torch.float64)
    rm = None if records is None else _dev(records[1], torch.float64)
    _check(lib().ams_probability(Q_dev.numel(), log_weight, _dev(Q_dev, torch.float64), nr, rl, rm,
                                 levels_dev.numel(), _dev(levels_dev, torch.float64), _dev(p_dev, torch.float64),
                                 _stream(stream)))


# ---------------------------------------------------------------- learned score
CNN_LAYER_K = (80, 304, 304, 304)   # padded columns of each conv layer's weight matrix
CNN_LAYER_CIN = (8, 32, 32, 32)


_cnn_shapes: dict = {}   # handle -> (height, width, max_batch), to check tensor shapes before a launch


def cnn_create(height: int, width: int, max_batch: int, seed: int):
    h = C.c_void_p()
    _check(lib().cnn_create(height, width, max_batch, seed, C.byref(h)))
    _cnn_shapes[h.value] = (height, width, max_batch)
    return h


def cnn_destroy(m):
    _cnn_shapes.pop(m.value, None)
    _check(lib().cnn_destroy(m))


def _cnn_input(m, x):
    ptr = _bf16_input(x)
    H, W, mb = _cnn_shapes[m.value]
    if tuple(x.shape[1:3]) != (H, W):
        raise TypeError(f"network input is {tuple(x.shape)}, the model takes [B][{H}][{W}][8]")
    return ptr


def cnn_param_count(m) -> int:
    return lib().cnn_param_count(m)


def cnn_get_params(m) -> np.ndarray:
    a = np.zeros(cnn_param_count(m), dtype=np.float32)
    _check(lib().cnn_get_params(m, _host(a)))
    return a


def cnn_set_params(m, params: np.ndarray):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != cnn_param_count(m):
        raise ValueError("parameter vector has the wrong length")
    _check(lib().cnn_set_params(m, _host(a)))


def _bf16_input(x):
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.bfloat16 or not x.is_contiguous():
        raise TypeError("network input must be a contiguous bfloat16 CUDA tensor [B][H][W][8]")
    if x.dim() != 4 or x.shape[3] != 8:
        raise TypeError("network input must have shape [B][H][W][8]")
    return C.c_void_p(x.data_ptr())


def _need(t, n, what):
    if t.numel() < n:
        raise TypeError(f"{what} holds {t.numel()} values, needs {n}")


def cnn_forward(m, x_dev, pred_dev, stream=None):
    import torch
    ptr = _cnn_input(m, x_dev)
    _need(pred_dev, x_dev.shape[0], "pred_dev")
    _check(lib().cnn_forward(m, ptr, x_dev.shape[0], _dev(pred_dev, torch.float32), _stream(stream)))


def cnn_gradient(m, x_dev, y_dev, loss_dev=None, stream=None):
    import torch
    ptr = _cnn_input(m, x_dev)
    _need(y_dev, x_dev.shape[0], "y_dev")
    _check(lib().cnn_gradient(m, ptr, _dev(y_dev, torch.float32), x_dev.shape[0],
                              _dev(loss_dev, torch.float32), _stream(stream)))


def cnn_get_gradient(m) -> np.ndarray:
    a = np.zeros(cnn_param_count(m), dtype=np.float32)
    _check(lib().cnn_get_gradient(m, _host(a)))
    return a


def cnn_adam_step(m, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().cnn_adam_step(m, lr, beta1, beta2, eps, _stream(stream)))


def cnn_train_step(m, x_dev, y_dev, lr: float, loss_dev=None, stream=None):
    import torch
    ptr = _cnn_input(m, x_dev)
    _need(y_dev, x_dev.shape[0], "y_dev")
    _check(lib().cnn_train_step(m, ptr, _dev(y_dev, torch.float32), x_dev.shape[0], lr,
                                _dev(loss_dev, torch.float32), _stream(stream)))


def lbm_ensemble_fields(e, clones, factor: int, rho_scale: float, u_scale: float, dst_dev, nx: int, ny: int):
    """dst_dev: bfloat16 CUDA tensor [len(clones)][ny/factor][nx/factor][8]"""
    a = np.ascontiguousarray(clones, dtype=np.int32)
    ptr = _bf16_input(dst_dev)
    if factor < 1 or factor > min(nx, ny):
        raise ValueError("factor must be in [1, min(nx, ny)]")
    if tuple(dst_dev.shape) != (len(a), ny // factor, nx // factor, 8):
        raise TypeError(f"dst_dev is {tuple(dst_dev.shape)}, needs {(len(a), ny // factor, nx // factor, 8)}")
    _check(lib().lbm_ensemble_fields(e, _host(a), len(a), factor, rho_scale, u_scale, ptr))


def cnn_shape(m):
    h, w, b = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().cnn_shape(m, C.byref(h), C.byref(w), C.byref(b)))
    return h.value, w.value, b.value


def cnn_set_conv_path(m, path: int):
    _check(lib().cnn_set_conv_path(m, int(path)))


def cnn_status(m, stream=None):
    _check(lib().cnn_status(m, _stream(stream)))


def cnn_tensor_core_paths(m, batch: int):
    """(hidden convolutions on tcgen05, their weight gradient on tcgen05) for a batch"""
    a, b = C.c_int32(), C.c_int32()
    _check(lib().cnn_tensor_core_paths(m, batch, C.byref(a), C.byref(b)))
    return bool(a.value), bool(b.value)


def cnn_predict(m, x_dev, pred_dev, stream=None):
    import torch
    ptr = _cnn_input(m, x_dev)
    _need(pred_dev, x_dev.shape[0], "pred_dev")
    _check(lib().cnn_predict(m, ptr, x_dev.shape[0], _dev(pred_dev, torch.float32), _stream(stream)))


def cnn_fit(m, x_dev, y_dev, batch: int, epochs: int, lr: float, seed: int, stream=None) -> np.ndarray:
    import torch
    ptr = _cnn_input(m, x_dev)
    _need(y_dev, x_dev.shape[0], "y_dev")
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(lib().cnn_fit(m, ptr, _dev(y_dev, torch.float32), x_dev.shape[0], batch, epochs, lr, seed,
                         _host(losses), _stream(stream)))
    return losses[:epochs]


def lbm_ensemble_attach_score(e, m, factor: int, rho_scale: float, u_scale: float):
    _check(lib().lbm_ensemble_attach_score(e, m, factor, rho_scale, u_scale))


def lbm_ensemble_evaluate_score(e, out_dev):
    import torch
    _check(lib().lbm_ensemble_evaluate_score(e, _dev(out_dev, torch.float64)))


def lbm_ensemble_score_history(e, n: int, n_ckpt: int) -> np.ndarray:
    a = np.zeros((n, n_ckpt))
    _check(lib().lbm_ensemble_score_history(e, _host(a)))
    return a


def lbm_surrogate_dataset(e, n_snaps: int, every: int, horizon: int, factor: int, rho_scale: float, u_scale: float,
                          x_dev, y_dev, n_clones: int, nx: int, ny: int):
    """returns (label_mean, label_std); x_dev [n_snaps*N][ny/f][nx/f][8] bf16, y_dev [n_snaps*N] fp32"""
    import torch
    ptr = _bf16_input(x_dev)
    if tuple(x_dev.shape) != (n_snaps * n_clones, ny // factor, nx // factor, 8):
        raise TypeError("x_dev has the wrong shape")
    _need(y_dev, n_snaps * n_clones, "y_dev")
    mu, sd = C.c_double(), C.c_double()
    _check(lib().lbm_surrogate_dataset(e, n_snaps, every, horizon, factor, rho_scale, u_scale, ptr,
                                       _dev(y_dev, torch.float32), C.byref(mu), C.byref(sd)))
    return mu.value, sd.value


# ---------------------------------------------------------------- no allocation
def lbm_step_noalloc(cfg: lbm_config, n_clones: int, f_in_dev, f_out_dev, drag_dev, stream=None):
    """One fused step over caller-owned buffers [n_clones][9][ny][pitch] (torch
    CUDA tensors of the storage dtype); drag_dev: float64 [n_clones]."""
    import torch
    want = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}.get(cfg.storage)
    need = n_clones * 9 * cfg.ny * noalloc_pitch(cfg.nx)
    for t in (f_in_dev, f_out_dev):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise TypeError("population buffers must be contiguous torch CUDA tensors")
        if want is not None and t.dtype != want:
            raise TypeError(f"population buffers of this storage are {want}, got {t.dtype}")
        _need(t, need, "population buffer")
    _need(drag_dev, n_clones, "drag_dev")
    _check(lib().lbm_step_noalloc(C.byref(cfg), n_clones, C.c_void_p(f_in_dev.data_ptr()),
                                  C.c_void_p(f_out_dev.data_ptr()), _dev(drag_dev, torch.float64), _stream(stream)))


def noalloc_pitch(nx: int) -> int:
    """row pitch (elements) of the buffers lbm_step_noalloc takes"""
    return ((nx + 255) // 256) * 256


# ---------------------------------------------------------------- selection
def gktl_weights(s_dev, W_dev, logR_dev, stream=None):
    import torch
    _check(lib().gktl_weights(s_dev.numel(), _dev(s_dev, torch.float64), _dev(W_dev, torch.float64),
                              _dev(logR_dev, torch.float64), _stream(stream)))


def gktl_select(W_dev, seed: int, it: int, parent_dev, status_dev=None, stream=None):
    import torch
    _check(lib().gktl_select(W_dev.numel(), _dev(W_dev, torch.float64), seed, it, _dev(parent_dev, torch.int32),
                             _dev(status_dev, torch.int32), _stream(stream)))


def ams_select(Q_dev, seed: int, it: int, killed_dev, n_killed_dev, survivor_dev, level_dev, stream=None):
    import torch
    _check(lib().ams_select(Q_dev.numel(), _dev(Q_dev, torch.float64), seed, it, _dev(killed_dev, torch.int32),
                            _dev(n_killed_dev, torch.int32), _dev(survivor_dev, torch.int32),
                            _dev(level_dev, torch.float64), _stream(stream)))
