"""The pins catch plausible mistakes: each case copies the oracle's C sources
(or its FP64 CNN, oracle/cnn.py, or its direct-sampling statistics in
oracle/__init__.py), plants one mistake in the copy (a dropped
factor, a wrong sign or index, a first-order formula for a second-order one,
an off-by-one), compiles or loads it on its own, and runs the existing pin
named beside it against that copy; the pin must fail.  A control copy without
a mistake passes every pin used here, so a failure comes from the planted
mistake and not from the harness."""
import os
import shutil

import pytest

from tests import test_oracle_lbm as T_lbm
from tests import test_oracle_mrt as T_mrt
from tests import test_oracle_observables as T_obs
from tests import test_oracle_open as T_open
from tests import test_oracle_rng as T_rng
from tests import test_oracle_estimators as T_est
from tests import test_oracle_select as T_sel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")


def momentum_balance(orc):
    T_lbm.test_momentum_balance_pins_drag(orc)


def equilibrium_moments(orc):
    T_lbm.test_equilibrium_moments(orc, 1.03, 0.05, -0.02)


def mean_copies(orc):
    T_sel.test_selection_mean_copies_equal_weights(orc, 4, 0.8, 40000)


def constructed_fields(orc):
    T_obs.test_constructed_fields(orc, 0.0)


def ou_normaliser(orc):
    T_sel.test_ou_gktl_normaliser_matches_scgf(orc, 1.0)


def guo_moments(orc):
    T_lbm.test_guo_source_moments(orc, 0.04, -0.03, 2e-4, -5e-4)


_DIRECT_WINDOW = []


def direct_window():
    """the brute-force tail probabilities of the estimator pins, computed once"""
    if not _DIRECT_WINDOW:
        mx = T_est.ou_direct_window_max(200000, T_est.PERIODS * T_est.STEPS_PER_PERIOD, T_est.WINDOW, T_est.DT, 2024)
        p = T_est.np.array([(mx >= a).mean() for a in T_est.LEVELS])
        _DIRECT_WINDOW.append((p, T_est.np.sqrt(p * (1 - p) / mx.size)))
    return _DIRECT_WINDOW[0]


def gktl_estimator(orc):
    T_est.test_gktl_estimator_matches_direct_sampling(orc, direct_window(), 0.5)


def gktl_potential(orc):
    T_est.test_gktl_with_potential_matches_direct_sampling(orc, direct_window())


PINS = {
    "momentum balance": momentum_balance,
    "equilibrium moments": equilibrium_moments,
    "perturbation keeps the mass": T_lbm.test_perturbation_preserves_mass,
    "GKTL weights sum to N": T_sel.test_weights_sum_to_n_and_normaliser,
    "AMS survivor uniform among the others": T_sel.test_ams_survivor_uniform,
    "inlet column": T_open.test_inlet_column_is_the_equilibrium_of_the_profile,
    "outlet column": T_open.test_outlet_column_is_regularized_with_the_extrapolated_velocity,
    "sponge profile": T_open.test_sponge_profile,
    "grid of bars": T_open.test_grid_of_bars_matches_the_stated_geometry,
    "drag counts the square only": T_open.test_drag_counts_the_square_only,
    "central moments relax at their rates": T_mrt.test_each_central_moment_relaxes_at_its_rate,
    "equal rates give BGK": T_mrt.test_equal_rates_is_bgk,
    "Philox against numpy": T_rng.test_philox_many_counters,
    "mean copies equal the weights": mean_copies,
    "observables on constructed fields": constructed_fields,
    "OU GKTL normaliser": ou_normaliser,
    "draws use their documented counters": T_rng.test_draws_of_the_method_use_their_documented_counters,
    "integer weights copied exactly": T_sel.test_integer_weights_are_copied_exactly,
    "Guo source moments": guo_moments,
    "initial state": T_lbm.test_init_is_equilibrium_with_bounded_velocity,
    "opposite shears in a symmetric flow": T_obs.test_symmetric_flow_has_opposite_shears,
    "OU AMS against direct sampling": T_sel.test_ou_ams_matches_direct_sampling,
    "GKTL estimator against direct sampling": gktl_estimator,
    "GKTL with a potential against direct sampling": gktl_potential,
    "GKTL potential bookkeeping": T_est.test_gktl_potential_bookkeeping,
    "AMS with another score against direct sampling": T_est.test_ams_estimator_with_another_score_matches_direct_sampling,
    "centred perturbation has no mean pull": T_lbm.test_centred_perturbation_has_no_mean_pull,
}

# (case, file, text in the oracle, planted text, pin that must fail)
MUTANTS = [
    ("Guo factor (1 - 1/(2 tau)) dropped", "lbm.c",
     "+ (1.0 - 1.0 / (2.0 * tau)) * S[i];", "+ S[i];", "momentum balance"),
    ("half-force velocity shift dropped", "lbm.c",
     "double ux = (jx + 0.5 * c->gx) / rho;", "double ux = jx / rho;", "momentum balance"),
    ("bounce-back into the same direction", "lbm.c",
     "fout[IDX(c, OPP[i], x, y)] = v;", "fout[IDX(c, i, x, y)] = v;", "momentum balance"),
    ("drag sign flipped", "lbm.c",
     "ox += 2.0 * CX[i] * v;", "ox -= 2.0 * CX[i] * v;", "momentum balance"),
    ("relaxation by tau instead of 1/tau", "lbm.c",
     "f[i] - (f[i] - feq[i]) / tau +", "f[i] - (f[i] - feq[i]) * tau +", "momentum balance"),
    ("equilibrium's second-order term doubled", "lbm.c",
     "quad / (2.0 * CS2 * CS2)", "quad / (CS2 * CS2)", "equilibrium moments"),
    ("perturbation not rescaled to the mass", "lbm.c",
     "double scale = m_before / m_after;", "double scale = 1.0;", "perturbation keeps the mass"),
    ("GKTL weights not scaled by N", "select.c",
     "W[i] = (double)n * exp(s[i] - m) / sum;", "W[i] = exp(s[i] - m) / sum;", "GKTL weights sum to N"),
    ("AMS survivor drawn among all, the killed included", "select.c",
     "if (Q[i] == z) continue;", "/* every index counts */", "AMS survivor uniform among the others"),
    ("inlet parabola through the node centres", "lbm.c",
     "double h = c->ny, yy = y + 0.5;", "double h = c->ny, yy = y;", "inlet column"),
    ("outlet velocity copied (first order)", "lbm.c",
     "ux[y] = 2.0 * vx[0] - vx[1];", "ux[y] = vx[0];", "outlet column"),
    ("outlet stress with the wrong sign", "lbm.c",
     "const double pre = -2.0 * CS2 * (tau_out - 1.0);", "const double pre = 2.0 * CS2 * (tau_out - 1.0);",
     "outlet column"),
    ("sponge ramp linear", "lbm.c",
     "return c->tau + (c->sponge_tau - c->tau) * s * s;", "return c->tau + (c->sponge_tau - c->tau) * s;",
     "sponge profile"),
    ("bar rows off by one", "lbm.c",
     "(y % (c->grid_bar + c->grid_gap)) >= c->grid_gap;", "(y % (c->grid_bar + c->grid_gap)) > c->grid_gap;",
     "grid of bars"),
    ("drag counts the links into the bars", "lbm.c",
     "} else if (in_obstacle(c, xn, yn)) {", "} else if (orc_is_solid(c, xn, yn)) {",
     "drag counts the square only"),
    ("k11 relaxed at the bulk rate", "lbm.c",
     "Om[5][5] = ws;", "Om[5][5] = wb;", "central moments relax at their rates"),
    ("central-moment forcing without its half step", "lbm.c",
     "d[i] = f[i] - feq[i] + 0.5 * S[i];", "d[i] = f[i] - feq[i];", "equal rates give BGK"),
    ("Philox multiplier altered", "philox.c",
     "M0 = 0xD2E7470EE14C6C93ULL", "M0 = 0xD2E7470EE14C6C95ULL", "Philox against numpy"),
    ("systematic resampling without its uniform", "select.c",
     "double point = (U + (double)k) * spacing;", "double point = (double)k * spacing;",
     "mean copies equal the weights"),
    ("wall shear from one row (first order)", "lbm.c",
     "gt += (9.0 * u1 - u2) / 3.0;", "gt += 2.0 * u1;", "observables on constructed fields"),
    ("initial velocity counter with clone and site swapped", "lbm.c",
     "uint64_t ctr[4] = {5u, (uint64_t)clone, site, 0u}", "uint64_t ctr[4] = {5u, site, (uint64_t)clone, 0u}",
     "draws use their documented counters"),
    ("App. D weight counter with iteration and slot swapped", "lbm.c",
     "uint64_t ctr[4] = {4u, iter, (uint64_t)slot, (uint64_t)n}",
     "uint64_t ctr[4] = {4u, (uint64_t)slot, iter, (uint64_t)n}", "draws use their documented counters"),
    ("AMS survivor counter with iteration and killed index swapped", "select.c",
     "stream_word(3u, seed, iter, (uint64_t)killed[k])", "stream_word(3u, seed, (uint64_t)killed[k], iter)",
     "draws use their documented counters"),
    ("extra copies placed for the parents in descending order", "select.c",
     "    for (int32_t i = 0; i < n; ++i)\n        for (int32_t e = 1; e < cnt[i]; ++e) {",
     "    for (int32_t i = n - 1; i >= 0; --i)\n        for (int32_t e = 1; e < cnt[i]; ++e) {",
     "integer weights copied exactly"),
    ("log R without the 1/N", "select.c",
     "*logR = m + log(sum / (double)n);", "*logR = m + log(sum);", "GKTL weights sum to N"),
    ("y force taken from g_x", "lbm.c",
     "double uy = (jy + 0.5 * c->gy) / rho;", "double uy = (jy + 0.5 * c->gx) / rho;", "momentum balance"),
    ("forebody pressure from the square's own column", "lbm.c",
     "node_macro(c, f, x0 - 1, y, &rho_at, &ux_at, &uy_at);", "node_macro(c, f, x0, y, &rho_at, &ux_at, &uy_at);",
     "observables on constructed fields"),
    ("central-moment bulk/shear coupling with the wrong sign", "lbm.c",
     "Om[3][4] = Om[4][3] = 0.5 * (wb - ws);", "Om[3][4] = Om[4][3] = 0.5 * (ws - wb);",
     "central moments relax at their rates"),
    ("Guo source without the -u term", "lbm.c",
     "double ax = (CX[i] - ux) / CS2 + cu * CX[i] / (CS2 * CS2);", "double ax = CX[i] / CS2 + cu * CX[i] / (CS2 * CS2);",
     "Guo source moments"),
    ("solid nodes initialised empty", "lbm.c",
     "for (int i = 0; i < 9; ++i) feq[i] = W[i];", "for (int i = 0; i < 9; ++i) feq[i] = 0.0;", "initial state"),
    ("base pressure from the square's last column", "lbm.c",
     "node_macro(c, f, x1, y, &rho_at, &ux_at, &uy_at);", "node_macro(c, f, x1 - 1, y, &rho_at, &ux_at, &uy_at);",
     "observables on constructed fields"),
    ("bottom-wall shear without its sign flip", "lbm.c",
     "gb -= (9.0 * u1 - u2) / 3.0;", "gb += (9.0 * u1 - u2) / 3.0;", "opposite shears in a symmetric flow"),
    ("forebody pressure without cs2", "lbm.c",
     "pfb += CS2 * rho_at;", "pfb += rho_at;", "observables on constructed fields"),
    ("AMS estimator without its weight", "ou.c",
     "logw += log1p(-(double)nk / (double)n);", "/* no weight */", "OU AMS against direct sampling"),
    ("AMS branch re-simulated from the start instead of the level crossing", "ou.c",
     "while (tb <= n_steps && !(ams_score_at(xs, tb, score_window) > z)) tb += stride;", "/* branch at t = 0 */",
     "OU AMS against direct sampling"),
    ("OU noise doubled in the GKTL process", "ou.c",
     "x[i] = a * x[i] + sig * orc_ou_noise(seed, (uint64_t)step, (uint64_t)i, 0u);",
     "x[i] = a * x[i] + 2.0 * sig * orc_ou_noise(seed, (uint64_t)step, (uint64_t)i, 0u);", "OU GKTL normaliser"),
    ("potential's start value not carried through the genealogy", "ou.c",
     "v0n[i] = v0[parent[i]];", "v0n[i] = v0[i];", "GKTL potential bookkeeping"),
    ("potential added with the wrong sign", "ou.c",
     "s[i] = k * acc + kappa * (x[i] - vprev[i]);", "s[i] = k * acc - kappa * (x[i] - vprev[i]);",
     "GKTL with a potential against direct sampling"),
    ("potential's previous value left at the start", "ou.c",
     "memcpy(vprev, xn, sizeof(double) * n);", "/* vprev kept */", "GKTL with a potential against direct sampling"),
    ("AMS killed trajectories left out of the estimate", "ou.c",
     "if (mk >= alev) p_killed += exp(logw) / (double)n;", "/* killed left out */",
     "AMS with another score against direct sampling"),
]


def build_copy(orc, tmp, file=None, old=None, new=None):
    src = os.path.join(tmp, "src")
    os.makedirs(src)
    for f in os.listdir(ORACLE):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(ORACLE, f), src)
    if file is not None:
        path = os.path.join(src, file)
        text = open(path).read()
        assert text.count(old) == 1, f"the oracle no longer holds {old!r} once: update this case"
        with open(path, "w") as fh:
            fh.write(text.replace(old, new))
    # references between the copy's own functions bind inside the copy
    return orc.compile_sources(src, os.path.join(tmp, "liboracle_copy.so"), extra=("-Wl,-Bsymbolic",))


def test_control_copy_passes_every_pin(orc, tmp_path):
    lib = build_copy(orc, str(tmp_path))
    with orc.using(lib):
        for pin in PINS.values():
            pin(orc)


@pytest.mark.parametrize("case,file,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(orc, tmp_path, case, file, old, new, pin):
    lib = build_copy(orc, str(tmp_path), file, old, new)
    with orc.using(lib):
        with pytest.raises(AssertionError):
            PINS[pin](orc)


# ---------------------------------------------------------------- the FP64 CNN (oracle/cnn.py)
from tests import test_oracle_cnn as T_cnn  # noqa: E402

CNN_PINS = {
    "identity kernel and shift": lambda: T_cnn.test_conv_identity_kernel_and_shift(),
    "gradient by central differences": lambda: T_cnn.test_gradient_by_central_differences(0),
    "Adam's first step": lambda: T_cnn.test_adam_first_step_moves_by_lr(),
    "block means on a ragged lattice": lambda: T_cnn.test_fields_block_means_on_ragged_lattices(13, 10, 4),
}

CNN_MUTANTS = [
    ("kernel flipped (convolution for correlation)",
     'out += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])',
     'out += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, 2 - ky, 2 - kx, :])',
     "identity kernel and shift"),
    ("input gradient without the tap's shift",
     "dxp[:, ky:ky + H, kx:kx + W, :] +=", "dxp[:, 1:1 + H, 1:1 + W, :] +=", "gradient by central differences"),
    ("weight gradient with transposed taps",
     "dw[:, ky, kx, :] = np.einsum", "dw[:, kx, ky, :] = np.einsum", "gradient by central differences"),
    ("ReLU derivative taken as 1 everywhere",
     "dpre = store(da * (acts[l + 1] > 0))", "dpre = store(da * (acts[l + 1] >= 0))",
     "gradient by central differences"),
    ("mean pool over the rows only",
     "P = acts[-1].shape[1] * acts[-1].shape[2]", "P = acts[-1].shape[1]", "gradient by central differences"),
    ("Adam without bias correction",
     "mh = self.m / (1 - self.b1 ** self.t)", "mh = self.m", "Adam's first step"),
    ("blocks cropped from the far corner",
     "a[:H * factor, :W * factor]", "a[-H * factor:, -W * factor:]", "block means on a ragged lattice"),
]


def cnn_copy(old=None, new=None):
    import types
    src = open(os.path.join(ORACLE, "cnn.py")).read()
    if old is not None:
        assert src.count(old) == 1, f"oracle/cnn.py no longer holds {old!r} once: update this case"
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_cnn_copy")
    exec(compile(src, "oracle/cnn.py (copy)", "exec"), mod.__dict__)
    return mod


def test_cnn_control_copy_passes_every_pin(orc, monkeypatch):
    monkeypatch.setattr(T_cnn, "cnn", cnn_copy())
    for pin in CNN_PINS.values():
        pin()


@pytest.mark.parametrize("case,old,new,pin", CNN_MUTANTS, ids=[m[0] for m in CNN_MUTANTS])
def test_cnn_pin_catches_planted_mistake(orc, monkeypatch, case, old, new, pin):
    monkeypatch.setattr(T_cnn, "cnn", cnn_copy(old, new))
    with pytest.raises(AssertionError):
        CNN_PINS[pin]()


# ---------------------------------------------------------------- direct-sampling statistics (oracle/__init__.py)
from tests import test_oracle_direct as T_dir  # noqa: E402

DIRECT_PINS = {
    "autocorrelation small cases": T_dir.test_autocorrelation_small_cases,
    "return times hand counted": T_dir.test_return_times_hand_counted,
    "AR(1) up-crossings": T_dir.test_return_time_of_ar1_matches_the_upcrossing_probability,
}

DIRECT_MUTANTS = [
    ("mean not removed", "    x = d - mu\n", "    x = d\n", "autocorrelation small cases"),
    ("lag products averaged over the whole length",
     "c[tau] = np.mean(x[:, tau:] * x[:, :length - tau]) / var",
     "c[tau] = np.sum(x[:, tau:] * x[:, :length - tau]) / x.size / var", "autocorrelation small cases"),
    ("observed time of one trajectory only",
     "r = np.where(events > 0, n * length / np.maximum(events, 1), np.inf)",
     "r = np.where(events > 0, length / np.maximum(events, 1), np.inf)", "AR(1) up-crossings"),
    ("same-fluctuation gap inclusive",
     "t - last_above > gap", "t - last_above >= gap", "return times hand counted"),
    ("a series starting above the level counts an event",
     "if t > 0 and row[t - 1] < a", "if (t == 0 or row[t - 1] < a)", "return times hand counted"),
]


def oracle_copy(old=None, new=None):
    import types
    path = os.path.join(ORACLE, "__init__.py")
    src = open(path).read()
    if old is not None:
        assert src.count(old) == 1, f"oracle/__init__.py no longer holds {old!r} once: update this case"
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_copy")
    mod.__file__ = path  # the copy finds the compiled library beside the original
    exec(compile(src, "oracle/__init__.py (copy)", "exec"), mod.__dict__)
    return mod


def test_direct_statistics_control_copy_passes_every_pin(orc):
    copy = oracle_copy()
    for pin in DIRECT_PINS.values():
        pin(copy)


@pytest.mark.parametrize("case,old,new,pin", DIRECT_MUTANTS, ids=[m[0] for m in DIRECT_MUTANTS])
def test_direct_statistics_pin_catches_planted_mistake(orc, case, old, new, pin):
    copy = oracle_copy(old, new)
    with pytest.raises(AssertionError):
        DIRECT_PINS[pin](copy)


# ---------------------------------------------------------------- estimator helpers (oracle/__init__.py)
ESTIMATOR_PINS = {
    "window sum hand computed": T_est.test_window_sum_hand_computed,
    "trailing mean max hand computed": T_est.test_trailing_mean_max_hand_computed,
    "return time of a Poisson process": T_est.test_return_time_of_a_poisson_process,
    "GKTL estimator against direct sampling": gktl_estimator,
    "GKTL with a potential against direct sampling": gktl_potential,
    "AMS estimator hand computed": T_est.test_ams_probability_hand_computed,
    "AMS with another score against direct sampling": T_est.test_ams_estimator_with_another_score_matches_direct_sampling,
    "centred perturbation has no mean pull": T_lbm.test_centred_perturbation_has_no_mean_pull,
}

ESTIMATOR_MUTANTS = [
    ("GKTL exponent's sign flipped (the printed e^{+kI})",
     "w = np.exp(log_z - k * integrals - corr)", "w = np.exp(log_z + k * integrals - corr)",
     "GKTL estimator against direct sampling"),
    ("potential's correction left out",
     "w = np.exp(log_z - k * integrals - corr)", "w = np.exp(log_z - k * integrals)",
     "GKTL with a potential against direct sampling"),
    ("time-averaged drag window one step late",
     "sliding_window_view(d[:, t_begin:t_end], window, axis=1)",
     "sliding_window_view(d[:, t_begin + 1:t_end + 1], window, axis=1)", "trailing mean max hand computed"),
    ("time-averaged drag window one step early",
     "sliding_window_view(d[:, t_begin:t_end], window, axis=1)",
     "sliding_window_view(d[:, max(t_begin - 1, 0):t_end - 1], window, axis=1)", "trailing mean max hand computed"),
    ("GKTL window sum one step late",
     "return k * np.sum(np.asarray(drag, dtype=np.float64)[:, t0:t1], axis=1)",
     "return k * np.sum(np.asarray(drag, dtype=np.float64)[:, t0 + 1:t1 + 1], axis=1)", "window sum hand computed"),
    ("return time over T_a instead of T_a - T",
     "return -(t_a - t_window) / np.log1p(-p)", "return -t_a / np.log1p(-p)", "return time of a Poisson process"),
    ("return time to first order in P",
     "return -(t_a - t_window) / np.log1p(-p)", "return (t_a - t_window) / p", "return time of a Poisson process"),
    ("AMS estimator without its weight",
     "p = np.exp(log_weight) * np.sum(maxima >= level) / n", "p = np.sum(maxima >= level) / n",
     "AMS estimator hand computed"),
    ("AMS killed records left out",
     "p += np.sum(np.exp(lw_k) * (mx_k >= level)) / n", "p += 0.0",
     "AMS with another score against direct sampling"),
    ("centred App. D coefficients left uncentred",
     "return a - 0.5 if centred else a", "return a if centred else a", "centred perturbation has no mean pull"),
    ("centred App. D coefficients shifted by a quarter",
     "return a - 0.5 if centred else a", "return a - 0.25 if centred else a", "centred perturbation has no mean pull"),
]


def test_estimator_control_copy_passes_every_pin(orc):
    copy = oracle_copy()
    for pin in ESTIMATOR_PINS.values():
        pin(copy)


@pytest.mark.parametrize("case,old,new,pin", ESTIMATOR_MUTANTS, ids=[m[0] for m in ESTIMATOR_MUTANTS])
def test_estimator_pin_catches_planted_mistake(orc, case, old, new, pin):
    copy = oracle_copy(old, new)
    with pytest.raises(AssertionError):
        ESTIMATOR_PINS[pin](copy)
