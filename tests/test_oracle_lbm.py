"""Pins of the oracle's D2Q9 lattice-BGK step against what App. A and the
mathematics of the scheme fix, independently of the oracle's own code."""
import os

import numpy as np
import pytest

from tests import seeded_inputs as si

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# D2Q9 velocities in the numbering used by the library and the oracle (the
# paper's lattice sketch is not legible; the numbering is a convention)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def load_golden_weights():
    vals = {}
    with open(os.path.join(GOLD, "d2q9_app_a.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(eval(v, {"__builtins__": {}}))
    return vals


def test_weights_and_sound_speed_from_paper(orc):
    g = load_golden_weights()
    w = orc.feq(1.0, 0.0, 0.0)  # rest equilibrium is the weight vector
    assert w[0] == g["w0"]
    assert np.all(w[1:5] == g["w_axis"])
    assert np.all(w[5:9] == g["w_diag"])
    assert abs(w.sum() - 1.0) < 1e-15
    # isotropy: sum w c_a c_b = cs^2 delta_ab
    assert abs((w * CX * CX).sum() - g["cs2"]) < 1e-15
    assert abs((w * CX * CY).sum()) < 1e-15


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.05, -0.02), (0.97, -0.08, 0.11)])
def test_equilibrium_moments(orc, rho, ux, uy):
    """App. A: sum f^eq = rho, sum f^eq c = rho u, and the second moment of the
    second-order equilibrium is rho (cs^2 delta + u u)."""
    f = orc.feq(rho, ux, uy)
    assert abs(f.sum() - rho) < 1e-15
    assert abs((f * CX).sum() - rho * ux) < 1e-15
    assert abs((f * CY).sum() - rho * uy) < 1e-15
    assert abs((f * CX * CX).sum() - rho * (1 / 3 + ux * ux)) < 1e-15
    assert abs((f * CX * CY).sum() - rho * ux * uy) < 1e-15
    assert abs((f * CY * CY).sum() - rho * (1 / 3 + uy * uy)) < 1e-15


@pytest.mark.parametrize("ux,uy,gx,gy", [(0.0, 0.0, 1e-3, 0.0), (0.04, -0.03, 2e-4, -5e-4)])
def test_guo_source_moments(orc, ux, uy, gx, gy):
    """Guo et al. (2002): the source has zero mass, momentum F and second
    moment u_a F_b + u_b F_a."""
    S = orc.guo(ux, uy, gx, gy)
    assert abs(S.sum()) < 1e-18
    assert abs((S * CX).sum() - gx) < 1e-17
    assert abs((S * CY).sum() - gy) < 1e-17
    assert abs((S * CX * CX).sum() - 2 * ux * gx) < 1e-17
    assert abs((S * CX * CY).sum() - (ux * gy + uy * gx)) < 1e-17
    assert abs((S * CY * CY).sum() - 2 * uy * gy) < 1e-17


def test_rest_state_is_invariant(orc):
    """Fluid at rest with no force, with walls and obstacle: nothing moves."""
    c = orc.cfg(40, 24, obstacle=si.channel(40, 24, 6), tau=0.55)
    w = orc.feq(1.0, 0.0, 0.0)
    f = np.broadcast_to(w[:, None, None], (9, 24, 40)).copy()
    g, drag = orc.run(c, f, 50)
    assert np.abs(g - f).max() < 1e-15
    assert np.abs(drag).max() < 1e-15


def test_mass_conserved_2000_steps(orc):
    """256x64 channel with an 8x8 obstacle, tau = 0.52, g_x = 1e-6 and a seeded
    0.01 velocity perturbation: fluid mass is conserved to rounding.  The
    weights 4/9, 1/9, 1/36 are not exact in binary64, so the collision loses
    or gains up to a few units of 2^-53 of the mass per step: the bound is
    steps x 4 eps."""
    c = orc.cfg(256, 64, obstacle=si.channel(256, 64, 8, 64), tau=0.52, gx=1e-6)
    f0 = orc.init(c, 0, 0, 0.01)
    m0, _, _ = orc.moments(c, f0)
    f, drag = orc.run(c, f0, 2000)
    m1, _, _ = orc.moments(c, f)
    assert abs(m1 - m0) / m0 < 2000 * 4 * 2.0 ** -53
    assert np.all(np.isfinite(drag))


def test_momentum_balance_pins_drag(orc):
    """Streaming moves momentum between nodes except on bounced links, where
    2 c f leaves the fluid; collision conserves momentum and the forcing adds F
    per fluid node.  Hence P(t+1) - P(t) = N_fluid F - F_wall(t) - F_obstacle(t)
    with the forces of the state at t: this fixes the drag to rounding."""
    nx, ny = 64, 32
    c = orc.cfg(nx, ny, obstacle=si.channel(nx, ny, 8), tau=0.6, gx=2e-5, gy=-1e-5)
    n_fluid = nx * ny - 64
    f = orc.init(c, 3, 1, 0.02)
    _, fo, fw = orc.step(c, f)  # forces of the initial state come from a step of it
    fo_prev = None
    # forces of state f are those returned by the step that produced f
    f, fo_prev, fw_prev = orc.step(c, f)
    for _ in range(60):
        _, px0, py0 = orc.moments(c, f)
        g, fo, fw = orc.step(c, f)
        _, px1, py1 = orc.moments(c, g)
        assert abs((px1 - px0) - (n_fluid * c.gx - fw_prev[0] - fo_prev[0])) < 1e-12
        assert abs((py1 - py0) - (n_fluid * c.gy - fw_prev[1] - fo_prev[1])) < 1e-12
        f, fo_prev, fw_prev = g, fo, fw
    assert abs(fo_prev[0]) > 1e-6  # the test exercised a non-trivial drag


def test_drag_symmetry_reverses_with_flow(orc):
    """Mirror x -> -x of the whole state reverses the drag (obstacle centred)."""
    nx, ny = 48, 24
    c = orc.cfg(nx, ny, obstacle=(20, 8, 8, 8), tau=0.7)
    f = orc.init(c, 5, 0, 0.03)
    mirror = [0, 3, 2, 1, 4, 6, 5, 8, 7]
    # reflect about the obstacle's axis x = 23.5: column x -> 47 - x
    fm = f[mirror][:, :, ::-1].copy()
    _, d1 = orc.run(c, f, 20)
    _, d2 = orc.run(c, fm, 20)
    assert np.allclose(d1, -d2, rtol=0, atol=1e-14)


def poiseuille_slip(tau, g):
    """Wall slip of the steady force-driven channel flow for BGK with halfway
    bounce-back and Guo forcing: u_s = g (16 (tau-1/2)^2 - 3) / (24 nu).
    Derived by reducing the steady x-invariant scheme to the x-odd parts of the
    diagonal populations (see test_poiseuille_reduced_model); it vanishes for
    (tau-1/2)^2 = 3/16, the known condition for an exactly halfway wall."""
    nu = (tau - 0.5) / 3
    return g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)


def reduced_model(H, tau, g):
    """Steady x-invariant channel flow written for the odd moments only:
    a_j = f5 - f6 (upward), b_j = f8 - f7 (downward) before collision.  Their
    equilibrium part is u/6 and their Guo source g/6, the axis pair f1 - f3
    relaxes to 2u/3 + (tau - 1/2) 2g/3, so u = 3 (a + b) + g (2 tau + 1/2).
    Streaming: a_j = a*_{j-1}, b_j = b*_{j+1}; bounce-back: a_0 = -b*_0 and
    b_{H-1} = -a*_{H-1}.  A linear solve gives u_j."""
    om = 1 / tau
    kap = 1 - om / 2
    c0 = g * (2 * tau + 0.5)
    n = 2 * H
    A = np.zeros((n, n))
    r = np.zeros(n)

    def post(row, own, j, sign):
        A[row, own] -= sign * (1 - om)
        A[row, j] -= sign * om * 3 / 6
        A[row, H + j] -= sign * om * 3 / 6
        r[row] += sign * (om * c0 / 6 + kap * g / 6)

    for j in range(H):
        A[j, j] += 1
        if j >= 1:
            post(j, j - 1, j - 1, +1)
        else:
            post(j, H + 0, 0, -1)
        A[H + j, H + j] += 1
        if j <= H - 2:
            post(H + j, H + j + 1, j + 1, +1)
        else:
            post(H + j, H - 1, H - 1, -1)
    x = np.linalg.solve(A, r)
    return 3 * (x[:H] + x[H:]) + c0


def test_poiseuille_reduced_model_closed_form():
    for tau in (0.6, 0.8, 0.5 + np.sqrt(3 / 16), 1.0):
        H, g = 32, 1e-6
        nu = (tau - 0.5) / 3
        y = np.arange(H)
        exact = g / (2 * nu) * (y + 0.5) * (H - 0.5 - y) + poiseuille_slip(tau, g)
        u = reduced_model(H, tau, g)
        assert np.abs(u - exact).max() < 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_poiseuille_steady_profile(orc, tau):
    """Obstacle-free channel 4 x 32, body force g: the steady profile is the
    parabola g/(2 nu) (y+1/2)(H-1/2-y) plus the bounce-back slip, with
    nu = (tau - 1/2)/3 (App. A)."""
    H, g = 32, 1e-6
    c = orc.cfg(4, H, tau=tau, gx=g)
    w = orc.feq(1.0, 0.0, 0.0)
    f = np.broadcast_to(w[:, None, None], (9, H, 4)).copy()
    nu = (tau - 0.5) / 3
    steps = int(40 * H * H / (np.pi ** 2 * nu))
    f, _ = orc.run(c, f, steps)
    rho, ux, uy = orc.macro(c, f)
    u = ux[:, 0]
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - 0.5 - y) + poiseuille_slip(tau, g)
    assert np.abs(u - exact).max() < 1e-9 * exact.max()
    # the second difference alone fixes the viscosity
    d2 = nu * (u[2:] - 2 * u[1:-1] + u[:-2])
    assert np.abs(d2 / (-g) - 1).max() < 1e-8
    assert np.abs(uy).max() < 1e-12
    assert np.abs(ux - ux[:, :1]).max() < 1e-15


def test_init_is_equilibrium_with_bounded_velocity(orc):
    c = orc.cfg(64, 16, obstacle=si.channel(64, 16, 4), tau=0.6)
    f = orc.init(c, 11, 2, 0.01)
    rho, ux, uy = orc.macro(c, f)
    fluid = ~orc.solid_mask(c)
    assert np.abs(rho[fluid] - 1).max() < 1e-15
    assert np.abs(ux[fluid]).max() <= 0.01 and np.abs(uy[fluid]).max() <= 0.01
    assert np.abs(ux[fluid]).max() > 0.009
    # different clones and seeds draw different fields
    assert not np.array_equal(f, orc.init(c, 11, 3, 0.01))
    assert not np.array_equal(f, orc.init(c, 12, 2, 0.01))
    assert np.array_equal(f, orc.init(c, 11, 2, 0.01))
    w = orc.feq(1.0, 0.0, 0.0)
    assert np.all(f[:, ~fluid] == w[:, None])


def test_perturbation_preserves_mass(orc):
    """App. D: eq. (perturb_pop) followed by a rescale to the original mass."""
    nx, ny = 48, 16
    c = orc.cfg(nx, ny, obstacle=si.channel(nx, ny, 4), tau=0.6, gx=1e-5)
    f = orc.init(c, 1, 0, 0.01)
    snaps = np.stack([orc.init(c, 2, k, 0.01) for k in range(10)])
    alpha = orc.perturb_alphas(9, 3, 5, 10)
    assert np.all((alpha >= 0) & (alpha < 1))
    g = orc.perturb(c, f, snaps, alpha, 0.002)
    m0, _, _ = orc.moments(c, f)
    m1, _, _ = orc.moments(c, g)
    assert abs(m1 - m0) / m0 < 1e-14
    assert np.abs(g - f).max() > 1e-6
    assert np.array_equal(orc.perturb(c, f, snaps, alpha, 0.0), f)
    # the perturbation is the mass-rescaled linear combination
    fluid = ~orc.solid_mask(c)
    lin = f + 0.002 * np.tensordot(alpha, snaps, axes=1)
    scale = m0 / lin[:, fluid].sum()
    assert np.abs(g[:, fluid] - scale * lin[:, fluid]).max() < 1e-15


def test_centred_perturbation_has_no_mean_pull(orc):
    """Reading 24 (App. D): with the coefficients as eq. (perturb_pop) prints
    them (uniform in [0, 1)) the mass-rescaled perturbation moves a state on
    average by eps/2 sum_n (f^(n) - f M^(n)/M), towards the snapshots, to first
    order in eps; with centred coefficients (alpha_n - 1/2) the mean
    displacement vanishes.  Averaged over 4000 draws of the counter-based
    coefficients, against the first-order expansion written out here."""
    nx, ny = 32, 12
    c = orc.cfg(nx, ny, obstacle=si.channel(nx, ny, 4), tau=0.6, gx=1e-5)
    f = orc.init(c, 1, 0, 0.05)
    snaps = np.stack([orc.init(c, 2, k, 0.05) for k in range(10)])
    eps, K = 0.002, 4000
    fluid = ~orc.solid_mask(c)
    m0 = orc.moments(c, f)[0]
    ms = np.array([orc.moments(c, sn)[0] for sn in snaps])
    pull = 0.5 * eps * (snaps.sum(axis=0) - f * ms.sum() / m0)
    mean = {False: np.zeros_like(f), True: np.zeros_like(f)}
    for it in range(K):
        for centred in (False, True):
            a = orc.perturb_alphas(5, it, 1, 10, centred=centred)
            assert np.all((a >= -0.5) & (a < 0.5)) if centred else np.all((a >= 0) & (a < 1))
            mean[centred] += (orc.perturb(c, f, snaps, a, eps) - f) / K
    scale = np.abs(pull[:, fluid]).max()
    assert np.abs(mean[False] - pull)[:, fluid].max() < 0.05 * scale
    assert np.abs(mean[True])[:, fluid].max() < 0.05 * scale
