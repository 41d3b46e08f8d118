"""Oracle pins for the central-moment collision (the multiple-relaxation-time
collision on central moments that the paper's production runs use, App. A):
  - all rates equal to 1/tau is the BGK collision with Guo forcing;
  - every central moment, summed directly over the nine directions (numpy,
    not the oracle's moment matrix), relaxes at its own rate;
  - mass is conserved and the momentum gains exactly F per node and step,
    whatever the rates;
  - a shear wave between the walls decays at nu (pi/H)^2 with
    nu = (tau - 1/2)/3, whatever the bulk and higher-order rates."""
import numpy as np
import pytest

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
PQ = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]


def central(x, ux, uy):
    return np.array([np.sum((CX - ux) ** p * (CY - uy) ** q * x) for p, q in PQ])


def random_node(rng, force=True):
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = w * (1 + 0.1 * rng.standard_normal(9))
    F = 1e-3 * rng.standard_normal(2) if force else np.zeros(2)
    rho = f.sum()
    ux, uy = (f @ CX + F[0] / 2) / rho, (f @ CY + F[1] / 2) / rho
    return f, F, rho, ux, uy


def test_equal_rates_is_bgk(orc):
    kw = dict(obstacle=(9, 3, 4, 3), gx=2e-5, gy=-5e-6)
    for tau in (0.55, 0.8, 1.4):
        bgk = orc.cfg(30, 11, tau=tau, **kw)
        cm = orc.cfg(30, 11, tau=tau, collision=1, omega_bulk=1 / tau, omega_3=1 / tau, omega_4=1 / tau, **kw)
        f0 = orc.init(bgk, 4, 0, 0.02)
        fb, db = orc.run(bgk, f0, 20)
        fc, dc = orc.run(cm, f0, 20)
        assert np.abs(fb - fc).max() < 1e-13
        assert np.abs(db - dc).max() < 1e-13


def test_each_central_moment_relaxes_at_its_rate(orc):
    """Without force: the non-equilibrium part of k20 + k02 shrinks by
    (1 - w_bulk), of k20 - k02 and k11 by (1 - w_shear), of k21 and k12 by
    (1 - w_3), of k22 by (1 - w_4); the conserved moments are unchanged.  With
    force the relation holds for k - k_eq + k_S / 2 and adds k_S."""
    rng = np.random.default_rng(3)
    for force in (False, True):
        for _ in range(50):
            f, F, rho, ux, uy = random_node(rng, force)
            ws, wb, w3, w4 = rng.uniform(0.4, 1.9, 4)
            feq = orc.feq(rho, ux, uy)
            S = orc.guo(ux, uy, F[0], F[1])
            out = orc.cm_collide(f, ux, uy, feq, S, [ws, wb, w3, w4])
            k_in = central(f, ux, uy) - central(feq, ux, uy) + central(S, ux, uy) / 2
            k_out = central(out, ux, uy) - central(feq, ux, uy) - central(S, ux, uy) / 2
            # bulk and deviatoric combinations of the second-order moments
            bulk_in, dev_in = k_in[3] + k_in[4], k_in[3] - k_in[4]
            bulk_out, dev_out = k_out[3] + k_out[4], k_out[3] - k_out[4]
            np.testing.assert_allclose(bulk_out, (1 - wb) * bulk_in, atol=1e-15)
            np.testing.assert_allclose(dev_out, (1 - ws) * dev_in, atol=1e-15)
            np.testing.assert_allclose(k_out[5], (1 - ws) * k_in[5], atol=1e-15)
            np.testing.assert_allclose(k_out[6:8], (1 - w3) * k_in[6:8], atol=1e-15)
            np.testing.assert_allclose(k_out[8], (1 - w4) * k_in[8], atol=1e-15)
            np.testing.assert_allclose(k_out[:3], 0.0, atol=1e-15)


def test_mass_and_momentum_for_any_rates(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        f, F, rho, ux, uy = random_node(rng)
        rates = rng.uniform(0.3, 1.95, 4)
        out = orc.cm_collide(f, ux, uy, orc.feq(rho, ux, uy), orc.guo(ux, uy, F[0], F[1]), rates)
        assert abs(out.sum() - f.sum()) < 1e-15
        assert abs(out @ CX - (f @ CX + F[0])) < 1e-15
        assert abs(out @ CY - (f @ CY + F[1])) < 1e-15


def shear_decay_rate(orc, tau, **rates):
    """decay rate of u_x(y) = U sin(pi (y + 1/2) / H) between the halfway walls"""
    H, nx = 32, 4
    c = orc.cfg(nx, H, tau=tau, collision=1, **rates)
    mode = np.sin(np.pi * (np.arange(H) + 0.5) / H)
    f = np.zeros((9, H, nx))
    for y in range(H):
        f[:, y, :] = orc.feq(1.0, 1e-3 * mode[y], 0.0)[:, None]
    amp = []
    for n in (200, 1000):
        f, _ = orc.run(c, f, n)
        ux = np.einsum("q,qyx->yx", CX, f).mean(axis=1)
        amp.append((ux * mode).sum() / (mode * mode).sum())
    return -np.log(amp[1] / amp[0]) / 1000


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_shear_wave_decays_at_the_viscosity_of_tau(orc, tau):
    ref = (tau - 0.5) / 3 * (np.pi / 32) ** 2
    for rates in (dict(), dict(omega_bulk=1.6, omega_3=1.3, omega_4=0.7)):
        assert abs(shear_decay_rate(orc, tau, **rates) / ref - 1) < 5e-3, rates
