"""Pins of the oracle's square observables: the forebody and base pressures of
eq. (drag_approx) and the mean wall shear of eq. (avg_shear_def).
  - on constructed equilibrium fields (numpy f^eq, not the oracle's) with a
    linear density and a velocity quadratic in the distance from each face,
    the pressures are the closed-form sums and the shear is the slope at the
    wall exactly, with the velocity carrying half the body force;
  - a flow symmetric about the channel's midline has gamma_top = -gamma_bottom;
  - in steady flow past the square the momentum-exchange drag balances the
    pressure difference plus the viscous shear on the top and bottom faces,
    D ~ (p_fb - p_base) + rho nu R (gamma_top - gamma_bottom), within the
    discretisation error of the face sums (12%)."""
import numpy as np
import pytest

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def numpy_feq(rho, ux, uy):
    cu = CX[:, None, None] * ux + CY[:, None, None] * uy
    return W[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


@pytest.mark.parametrize("gx", [0.0, 3e-4])
def test_constructed_fields(orc, gx):
    nx, ny, sq = 40, 24, (14, 8, 6, 5)
    x0, y0, w, h = sq
    c = orc.cfg(nx, ny, obstacle=sq, tau=0.7, gx=gx)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    a, b = 2e-3, -1e-3
    rho = 1.0 + a * X + b * Y
    # u_x quadratic in the distance from the top wall above the square (slope
    # depending on x) and from the bottom wall below it
    top, bot = y0 + h - 0.5, y0 - 0.5
    s_top = 0.01 + 1e-3 * X
    s_bot = -0.02 + 5e-4 * X
    ux = np.where(Y >= y0 + h, s_top * (Y - top) + 3e-4 * (Y - top) ** 2,
                  np.where(Y < y0, s_bot * (bot - Y) - 2e-4 * (bot - Y) ** 2, 0.01))
    uy = 1e-3 * np.sin(X)
    # populations whose momentum carries the step's full force: u = (sum c f - F/2) / rho
    f = numpy_feq(rho, ux + 0.5 * gx / rho, uy)
    o = orc.observables(c, f)
    rows = np.arange(y0, y0 + h)
    np.testing.assert_allclose(o[0], CS2 * (1.0 + a * (x0 - 1) + b * rows).sum(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(o[1], CS2 * (1.0 + a * (x0 + w) + b * rows).sum(), rtol=0, atol=1e-14)
    xs = np.arange(x0, x0 + w)
    np.testing.assert_allclose(o[2], (0.01 + 1e-3 * xs).mean(), rtol=0, atol=1e-14)
    # below the square u grows downward: the slope in +y is minus the slope in the distance
    np.testing.assert_allclose(o[3], -(-0.02 + 5e-4 * xs).mean(), rtol=0, atol=1e-14)


def test_geometry_checks(orc):
    f = orc.init(orc.cfg(30, 12, obstacle=(10, 2, 4, 4)), 0, 0, 0.0)
    for sq in [(10, 1, 4, 4), (10, 4, 4, 7), (0, 4, 4, 4), (0, 0, 0, 0)]:
        with pytest.raises(ValueError):
            orc.observables(orc.cfg(30, 12, obstacle=sq), f)


def test_symmetric_flow_has_opposite_shears(orc):
    c = orc.cfg(80, 30, obstacle=(30, 11, 8, 8), tau=0.56, open_x=1, u_in=0.04, sponge_len=12, sponge_tau=0.9)
    f, _ = orc.run(c, orc.init(c, 0, 0, 0.0), 300)
    o = orc.observables(c, f)
    assert abs(o[2]) > 1e-4
    assert abs(o[2] + o[3]) < 1e-12 * abs(o[2]) * 1e3


@pytest.mark.parametrize("tau,gx,n", [(0.6, 1e-5, 8000), (0.8, 2e-5, 6000), (1.0, 4e-5, 4000)])
def test_drag_balances_pressure_and_viscous_shear(orc, tau, gx, n):
    R = 8
    c = orc.cfg(96, 32, obstacle=(30, 12, R, R), tau=tau, gx=gx)
    f, d = orc.run(c, orc.init(c, 0, 0, 0.0), n)
    o = orc.observables(c, f)
    nu = (tau - 0.5) / 3
    estimate = (o[0] - o[1]) + nu * R * (o[2] - o[3])
    assert o[0] > o[1]  # the forebody carries the higher pressure
    assert abs(estimate / d[-1] - 1) < 0.12
