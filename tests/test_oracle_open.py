"""Pins of the oracle's open channel (Sec. 2: inlet with a parabolic profile and
unit density, entrance grid of bars, sponge zone of raised viscosity, outlet
with extrapolated velocity and regularized populations) against what the
scheme's conservation laws and the Navier-Stokes limit fix:
  - the rest state stays at rest, whatever the geometry and the collision;
  - one step changes the mass between the boundary columns by exactly what
    streams in from them minus what streams out into them;
  - developed flow carries the same mass flux through every cut, is parabolic
    across the channel, and its pressure gradient balances the viscous stress,
    cs2 d(rho)/dx = nu(x) rho d2u/dy2, with nu(x) = (tau(x) - 1/2)/3 in the
    bulk and inside the sponge;
  - the inlet column is the equilibrium of rho = 1 and the parabola that
    vanishes on the halfway walls; the outlet column carries rho = 1, the
    second-order extrapolated velocity and the non-equilibrium stress of the
    finite-difference strain rate;
  - the grid has bars of the stated height and spacing, and the drag counts
    the links into the square only."""
import ctypes

import numpy as np
import pytest

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def taus(orc, c):
    return np.array([orc.lib().orc_tau_at(ctypes.byref(c), x) for x in range(c.nx)])


def solid(orc, c):
    return np.array([[orc.lib().orc_is_solid(ctypes.byref(c), x, y) for x in range(c.nx)] for y in range(c.ny)],
                    dtype=bool)


def numpy_feq(rho, ux, uy):
    cu = CX * ux + CY * uy
    return W * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


def fluid_moments(f, x):
    rho = f[:, :, x].sum(0)
    return rho, (CX[:, None] * f[:, :, x]).sum(0) / rho, (CY[:, None] * f[:, :, x]).sum(0) / rho


@pytest.mark.parametrize("collision", [0, 1])
def test_rest_state_stays_at_rest(orc, collision):
    c = orc.cfg(60, 24, obstacle=(30, 8, 6, 6), tau=0.55, open_x=1, u_in=0.0, grid=(6, 3, 3, 3), sponge_len=12,
                sponge_tau=0.9, collision=collision, omega_bulk=1.4, omega_3=1.1, omega_4=1.6)
    f0 = orc.init(c, 0, 0, 0.0)
    f, drag = orc.run(c, f0, 40)
    assert np.abs(f - f0).max() < 1e-14  # rounding of the moment sums only
    assert np.abs(drag).max() < 1e-14


@pytest.mark.parametrize("collision", [0, 1])
def test_mass_balance_between_the_boundary_columns(orc, collision):
    nx, ny = 48, 20
    c = orc.cfg(nx, ny, obstacle=(24, 7, 5, 5), tau=0.6, open_x=1, u_in=0.04, grid=(4, 2, 3, 4), sponge_len=10,
                sponge_tau=0.95, collision=collision, omega_bulk=1.2, omega_3=0.9, omega_4=1.3)
    f = orc.init(c, 3, 0, 0.02)
    f, _ = orc.run(c, f, 25)  # a developing, unsteady state
    sol = solid(orc, c)
    inner = ~sol.copy()
    inner[:, 0] = inner[:, nx - 1] = False
    for _ in range(5):
        g, _, _ = orc.step(c, f)
        gain = 0.0
        for i in range(9):
            for y in range(ny):
                yn = y + CY[i]
                if not 0 <= yn < ny:
                    continue
                for src, dst in ((0, 1), (nx - 1, nx - 2)):  # into the interior
                    if src + CX[i] == dst and not sol[yn, dst]:
                        gain += f[i, y, src]
                for src, dst in ((1, 0), (nx - 2, nx - 1)):  # out of it
                    if src + CX[i] == dst and not sol[y, src]:
                        gain -= f[i, y, src]
        m0 = (f.sum(0) * inner).sum()
        m1 = (g.sum(0) * inner).sum()
        assert abs(m1 - m0 - gain) < 1e-12
        f = g


@pytest.fixture(scope="module")
def developed(orc):
    """a 64 x 16 open channel run to its steady state (8000 steps = 3 diffusion
    times H^2/nu), sponge over the last 16 columns"""
    c = orc.cfg(64, 16, tau=0.8, open_x=1, u_in=0.01, sponge_len=16, sponge_tau=1.0)
    f, _ = orc.run(c, orc.init(c, 0, 0, 0.0), 8000)
    return c, f


def test_developed_flow_carries_one_mass_flux(developed):
    c, f = developed
    fl = []
    for x in range(c.nx - 1):
        s = 0.0
        for i in range(9):
            for y in range(c.ny):
                if not 0 <= y + CY[i] < c.ny:  # a diagonal into a wall is bounced back
                    continue
                if CX[i] == 1:
                    s += f[i, y, x]
                elif CX[i] == -1:
                    s -= f[i, y, x + 1]
        fl.append(s)
    fl = np.array(fl)
    assert fl.min() > 0
    assert np.abs(fl / fl.mean() - 1).max() < 1e-9


def test_developed_flow_is_parabolic_and_balances_viscous_stress(orc, developed):
    c, f = developed
    t = taus(orc, c)
    for x in (16, 24, 32):
        rho, ux, uy = fluid_moments(f, x)
        d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.abs(d2 / d2.mean() - 1).max() < 2e-3  # constant curvature: a parabola
        assert np.abs(uy).max() < 3e-5 * np.abs(ux).max()  # no cross flow
    for x, tol in ((20, 1e-3), (30, 1e-3), (40, 1e-3), (52, 2e-2), (56, 2e-2), (59, 2e-2)):
        rho, ux, _ = fluid_moments(f, x)
        d2 = (ux[2:] - 2 * ux[1:-1] + ux[:-2]).mean()
        drho = (f[:, :, x + 1].sum(0) - f[:, :, x - 1].sum(0)).mean() / 2
        nu = (t[x] - 0.5) / 3
        assert abs(CS2 * drho / (nu * rho.mean() * d2) - 1) < tol, x


def test_sponge_profile(orc):
    c = orc.cfg(50, 8, tau=0.52, open_x=1, sponge_len=10, sponge_tau=0.9)
    t = taus(orc, c)
    assert np.all(t[:40] == 0.52)
    assert t[49] == 0.9
    assert np.all(np.diff(t[39:]) > 0)
    # quadratic in the distance into the zone
    s = (np.arange(40, 50) - 39) / 10
    np.testing.assert_allclose(t[40:], 0.52 + 0.38 * s * s, rtol=0, atol=1e-15)
    assert np.all(taus(orc, orc.cfg(50, 8, tau=0.52, sponge_len=10, sponge_tau=0.9)) == 0.52)  # periodic: none


def test_inlet_column_is_the_equilibrium_of_the_profile(orc):
    ny, u_in = 12, 0.05
    c = orc.cfg(30, ny, tau=0.6, open_x=1, u_in=u_in, sponge_len=5, sponge_tau=0.8)
    f, _ = orc.run(c, orc.init(c, 2, 0, 0.03), 7)
    for y in range(ny):
        # the parabola through zero on both halfway walls with u_in halfway between them
        yy = y + 0.5
        u = u_in * (yy * (ny - yy)) / (ny / 2) ** 2
        np.testing.assert_allclose(f[:, y, 0], numpy_feq(1.0, u, 0.0), rtol=0, atol=1e-16)
    assert abs(orc.lib().orc_inlet_u(ctypes.byref(orc.cfg(30, 13, open_x=1, u_in=u_in)), 6) - u_in) < 1e-16


def test_outlet_column_is_regularized_with_the_extrapolated_velocity(orc):
    nx, ny = 40, 14
    c = orc.cfg(nx, ny, obstacle=(14, 5, 4, 4), tau=0.56, open_x=1, u_in=0.05, sponge_len=8, sponge_tau=0.85)
    f, _ = orc.run(c, orc.init(c, 1, 0, 0.02), 60)
    _, u2, v2 = fluid_moments(f, nx - 2)
    _, u3, v3 = fluid_moments(f, nx - 3)
    out = f[:, :, nx - 1]
    ux, uy = 2 * u2 - u3, 2 * v2 - v3
    np.testing.assert_allclose(out.sum(0), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose((CX[:, None] * out).sum(0), ux, rtol=0, atol=1e-15)
    np.testing.assert_allclose((CY[:, None] * out).sum(0), uy, rtol=0, atol=1e-15)
    # non-equilibrium second moment against the strain rate: x from the two
    # upstream columns, y by central differences (one-sided on the wall rows)
    dxux, dxuy = u2 - u3, v2 - v3
    dyux, dyuy = np.gradient(ux), np.gradient(uy)
    sxx, syy, sxy = dxux, dyuy, 0.5 * (dyux + dxuy)
    pref = -2 * CS2 * (0.85 - 1.0)
    neq = out - np.stack([numpy_feq(1.0, ux[y], uy[y]) for y in range(ny)], 1)
    np.testing.assert_allclose((CX[:, None] ** 2 * neq).sum(0), pref * sxx, rtol=0, atol=1e-15)
    np.testing.assert_allclose((CY[:, None] ** 2 * neq).sum(0), pref * syy, rtol=0, atol=1e-15)
    np.testing.assert_allclose(((CX * CY)[:, None] * neq).sum(0), pref * sxy, rtol=0, atol=1e-15)


def test_grid_of_bars_matches_the_stated_geometry(orc):
    """the channel of Sec. 2: 129 rows, bar height and spacing R/2 = 8"""
    c = orc.cfg(40, 129, open_x=1, grid=(8, 8, 8, 8))
    s = solid(orc, c)
    col = s[:, 10]
    assert not s[:, :8].any() and not s[:, 16:].any()
    assert np.all(s[:, 8:16] == col[:, None])
    # runs of solid rows: eight bars of eight rows, eight fluid rows before each
    edges = np.flatnonzero(np.diff(np.concatenate([[0], col.astype(int), [0]])))
    starts, ends = edges[::2], edges[1::2]
    assert len(starts) == 8
    assert np.all(ends - starts == 8)
    assert np.all(np.diff(starts) == 16) and starts[0] == 8


def test_drag_counts_the_square_only(orc):
    nx, ny = 44, 18
    kw = dict(tau=0.6, open_x=1, u_in=0.05, grid=(4, 2, 3, 3), sponge_len=8, sponge_tau=0.9)
    c = orc.cfg(nx, ny, obstacle=(20, 6, 5, 5), **kw)
    f, _ = orc.run(c, orc.init(c, 4, 0, 0.02), 30)
    g, fo, _ = orc.step(c, f)
    sq = np.zeros((ny, nx), dtype=bool)
    sq[6:11, 20:25] = True
    sol = solid(orc, c)
    d = 0.0
    for y in range(ny):
        for x in range(1, nx - 1):
            if sol[y, x]:
                continue
            for i in range(9):
                xn, yn = x + CX[i], y + CY[i]
                if 0 <= yn < ny and sq[yn, xn]:
                    d += 2 * CX[i] * g[i, y, x]
    assert abs(fo[0] - d) < 1e-15
    assert abs(fo[0]) > 1e-4
    # the grid alone exchanges momentum with the flow, but it is not the body
    c0 = orc.cfg(nx, ny, **kw)
    _, drag0 = orc.run(c0, orc.init(c0, 4, 0, 0.02), 30)
    assert np.all(drag0 == 0.0)
