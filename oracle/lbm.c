/*
 * Oracle (test infrastructure): D2Q9 lattice-BGK channel flow, FP64, one thread.
 *
 * Follows App. A of the paper step by step:
 *   moments            rho = sum_i f_i,  rho u = sum_i f_i c_i
 *   exact streaming    f_i(x + c_i, t+1) = f_i^out(x, t)
 *   BGK collision      f_i^out = f_i - (f_i - f_i^eq) / tau
 *                      (the printed formula lacks the leading f_i; the
 *                      viscosity nu = (tau - 1/2) c_s^2 fixes this reading)
 *   equilibrium        w_i rho (1 + u.c_i/cs2 + u_a u_b (c_ia c_ib - cs2 d_ab)/(2 cs2^2)),
 *                      w = 4/9, 1/9 (axis), 1/36 (diagonal), cs2 = 1/3
 * and Sec. 2: halfway bounce-back no-slip on the channel walls and on the square
 * obstacle.  The channel is periodic in x and driven by a constant body-force
 * density F on fluid nodes through the forcing scheme of Guo, Zheng & Shi
 * (Phys. Rev. E 65, 046308, 2002): the velocity carries half the force,
 *   rho u = sum_i f_i c_i + F/2,
 * and the collision adds (1 - 1/(2 tau)) S_i with
 *   S_i = w_i [ (c_i - u)/cs2 + (c_i.u) c_i / cs2^2 ] . F.
 * The force on the obstacle is the momentum exchanged by the links that are
 * bounced back at the next streaming step, 2 c_i f_i^out over fluid nodes x and
 * directions i with x + c_i inside the obstacle: the surface integral of the
 * stress of eq. (drag_definition) for the halfway bounce-back surface.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities: rest, four axis links, four diagonal links */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double CS2 = 1.0 / 3.0;

#define IDX(c, q, x, y) ((((size_t)(q)) * (c)->ny + (size_t)(y)) * (c)->nx + (size_t)(x))

/* the square whose drag is measured */
static int in_obstacle(const orc_cfg* c, int x, int y)
{
    return c->ow > 0 && x >= c->ox0 && x < c->ox0 + c->ow && y >= c->oy0 && y < c->oy0 + c->oh;
}

/* Open channel of Sec. 2: a grid of bars at the entrance generates the
 * turbulence; bars of height grid_bar separated by grid_gap fluid rows,
 * starting with a gap at the bottom wall, grid_w columns thick. */
static int in_grid(const orc_cfg* c, int x, int y)
{
    return c->grid_w > 0 && x >= c->grid_x0 && x < c->grid_x0 + c->grid_w &&
           (y % (c->grid_bar + c->grid_gap)) >= c->grid_gap;
}

int orc_is_solid(const orc_cfg* c, int x, int y) { return in_obstacle(c, x, y) || in_grid(c, x, y); }

/* sponge zone (Sec. 2, "viscosity artificially enhanced" near the end of the
 * channel): tau rises quadratically from tau to sponge_tau over the last
 * sponge_len columns, reaching sponge_tau at x = nx - 1 */
double orc_tau_at(const orc_cfg* c, int x)
{
    if (!c->open_x || c->sponge_len <= 0 || x < c->nx - c->sponge_len) return c->tau;
    double s = (double)(x - (c->nx - c->sponge_len) + 1) / c->sponge_len;
    return c->tau + (c->sponge_tau - c->tau) * s * s;
}

/* parabolic inlet profile vanishing on the halfway walls y = -1/2 and
 * y = ny - 1/2, u_in on the centreline */
double orc_inlet_u(const orc_cfg* c, int y)
{
    double h = c->ny, yy = y + 0.5;
    return c->u_in * 4.0 * yy * (h - yy) / (h * h);
}

void orc_feq(double rho, double ux, double uy, double feq[9])
{
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        double quad = 0.0; /* u_a u_b (c_ia c_ib - cs2 delta_ab) */
        quad += ux * ux * (CX[i] * CX[i] - CS2);
        quad += 2.0 * ux * uy * (CX[i] * CY[i]);
        quad += uy * uy * (CY[i] * CY[i] - CS2);
        feq[i] = W[i] * rho * (1.0 + cu / CS2 + quad / (2.0 * CS2 * CS2));
    }
}

void orc_guo(double ux, double uy, double gx, double gy, double S[9])
{
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        double ax = (CX[i] - ux) / CS2 + cu * CX[i] / (CS2 * CS2);
        double ay = (CY[i] - uy) / CS2 + cu * CY[i] / (CS2 * CS2);
        S[i] = W[i] * (ax * gx + ay * gy);
    }
}

void orc_init(const orc_cfg* c, uint64_t seed, int32_t clone, double amp, double* f)
{
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            double feq[9];
            if (orc_is_solid(c, x, y)) {
                for (int i = 0; i < 9; ++i) feq[i] = W[i];
            } else {
                uint64_t site = (uint64_t)y * (uint64_t)c->nx + (uint64_t)x;
                uint64_t ctr[4] = {5u, (uint64_t)clone, site, 0u}, key[2] = {seed, 0u}, o[4];
                orc_philox4x64(ctr, key, o);
                double ux = amp * (2.0 * orc_u01(o[0]) - 1.0);
                double uy = amp * (2.0 * orc_u01(o[1]) - 1.0);
                if (c->open_x) ux += orc_inlet_u(c, y);  /* open channel: the inlet profile everywhere */
                orc_feq(1.0, ux, uy, feq);
            }
            for (int i = 0; i < 9; ++i) f[IDX(c, i, x, y)] = feq[i];
        }
}

/* density and velocity of node (x, y) of post-collision populations: their
 * momentum carries the whole force of the step, the fluid velocity half of it */
static void node_macro(const orc_cfg* c, const double* f, int x, int y, double* rho, double* ux, double* uy)
{
    double r = 0, jx = 0, jy = 0;
    for (int i = 0; i < 9; ++i) {
        double v = f[IDX(c, i, x, y)];
        r += v;
        jx += v * CX[i];
        jy += v * CY[i];
    }
    *rho = r;
    *ux = (jx - 0.5 * c->gx) / r;
    *uy = (jy - 0.5 * c->gy) / r;
}

void orc_macro(const orc_cfg* c, const double* f, double* rho, double* ux, double* uy)
{
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            size_t s = (size_t)y * c->nx + x;
            node_macro(c, f, x, y, rho + s, ux + s, uy + s);
        }
}

static void link_forces(const orc_cfg* c, const double* f, double* fo, double* fw)
{
    double ox = 0, oy = 0, wx = 0, wy = 0;
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            if (orc_is_solid(c, x, y)) continue;
            for (int i = 1; i < 9; ++i) {
                int xn = ((x + CX[i]) % c->nx + c->nx) % c->nx;
                int yn = y + CY[i];
                double v = f[IDX(c, i, x, y)];
                if (yn < 0 || yn >= c->ny) {
                    wx += 2.0 * CX[i] * v;
                    wy += 2.0 * CY[i] * v;
                } else if (in_obstacle(c, xn, yn)) {  /* the drag: links into the square only */
                    ox += 2.0 * CX[i] * v;
                    oy += 2.0 * CY[i] * v;
                }
            }
        }
    if (fo) { fo[0] = ox; fo[1] = oy; }
    if (fw) { fw[0] = wx; fw[1] = wy; }
}

/* Central-moment collision with multiple relaxation times.  The paper's
 * production runs replace the BGK collision by a multi-relaxation-time
 * collision on central moments (App. A, after De Rosis 2016).  Written here
 * as the generalisation of the BGK collision above:
 *   central moments       k_pq = sum_i (c_ix - u_x)^p (c_iy - u_y)^q f_i,
 *                         i.e. k = T f for the nine D2Q9 moments
 *                         pq = 00 10 01 20 02 11 21 12 22;
 *   discrete equilibrium  k^eq = T f^eq (the same second-order f^eq);
 *   forcing               the Guo term S enters as in BGK, with (I - Omega/2)
 *                         on its moments;
 *   collision             f* = f - T^{-1} Omega T (f - f^eq) + T^{-1} (I - Omega/2) T S
 *                            = f + S - T^{-1} Omega T (f - f^eq + S/2).
 * Omega relaxes the shear moments (k20 - k02 and k11) at 1/tau, the bulk
 * moment k20 + k02, the third-order k21, k12 and the fourth-order k22 at
 * their own rates; Omega = omega I is the BGK collision with Guo forcing.  T
 * is built and inverted numerically (Gauss-Jordan) at every node.            */
static const int MP[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MQ[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}

/* inverse of a 9 x 9 matrix by Gauss-Jordan elimination with partial pivoting */
static void invert9(const double a_in[9][9], double inv[9][9])
{
    double a[9][18];
    for (int r = 0; r < 9; ++r)
        for (int j = 0; j < 18; ++j) a[r][j] = j < 9 ? a_in[r][j] : (j - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 18; ++j) {
                double t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        double d = a[col][col];
        for (int j = 0; j < 18; ++j) a[col][j] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m != 0.0)
                for (int j = 0; j < 18; ++j) a[r][j] -= m * a[col][j];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int j = 0; j < 9; ++j) inv[r][j] = a[r][j + 9];
}

void orc_cm_collide(const double f[9], double ux, double uy, const double feq[9], const double S[9],
                    const double rates[4], double out[9])
{
    double T[9][9], Ti[9][9], Om[9][9];
    for (int r = 0; r < 9; ++r)
        for (int i = 0; i < 9; ++i) T[r][i] = ipow(CX[i] - ux, MP[r]) * ipow(CY[i] - uy, MQ[r]);
    invert9(T, Ti);
    for (int r = 0; r < 9; ++r)
        for (int j = 0; j < 9; ++j) Om[r][j] = 0.0;
    const double ws = rates[0], wb = rates[1], w3 = rates[2], w4 = rates[3];
    Om[0][0] = Om[1][1] = Om[2][2] = 1.0;  /* conserved: their moments of d are zero */
    Om[3][3] = Om[4][4] = 0.5 * (wb + ws);  /* k20, k02: bulk sum at wb, difference at ws */
    Om[3][4] = Om[4][3] = 0.5 * (wb - ws);
    Om[5][5] = ws;                          /* k11 */
    Om[6][6] = Om[7][7] = w3;               /* k21, k12 */
    Om[8][8] = w4;                          /* k22 */
    double d[9], k[9], rk[9];
    for (int i = 0; i < 9; ++i) d[i] = f[i] - feq[i] + 0.5 * S[i];
    for (int r = 0; r < 9; ++r) {
        k[r] = 0.0;
        for (int i = 0; i < 9; ++i) k[r] += T[r][i] * d[i];
    }
    for (int r = 0; r < 9; ++r) {
        rk[r] = 0.0;
        for (int j = 0; j < 9; ++j) rk[r] += Om[r][j] * k[j];
    }
    for (int i = 0; i < 9; ++i) {
        double x = 0.0;
        for (int r = 0; r < 9; ++r) x += Ti[i][r] * rk[r];
        out[i] = f[i] + S[i] - x;
    }
}

/* Boundary columns of the open channel (Sec. 2), applied to post-collision
 * populations:
 *   inlet  x = 0:      f = f^eq(rho = 1, u = (u_in(y), 0))  ("constant
 *                      parabolic velocity profile and constant mass density");
 *   outlet x = nx-1:   u extrapolated to second order from the two columns
 *                      upstream, u(nx-1) = 2 u(nx-2) - u(nx-3), rho = 1, and
 *                      the populations regularized (Latt et al. 2008):
 *                      f = f^eq(rho, u) + w_i / (2 cs2^2) Q_i : Pi,
 *                      Q_i = c_i c_i - cs2 I,  Pi = -2 rho cs2 (tau_out - 1) S,
 *                      S the strain rate from finite differences (one-sided
 *                      second order in x, central in y, one-sided at the walls);
 *                      tau_out - 1, not tau_out: the post-collision
 *                      non-equilibrium is (1 - 1/tau) times the pre-collision one.
 * The outlet density is the reference density rather than extrapolated: with
 * the inlet holding rho = 1, an extrapolated outlet density leaves the mean
 * pressure drop free, and that neutral mode drifts (the channel either
 * accelerates or fills up and stalls within a few thousand steps).
 * The macroscopic fields of a post-collision state are rho = sum f,
 * rho u = sum c f (an open channel has no body force).                       */
static void open_boundaries(const orc_cfg* c, double* f)
{
    const int nx = c->nx, ny = c->ny;
    for (int y = 0; y < ny; ++y) {
        if (orc_is_solid(c, 0, y)) continue;
        double feq[9];
        orc_feq(1.0, orc_inlet_u(c, y), 0.0, feq);
        for (int i = 0; i < 9; ++i) f[IDX(c, i, 0, y)] = feq[i];
    }
    double* ux = malloc(sizeof(double) * ny);
    double* uy = malloc(sizeof(double) * ny);
    double* u2x = malloc(sizeof(double) * ny);  /* u at nx-2 minus u at nx-3: the x derivative */
    double* u2y = malloc(sizeof(double) * ny);
    for (int y = 0; y < ny; ++y) {
        double vx[2], vy[2];
        for (int k = 0; k < 2; ++k) {
            const int x = nx - 2 - k;
            double m = 0, jx = 0, jy = 0;
            for (int i = 0; i < 9; ++i) {
                double v = f[IDX(c, i, x, y)];
                m += v;
                jx += v * CX[i];
                jy += v * CY[i];
            }
            vx[k] = jx / m;
            vy[k] = jy / m;
        }
        ux[y] = 2.0 * vx[0] - vx[1];
        uy[y] = 2.0 * vy[0] - vy[1];
        u2x[y] = vx[0] - vx[1];  /* (3 u(nx-1) - 4 u(nx-2) + u(nx-3)) / 2 */
        u2y[y] = vy[0] - vy[1];
    }
    const double tau_out = orc_tau_at(c, nx - 1);
    for (int y = 0; y < ny; ++y) {
        const int ym = y > 0 ? y - 1 : y, yp = y < ny - 1 ? y + 1 : y;
        const double dy = (double)(yp - ym);
        const double dxux = u2x[y], dxuy = u2y[y];
        const double dyux = (ux[yp] - ux[ym]) / dy, dyuy = (uy[yp] - uy[ym]) / dy;
        const double sxx = dxux, syy = dyuy, sxy = 0.5 * (dyux + dxuy);
        const double pre = -2.0 * CS2 * (tau_out - 1.0);  /* rho = 1 */
        const double pxx = pre * sxx, pyy = pre * syy, pxy = pre * sxy;
        double feq[9];
        orc_feq(1.0, ux[y], uy[y], feq);
        for (int i = 0; i < 9; ++i) {
            const double q = (CX[i] * CX[i] - CS2) * pxx + 2.0 * CX[i] * CY[i] * pxy + (CY[i] * CY[i] - CS2) * pyy;
            f[IDX(c, i, nx - 1, y)] = feq[i] + W[i] / (2.0 * CS2 * CS2) * q;
        }
    }
    free(ux);
    free(uy);
    free(u2x);
    free(u2y);
}

void orc_step(const orc_cfg* c, const double* fin, double* fout, double* force_obs, double* force_wall)
{
    const int nx = c->nx, ny = c->ny;
    /* 1. streaming into fout, links into a wall or the obstacle reflect back
     *    into the opposite direction at the same node */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (orc_is_solid(c, x, y)) continue;
            for (int i = 0; i < 9; ++i) {
                int xn = ((x + CX[i]) % nx + nx) % nx;
                int yn = y + CY[i];
                double v = fin[IDX(c, i, x, y)];
                /* open channel: a population leaving through the inlet or the
                 * outlet column is gone (those columns are set by their
                 * boundary conditions after the collision) */
                if (c->open_x && (x + CX[i] < 0 || x + CX[i] >= nx) && yn >= 0 && yn < ny) continue;
                if (yn < 0 || yn >= ny || orc_is_solid(c, xn, yn))
                    fout[IDX(c, OPP[i], x, y)] = v;
                else
                    fout[IDX(c, i, xn, yn)] = v;
            }
        }
    /* 2. collision at every fluid node; solid nodes hold the rest weights */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (orc_is_solid(c, x, y)) {
                for (int i = 0; i < 9; ++i) fout[IDX(c, i, x, y)] = W[i];
                continue;
            }
            double f[9], rho = 0, jx = 0, jy = 0;
            for (int i = 0; i < 9; ++i) {
                f[i] = fout[IDX(c, i, x, y)];
                rho += f[i];
                jx += f[i] * CX[i];
                jy += f[i] * CY[i];
            }
            double ux = (jx + 0.5 * c->gx) / rho;
            double uy = (jy + 0.5 * c->gy) / rho;
            double feq[9], S[9];
            orc_feq(rho, ux, uy, feq);
            orc_guo(ux, uy, c->gx, c->gy, S);
            const double tau = orc_tau_at(c, x);
            if (c->collision == 1) {
                const double rates[4] = {1.0 / tau, c->omega_bulk, c->omega_3, c->omega_4};
                double out[9];
                orc_cm_collide(f, ux, uy, feq, S, rates, out);
                for (int i = 0; i < 9; ++i) fout[IDX(c, i, x, y)] = out[i];
            } else {
                for (int i = 0; i < 9; ++i)
                    fout[IDX(c, i, x, y)] = f[i] - (f[i] - feq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * S[i];
            }
        }
    /* 3. open channel: the boundary columns (Sec. 2) */
    if (c->open_x) open_boundaries(c, fout);
    /* 4. momentum exchanged with the obstacle and the walls by the links that
     *    the next streaming step bounces back */
    if (force_obs || force_wall) link_forces(c, fout, force_obs, force_wall);
}

void orc_run(const orc_cfg* c, double* f, double* scratch, int32_t n, double* drag)
{
    size_t sz = (size_t)9 * c->nx * c->ny;
    for (int32_t t = 0; t < n; ++t) {
        double fo[2];
        orc_step(c, f, scratch, drag ? fo : NULL, NULL);
        memcpy(f, scratch, sz * sizeof(double));
        if (drag) drag[t] = fo[0];
    }
}

void orc_moments(const orc_cfg* c, const double* f, double* mass, double* px, double* py)
{
    double m = 0, jx = 0, jy = 0;
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            if (orc_is_solid(c, x, y)) continue;
            for (int i = 0; i < 9; ++i) {
                double v = f[IDX(c, i, x, y)];
                m += v;
                jx += v * CX[i];
                jy += v * CY[i];
            }
        }
    if (mass) *mass = m;
    if (px) *px = jx;
    if (py) *py = jy;
}

void orc_perturb_alphas(uint64_t seed, uint64_t iter, int32_t slot, int32_t n_s, double* alpha)
{
    for (int32_t n = 0; n < n_s; ++n) {
        uint64_t ctr[4] = {4u, iter, (uint64_t)slot, (uint64_t)n}, key[2] = {seed, 0u}, o[4];
        orc_philox4x64(ctr, key, o);
        alpha[n] = orc_u01(o[0]);
    }
}

/* App. D, eq. (perturb_pop): add a random combination of snapshots, then
 * rescale so that the mass of the fluid is that of the unperturbed state */
void orc_perturb(const orc_cfg* c, const double* f, int32_t n_s, const double* snaps,
                 const double* alpha, double eps, double* f_out)
{
    size_t sz = (size_t)9 * c->nx * c->ny;
    double m_before, m_after;
    orc_moments(c, f, &m_before, NULL, NULL);
    for (size_t k = 0; k < sz; ++k) {
        double v = f[k];
        for (int32_t n = 0; n < n_s; ++n) v += eps * alpha[n] * snaps[(size_t)n * sz + k];
        f_out[k] = v;
    }
    orc_moments(c, f_out, &m_after, NULL, NULL);
    double scale = m_before / m_after;
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x)
            for (int i = 0; i < 9; ++i) {
                if (orc_is_solid(c, x, y))
                    f_out[IDX(c, i, x, y)] = W[i];
                else
                    f_out[IDX(c, i, x, y)] *= scale;
            }
}

/* Sec. 2.1 eq. (drag_approx) and Sec. 3.2 eq. (avg_shear_def); see oracle.h */
int orc_observables(const orc_cfg* c, const double* f, double out[4])
{
    const int x0 = c->ox0, x1 = c->ox0 + c->ow, y0 = c->oy0, y1 = c->oy0 + c->oh;
    if (c->ow <= 0 || x0 < 1 || x1 > c->nx - 1 || y0 < 2 || y1 > c->ny - 2) return -1;
    double rho_at, ux_at, uy_at;
    double pfb = 0.0, pbase = 0.0;
    for (int y = y0; y < y1; ++y) {
        node_macro(c, f, x0 - 1, y, &rho_at, &ux_at, &uy_at);
        pfb += CS2 * rho_at;
        node_macro(c, f, x1, y, &rho_at, &ux_at, &uy_at);
        pbase += CS2 * rho_at;
    }
    double gt = 0.0, gb = 0.0;
    for (int x = x0; x < x1; ++x) {
        double u1, u2;
        node_macro(c, f, x, y1, &rho_at, &u1, &uy_at);      /* 1/2 above the top wall */
        node_macro(c, f, x, y1 + 1, &rho_at, &u2, &uy_at);  /* 3/2 above */
        gt += (9.0 * u1 - u2) / 3.0;
        node_macro(c, f, x, y0 - 1, &rho_at, &u1, &uy_at);  /* 1/2 below the bottom wall */
        node_macro(c, f, x, y0 - 2, &rho_at, &u2, &uy_at);  /* 3/2 below */
        gb -= (9.0 * u1 - u2) / 3.0;
    }
    out[0] = pfb;
    out[1] = pbase;
    out[2] = gt / c->ow;
    out[3] = gb / c->ow;
    return 0;
}

