/*
 * imb_oracle.c -- plain, slow FP64 CPU oracle of one coupled LBM-DEM step with
 * the Noble-Torczynski immersed moving boundary, after Yang, Jing, Kwok &
 * Sobral, "A comprehensive study of coupled LBM-DEM with immersed moving
 * boundary" (arXiv 1809.07008).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline and reference legs may load it.  It shares no code with the
 * CUDA library.  Compile with -ffp-contract=off: the two places where floating
 * point decides an integer (cell coverage, contact detection) must round every
 * operation separately, as the CUDA kernels do.
 *
 * One step, in the order of the paper's coupling cycle (Sec. 2.4, Fig. 4):
 *   1. DEM: N_sub sub-cycles with dt = 1/N_sub (Eq. 17), the hydrodynamic
 *      force and torque of the previous collision held fixed (Sec. 2.4);
 *      contacts by Eqs. 7-9 (linear spring-dashpot), motion by Eqs. 10-11
 *      integrated with the leapfrog form of Verlet's method.
 *   2. Map particles onto the lattice: per cell the covering particles and
 *      their solid ratios (Sec. 2.3, Fig. 3).
 *   3. Collide every node: BGK (Eq. 1 RHS, Eq. 2) with a Smagorinsky effective
 *      relaxation time (Sec. 3.3), blended with the solid operator of Eq. 12
 *      by the weight of Eq. 14 (Eq. 13); hydrodynamic force and torque by
 *      Eqs. 15-16 (force on the particle = minus the fluid's momentum gain).
 *   4. Stream (Eq. 1 LHS) with periodic, halfway bounce-back and
 *      inlet/outlet boundaries.
 *
 * Where the paper leaves a point open (lattice order, force sign, which tau enters
 * B, forcing scheme, wall placement, contact constants), the reading taken is
 * stated at the code that applies it.
 */
#include "imb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities, opposites and weights (Qian et al. 1992, cited in Sec. 2). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Host threads of the collide and stream loops (1 unless orc_set_threads says otherwise).
 * Every cell is computed by the same arithmetic whatever the count, and the particles'
 * forces are summed in the same order, so the results do not depend on it. */
static int g_threads = 1;

void orc_set_threads(int n)
{
    g_threads = n > 0 ? n : 1;
}

struct orc_sim {
    orc_params p;
    double *f;    /* f(x,t): post-stream, pre-collision  [9][ny][nx] */
    double *fs;   /* post-collision scratch                [9][ny][nx] */
    int np;
    double *px, *py, *vx, *vy, *w, *r, *m, *I;
    double *Ffx, *Ffy, *Tf;        /* hydrodynamic force/torque (Eqs. 15-16) */
    double *xi;                    /* tangential spring per pair, [np][np], a < b */
    double *xiw;                   /* tangential spring per particle-wall, [np][4] */
    int *cnt, *ids;                /* per cell: covering particles (ascending id) */
    double *eps;                   /* per cell and slot: solid ratio of that particle */
    double *fterm;                 /* per cell and slot: force x, y and torque terms (Eqs. 15-16) */
    int *fns;                      /* per cell: slots whose terms were computed */
    double zeta;                   /* damping ratio from the restitution coefficient */
    double gx_eff, gy_eff;         /* buoyancy-reduced gravity */
    double hm_kn0, hm_sn0, hm_kt0, hm_c0; /* Hertz-Mindlin: 4/3 E*, 2 E*, 8 G*, 2 sqrt(5/6) |beta| */
};

#define IDX(s, q, k, i) (((size_t)(q) * (s)->p.ny + (size_t)(k)) * (s)->p.nx + (size_t)(i))

/* ---------------------------------------------------------------- Eq. 2 */
void orc_feq(double rho, double ux, double uy, double *feq)
{
    double usq = ux * ux + uy * uy;
    for (int q = 0; q < 9; ++q) {
        double cu = CX[q] * ux + CY[q] * uy;
        /* c.u/cs^2 + (c.u)^2/(2 cs^4) - u^2/(2 cs^2) with cs^2 = 1/3 */
        feq[q] = W[q] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* ---------------------------------------------------------------- Eq. 14 */
double orc_B(double eps, double tau)
{
    double t = tau - 0.5;
    return eps * t / ((1.0 - eps) + t);
}

/* Moments (Eqs. 3-4, the garbled "u_i" of Eq. 4 read as c_i) with the
 * half-force velocity shift of Guo forcing. */
static void moments(const double *f9, double Fx, double Fy, double *rho, double *ux, double *uy)
{
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int q = 0; q < 9; ++q) {
        r += f9[q];
        jx += CX[q] * f9[q];
        jy += CY[q] * f9[q];
    }
    *rho = r;
    *ux = (jx + 0.5 * Fx) / r;
    *uy = (jy + 0.5 * Fy) / r;
}

/* Smagorinsky effective relaxation time (Sec. 3.3; the paper names the model
 * but not its formula -- this is the closure of Hou et al. 1996 it cites):
 * Pi = sum_i c_i c_i (f_i - f_i^eq), Q = Pi:Pi,
 * tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 sqrt(Q) / rho)) / 2. */
double orc_tau_eff(const double *f9, double Fx, double Fy, double tau, double C_smag)
{
    if (C_smag <= 0.0)
        return tau;
    double rho, ux, uy, fe[9];
    moments(f9, Fx, Fy, &rho, &ux, &uy);
    orc_feq(rho, ux, uy, fe);
    double pxx = 0.0, pyy = 0.0, pxy = 0.0;
    for (int q = 0; q < 9; ++q) {
        double ne = f9[q] - fe[q];
        pxx += CX[q] * CX[q] * ne;
        pyy += CY[q] * CY[q] * ne;
        pxy += CX[q] * CY[q] * ne;
    }
    double Q = pxx * pxx + pyy * pyy + 2.0 * pxy * pxy;
    return 0.5 * (tau + sqrt(tau * tau + 18.0 * sqrt(2.0) * C_smag * C_smag * sqrt(Q) / rho));
}

/* ------------------------------------------------ solid ratio (Sec. 2.3) */
/* int_0^x sqrt(r^2 - t^2) dt for |x| <= r. */
static double half_chord_prim(double x, double r)
{
    double h = sqrt(fmax(0.0, r * r - x * x));
    double s = x / r;
    if (s > 1.0) s = 1.0;
    if (s < -1.0) s = -1.0;
    return 0.5 * (x * h + r * r * asin(s));
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Exact area of the disk X^2 + Y^2 <= r^2 inside the rectangle [a0,a1]x[b0,b1]
 * (coordinates relative to the disk centre): the integral over X of the length
 * of [b0,b1] cut by the chord [-h(X), h(X)], h = sqrt(r^2 - X^2), taken piece by
 * piece between the points where h meets |b0| or |b1|. */
double orc_cell_area(double a0, double a1, double b0, double b1, double r)
{
    double A = fmax(a0, -r), B = fmin(a1, r);
    if (!(A < B))
        return 0.0;
    double bp[6];
    int nb = 0;
    bp[nb++] = A;
    bp[nb++] = B;
    const double lev[2] = {b0, b1};
    for (int k = 0; k < 2; ++k) {
        double c = fabs(lev[k]);
        if (c < r) {
            double s = sqrt(r * r - c * c);
            if (s > A && s < B) bp[nb++] = s;
            if (-s > A && -s < B) bp[nb++] = -s;
        }
    }
    qsort(bp, (size_t)nb, sizeof(double), cmp_double);
    double area = 0.0;
    for (int k = 0; k + 1 < nb; ++k) {
        double p = bp[k], q = bp[k + 1];
        if (!(q > p))
            continue;
        double xm = 0.5 * (p + q);
        double hm = sqrt(fmax(0.0, r * r - xm * xm));
        int upper_is_arc = hm < b1;     /* top of the chord inside the strip */
        int lower_is_arc = -hm > b0;    /* bottom of the chord inside the strip */
        double top = upper_is_arc ? hm : b1;
        double bot = lower_is_arc ? -hm : b0;
        if (!(top > bot))
            continue;
        double hint = half_chord_prim(q, r) - half_chord_prim(p, r);
        double up = upper_is_arc ? hint : b1 * (q - p);
        double lo = lower_is_arc ? -hint : b0 * (q - p);
        area += up - lo;
    }
    return area;
}

/* Cell decomposition of Sec. 2.3 (Fig. 3b) in 2D: n x n sub-cells, a sub-cell
 * counts as solid when its centre lies in the disk (a tie counts as inside).
 * Decided in single precision, operation for operation as the kernel does. */
double orc_eps_subcell(float lox, float loy, float r, int n)
{
    float r2 = r * r;
    int inside = 0;
    for (int ky = 0; ky < n; ++ky) {
        float ty = ((float)ky + 0.5f) / (float)n;
        float py = loy + ty;
        for (int kx = 0; kx < n; ++kx) {
            float tx = ((float)kx + 0.5f) / (float)n;
            float px = lox + tx;
            float d2 = px * px + py * py;
            if (d2 <= r2)
                inside++;
        }
    }
    return (double)inside / (double)(n * n);
}

/* Does the disk of radius r reach into the open unit cell whose lower-left
 * corner is (lox, loy) relative to the disk centre?  Nearest point of the cell
 * to the centre, strictly inside the circle.  Single precision, every
 * operation rounded separately. */
int orc_covers(float lox, float loy, float r)
{
    float hix = lox + 1.0f, hiy = loy + 1.0f;
    float dx = lox > 0.0f ? lox : (hix < 0.0f ? hix : 0.0f);
    float dy = loy > 0.0f ? loy : (hiy < 0.0f ? hiy : 0.0f);
    float d2 = dx * dx + dy * dy;
    return d2 < r * r;
}

/* Solid collision operator, Eq. 12:
 * Omega^s_i = f_{-i} - f^eq_{-i}(rho, u_f) + f^eq_i(rho, u_s) - f_i. */
void orc_omega_s(const double *f9, double rho, double ux, double uy, double usx, double usy,
                 double *om)
{
    double fe[9], fes[9];
    orc_feq(rho, ux, uy, fe);
    orc_feq(rho, usx, usy, fes);
    for (int q = 0; q < 9; ++q)
        om[q] = f9[OPP[q]] - fe[OPP[q]] + fes[q] - f9[q];
}

/* --------------------------------------------------------- simulation */
static void stream(orc_sim *s)
{
    const int nx = s->p.nx, ny = s->p.ny;
    /* every (direction, destination) is written by one source cell, so rows run in parallel */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int k = 0; k < ny; ++k)
        for (int i = 0; i < nx; ++i)
            for (int q = 0; q < 9; ++q) {
                double v = s->fs[IDX(s, q, k, i)];
                int xn = i + CX[q], yn = k + CY[q];
                if (yn < 0 || yn >= ny) {
                    if (s->p.bc_y == ORC_PERIODIC) {
                        yn = (yn + ny) % ny;
                    } else { /* halfway bounce-back at y = 0 and y = ny; a wall moving along x
                              * returns the population with the momentum term
                              * -2 w_q rho_w (c_q . u_w) / c_s^2, rho_w = 1 */
                        const double uw = yn < 0 ? s->p.wall_u_bot : s->p.wall_u_top;
                        s->f[IDX(s, OPP[q], k, i)] = v - 6.0 * W[q] * CX[q] * uw;
                        continue;
                    }
                }
                if (xn < 0 || xn >= nx) {
                    if (s->p.bc_x == ORC_PERIODIC) {
                        xn = (xn + nx) % nx;
                    } else if (s->p.bc_x == ORC_WALL) {
                        s->f[IDX(s, OPP[q], k, i)] = v;
                        continue;
                    } else {
                        continue; /* leaves through inlet/outlet; columns rebuilt below */
                    }
                }
                s->f[IDX(s, q, yn, xn)] = v;
            }
    if (s->p.bc_x == ORC_INLET_OUTLET) {
        /* inlet column x = 0: equilibrium at the prescribed velocity with the
         * density of the first interior column; outlet column x = nx-1:
         * equilibrium at the reference density 1 with the velocity of column nx-2
         * (zero velocity gradient).  The outlet holds the pressure level: with a
         * velocity inlet, copying every population of column nx-2 leaves the
         * density free and the channel's mass drifts without bound. */
        for (int k = 0; k < ny; ++k) {
            double rho1 = 0.0, fe[9], fo[9], ro = 0.0, jox = 0.0, joy = 0.0;
            for (int q = 0; q < 9; ++q) {
                const double g = s->f[IDX(s, q, k, nx - 2)];
                rho1 += s->f[IDX(s, q, k, 1)];
                ro += g;
                jox += CX[q] * g;
                joy += CY[q] * g;
            }
            orc_feq(rho1, s->p.u_in_x, s->p.u_in_y, fe);
            orc_feq(1.0, jox / ro, joy / ro, fo);
            for (int q = 0; q < 9; ++q) {
                s->f[IDX(s, q, k, 0)] = fe[q];
                s->f[IDX(s, q, k, nx - 1)] = fo[q];
            }
        }
    }
}

orc_sim *orc_new(const orc_params *p)
{
    if (p->nx < 3 || p->ny < 3 || !(p->tau > 0.5) || p->C_smag < 0.0)
        return NULL;
    if (p->contact_model < 0 || p->contact_model > 1 ||
        (p->contact_model == 1 && !(p->E_young > 0.0 && p->nu_poisson >= 0.0 && p->nu_poisson < 0.5)))
        return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    size_t n = (size_t)9 * p->nx * p->ny;
    s->f = (double *)calloc(n, sizeof(double));
    s->fs = (double *)calloc(n, sizeof(double));
    s->cnt = (int *)calloc((size_t)p->nx * p->ny, sizeof(int));
    s->ids = (int *)calloc((size_t)p->nx * p->ny * ORC_MAX_SLOTS, sizeof(int));
    s->eps = (double *)calloc((size_t)p->nx * p->ny * ORC_MAX_SLOTS, sizeof(double));
    s->fterm = (double *)calloc((size_t)p->nx * p->ny * ORC_MAX_SLOTS * 3, sizeof(double));
    s->fns = (int *)calloc((size_t)p->nx * p->ny, sizeof(int));
    double le = log(p->e_rest > 0.0 ? p->e_rest : 1.0);
    s->zeta = -le / sqrt(M_PI * M_PI + le * le);
    {   /* Hertz-Mindlin constants, identical materials: E* = E / (2 (1 - nu^2)),
         * G* = E / (4 (2 - nu)(1 + nu)) */
        const double E = p->E_young, nu = p->nu_poisson;
        const double Es = E / (2.0 * (1.0 - nu * nu));
        const double Gs = E / (4.0 * (2.0 - nu) * (1.0 + nu));
        s->hm_kn0 = 4.0 / 3.0 * Es;
        s->hm_sn0 = 2.0 * Es;
        s->hm_kt0 = 8.0 * Gs;
        s->hm_c0 = 2.0 * sqrt(5.0 / 6.0) * s->zeta;
    }
    s->gx_eff = (1.0 - 1.0 / p->rho_s) * p->gx;
    s->gy_eff = (1.0 - 1.0 / p->rho_s) * p->gy;
    /* initial condition: the post-collision field is f^eq(rho0, u0); streaming
     * it once (with the boundary rules) gives f(x, 0) */
    double fe[9];
    orc_feq(p->rho0, p->ux0, p->uy0, fe);
    for (int q = 0; q < 9; ++q)
        for (size_t c = 0; c < (size_t)p->nx * p->ny; ++c)
            s->fs[(size_t)q * p->nx * p->ny + c] = fe[q];
    stream(s);
    return s;
}

static void free_particles(orc_sim *s)
{
    free(s->px); free(s->py); free(s->vx); free(s->vy); free(s->w); free(s->r);
    free(s->m); free(s->I); free(s->Ffx); free(s->Ffy); free(s->Tf); free(s->xi); free(s->xiw);
    s->px = s->py = s->vx = s->vy = s->w = s->r = s->m = s->I = NULL;
    s->Ffx = s->Ffy = s->Tf = s->xi = s->xiw = NULL;
    s->np = 0;
}

void orc_free(orc_sim *s)
{
    if (!s) return;
    free_particles(s);
    free(s->f); free(s->fs); free(s->cnt); free(s->ids); free(s->eps); free(s->fterm); free(s->fns);
    free(s);
}

int orc_set_particles(orc_sim *s, int n, const double *x, const double *v, const double *w,
                      const double *r)
{
    free_particles(s);
    s->np = n;
    if (n == 0) return 0;
    s->px = malloc(n * sizeof(double)); s->py = malloc(n * sizeof(double));
    s->vx = malloc(n * sizeof(double)); s->vy = malloc(n * sizeof(double));
    s->w = malloc(n * sizeof(double)); s->r = malloc(n * sizeof(double));
    s->m = malloc(n * sizeof(double)); s->I = malloc(n * sizeof(double));
    s->Ffx = calloc(n, sizeof(double)); s->Ffy = calloc(n, sizeof(double));
    s->Tf = calloc(n, sizeof(double));
    s->xi = calloc((size_t)n * n, sizeof(double));
    s->xiw = calloc((size_t)n * 4, sizeof(double));
    for (int p = 0; p < n; ++p) {
        if (!(r[p] > 0.0)) return -1;
        s->px[p] = x[2 * p]; s->py[p] = x[2 * p + 1];
        s->vx[p] = v[2 * p]; s->vy[p] = v[2 * p + 1];
        s->w[p] = w[p]; s->r[p] = r[p];
        /* disk of unit depth: m = rho_s pi r^2, I = m r^2 / 2 */
        s->m[p] = s->p.rho_s * M_PI * r[p] * r[p];
        s->I[p] = 0.5 * s->m[p] * r[p] * r[p];
    }
    return 0;
}

/* ---------------------------------------------------------------- DEM */
/* Spring-dashpot contact between particle a and a partner seen from a (Eqs. 7-9).
 * n points from a to the partner, t = z x n.  dvx,dvy is the partner's
 * translational velocity minus a's; rot = w_a r_a + w_b r_b; R* and m* the pair's
 * reduced radius and mass.  Linear law: constant k_n, k_t, c_n = 2 zeta sqrt(m* k_n),
 * c_t = ct_ratio c_n.  Simplified Hertz-Mindlin (the paper's law, Sec. 2.2, after di
 * Renzo and di Maio): with s = sqrt(R* delta), k_n = 4/3 E* s, k_t = 8 G* s and the
 * dashpots 2 sqrt(5/6) |beta| sqrt(S m*) for S_n = 2 E* s and S_t = 8 G* s, where
 * |beta| = zeta.  Returns the force on a (fx, fy) and the tangential force magnitude Ft
 * (the torque on each side is its own radius times Ft). */
static void contact_law(const orc_sim *s, double nxv, double nyv, double delta, double dvx,
                        double dvy, double rot, double Rstar, double mstar, double dt, double *xi,
                        double *fx, double *fy, double *Ft_out)
{
    double tx = -nyv, ty = nxv;
    double vn = dvx * nxv + dvy * nyv;
    double vt = (dvx * tx + dvy * ty) - rot;
    double kn, kt, cn, ct;
    if (s->p.contact_model == 1) {
        double sq = sqrt(Rstar * delta);
        kn = s->hm_kn0 * sq;
        kt = s->hm_kt0 * sq;
        cn = s->hm_c0 * sqrt(s->hm_sn0 * sq * mstar);
        ct = s->hm_c0 * sqrt(s->hm_kt0 * sq * mstar);
    } else {
        kn = s->p.kn;
        kt = s->p.kt;
        cn = 2.0 * s->zeta * sqrt(mstar * s->p.kn);
        ct = s->p.ct_ratio * cn;
    }
    *xi = *xi + vt * dt;                      /* incremental spring of Eq. 9 */
    double Fn = kn * delta - cn * vn;         /* Eq. 8, repulsive when positive */
    double Ft = kt * *xi + ct * vt;           /* Eq. 9 */
    double lim = s->p.mu * fabs(Fn);          /* Coulomb cap */
    if (fabs(Ft) > lim) {
        Ft = copysign(lim, Ft);
        *xi = copysign(lim / kt, *xi);
    }
    *fx = -Fn * nxv + Ft * tx;
    *fy = -Fn * nyv + Ft * ty;
    *Ft_out = Ft;
}

static double min_image(double d, int periodic, int L)
{
    if (periodic) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

static void dem_substep(orc_sim *s, double dt, double *Fcx, double *Fcy, double *Tc)
{
    const int n = s->np;
    const int perx = s->p.bc_x == ORC_PERIODIC, pery = s->p.bc_y == ORC_PERIODIC;
    for (int p = 0; p < n; ++p) Fcx[p] = Fcy[p] = Tc[p] = 0.0;
    /* particle-particle, brute force over all pairs a < b */
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            double dx = min_image(s->px[b] - s->px[a], perx, s->p.nx);
            double dy = min_image(s->py[b] - s->py[a], pery, s->p.ny);
            double d2 = dx * dx + dy * dy;
            double R = s->r[a] + s->r[b];
            double *xi = &s->xi[(size_t)a * n + b];
            if (!(d2 < R * R)) { /* Eq. 7: no overlap, the spring is released */
                *xi = 0.0;
                continue;
            }
            double d = sqrt(d2);
            double nxv = dx / d, nyv = dy / d;
            double delta = R - d;
            double mstar = s->m[a] * s->m[b] / (s->m[a] + s->m[b]);
            double Rstar = s->r[a] * s->r[b] / (s->r[a] + s->r[b]);
            double rot = s->w[a] * s->r[a] + s->w[b] * s->r[b];
            double fx, fy, Ft;
            contact_law(s, nxv, nyv, delta, s->vx[b] - s->vx[a], s->vy[b] - s->vy[a], rot, Rstar, mstar,
                        dt, xi, &fx, &fy, &Ft);
            Fcx[a] += fx; Fcy[a] += fy; Tc[a] += s->r[a] * Ft;
            Fcx[b] -= fx; Fcy[b] -= fy; Tc[b] += s->r[b] * Ft;
        }
    /* particle-wall: walls on the domain edges, an immovable partner of
     * infinite mass (m* = m) */
    for (int p = 0; p < n; ++p)
        for (int wl = 0; wl < 4; ++wl) {
            int active = (wl < 2) ? s->p.bc_x == ORC_WALL : s->p.bc_y == ORC_WALL;
            if (!active) continue;
            double dist, nxv, nyv;
            switch (wl) {
            case 0: dist = s->px[p]; nxv = -1.0; nyv = 0.0; break;
            case 1: dist = (double)s->p.nx - s->px[p]; nxv = 1.0; nyv = 0.0; break;
            case 2: dist = s->py[p]; nxv = 0.0; nyv = -1.0; break;
            default: dist = (double)s->p.ny - s->py[p]; nxv = 0.0; nyv = 1.0; break;
            }
            double *xi = &s->xiw[(size_t)p * 4 + wl];
            if (!(dist < s->r[p])) {
                *xi = 0.0;
                continue;
            }
            double delta = s->r[p] - dist;
            double fx, fy, Ft;
            contact_law(s, nxv, nyv, delta, -s->vx[p], -s->vy[p], s->w[p] * s->r[p], s->r[p], s->m[p], dt,
                        xi, &fx, &fy, &Ft);
            Fcx[p] += fx; Fcy[p] += fy; Tc[p] += s->r[p] * Ft;
        }
    /* Eqs. 10-11, leapfrog: kick with a(x^n), then drift with v^{n+1/2} */
    for (int p = 0; p < n; ++p) {
        double ax = (Fcx[p] + s->Ffx[p]) / s->m[p] + s->gx_eff;
        double ay = (Fcy[p] + s->Ffy[p]) / s->m[p] + s->gy_eff;
        double al = (Tc[p] + s->Tf[p]) / s->I[p];
        s->vx[p] = s->vx[p] + ax * dt;
        s->vy[p] = s->vy[p] + ay * dt;
        s->w[p] = s->w[p] + al * dt;
        s->px[p] = s->px[p] + s->vx[p] * dt;
        s->py[p] = s->py[p] + s->vy[p] * dt;
        if (perx) {
            if (s->px[p] >= s->p.nx) s->px[p] -= s->p.nx;
            else if (s->px[p] < 0.0) s->px[p] += s->p.nx;
        }
        if (pery) {
            if (s->py[p] >= s->p.ny) s->py[p] -= s->p.ny;
            else if (s->py[p] < 0.0) s->py[p] += s->p.ny;
        }
    }
}

int orc_dem_substeps(orc_sim *s, int nsub)
{
    if (s->np == 0 || nsub <= 0) return 0;
    double dt = 1.0 / (double)s->p.N_sub;
    double *Fcx = malloc(s->np * sizeof(double));
    double *Fcy = malloc(s->np * sizeof(double));
    double *Tc = malloc(s->np * sizeof(double));
    for (int k = 0; k < nsub; ++k)
        dem_substep(s, dt, Fcx, Fcy, Tc);
    free(Fcx); free(Fcy); free(Tc);
    return 0;
}

/* ------------------------------------------------ map particles (Sec. 2.4) */
/* Particle p seen from cell (i,k): lower-left corner of the cell relative to
 * the centre in single precision, decided from the integer cell of the centre
 * and the fractional offset, with the minimum image in periodic directions. */
static int rel_index(int i, int ci, int periodic, int L)
{
    int d = i - ci;
    if (periodic) {
        while (d >= L / 2) d -= L;
        while (d < -(L / 2)) d += L;
    }
    return d;
}

static int map_particles(orc_sim *s)
{
    const int nx = s->p.nx, ny = s->p.ny;
    const int perx = s->p.bc_x == ORC_PERIODIC, pery = s->p.bc_y == ORC_PERIODIC;
    memset(s->cnt, 0, sizeof(int) * (size_t)nx * ny);
    int overflow = 0;
    for (int p = 0; p < s->np; ++p) {
        double cx = s->px[p], cy = s->py[p], r = s->r[p];
        int ci = (int)floor(cx), cj = (int)floor(cy);
        float fx = (float)(cx - ci), fy = (float)(cy - cj);
        float rf = (float)r;
        int span = (int)ceil(r) + 2;
        for (int dk = -span; dk <= span; ++dk)
            for (int di = -span; di <= span; ++di) {
                int i = ci + di, k = cj + dk;
                if (perx) i = ((i % nx) + nx) % nx;
                else if (i < 0 || i >= nx) continue;
                if (pery) k = ((k % ny) + ny) % ny;
                else if (k < 0 || k >= ny) continue;
                int ri = rel_index(i, ci, perx, nx), rk = rel_index(k, cj, pery, ny);
                float lox = (float)ri - fx, loy = (float)rk - fy;
                if (!orc_covers(lox, loy, rf))
                    continue;
                double e;
                if (s->p.eps_mode == ORC_EPS_SUBCELL) {
                    e = orc_eps_subcell(lox, loy, rf, s->p.n_sub);
                } else {
                    double a0 = (double)ri - (cx - ci), b0 = (double)rk - (cy - cj);
                    e = orc_cell_area(a0, a0 + 1.0, b0, b0 + 1.0, r);
                }
                size_t c = (size_t)k * nx + i;
                int slot = s->cnt[c];
                /* a cell can be listed for the same particle once only; the
                 * periodic wrap of a small lattice could revisit it */
                int dup = 0;
                for (int t = 0; t < slot; ++t)
                    if (s->ids[c * ORC_MAX_SLOTS + t] == p) dup = 1;
                if (dup) continue;
                if (slot >= ORC_MAX_SLOTS) {
                    overflow = 1;
                    continue;
                }
                s->ids[c * ORC_MAX_SLOTS + slot] = p;
                s->eps[c * ORC_MAX_SLOTS + slot] = e;
                s->cnt[c] = slot + 1;
            }
    }
    return overflow ? -2 : 0;
}

/* ------------------------------------------------------------ collide */
static void collide(orc_sim *s)
{
    const int nx = s->p.nx, ny = s->p.ny;
    const int perx = s->p.bc_x == ORC_PERIODIC, pery = s->p.bc_y == ORC_PERIODIC;
    const double Fx = s->p.Fx, Fy = s->p.Fy;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int k = 0; k < ny; ++k)
        for (int i = 0; i < nx; ++i) {
            double f[9], fe[9], fo[9];
            for (int q = 0; q < 9; ++q) f[q] = s->f[IDX(s, q, k, i)];
            double rho, ux, uy;
            moments(f, Fx, Fy, &rho, &ux, &uy);
            orc_feq(rho, ux, uy, fe);
            double te = orc_tau_eff(f, Fx, Fy, s->p.tau, s->p.C_smag);
            size_t c = (size_t)k * nx + i;
            int nc = s->cnt[c];
            double esum = 0.0;
            for (int t = 0; t < nc; ++t) esum += s->eps[c * ORC_MAX_SLOTS + t];
            double B = 0.0;
            if (nc > 0 && esum > 0.0)
                B = orc_B(esum < 1.0 ? esum : 1.0, te);   /* Eq. 14 with tau_eff */
            for (int q = 0; q < 9; ++q) {
                double omf = -(f[q] - fe[q]) / te;          /* Eq. 1 RHS */
                double cmu_x = CX[q] - ux, cmu_y = CY[q] - uy;
                double cu = CX[q] * ux + CY[q] * uy;
                /* Guo forcing term, switched off inside solids with (1 - B) */
                double S = (1.0 - 0.5 / te) * W[q] *
                           (3.0 * (cmu_x * Fx + cmu_y * Fy) + 9.0 * cu * (CX[q] * Fx + CY[q] * Fy));
                fo[q] = f[q] + (1.0 - B) * (omf + S);       /* Eq. 13, fluid part */
            }
            s->fns[c] = B > 0.0 ? nc : 0;
            for (int t = 0; t < nc && B > 0.0; ++t) {
                int p = s->ids[c * ORC_MAX_SLOTS + t];
                double Bp = B * s->eps[c * ORC_MAX_SLOTS + t] / esum;
                /* lever arm from the particle centre to the node (Eq. 16) */
                double dx = min_image((i + 0.5) - s->px[p], perx, nx);
                double dy = min_image((k + 0.5) - s->py[p], pery, ny);
                double usx = s->vx[p] - s->w[p] * dy;    /* u_s = v + w z x (x_j - x_s) */
                double usy = s->vy[p] + s->w[p] * dx;
                double om[9];
                orc_omega_s(f, rho, ux, uy, usx, usy, om);
                double mx = 0.0, my = 0.0;
                for (int q = 0; q < 9; ++q) {
                    fo[q] += Bp * om[q];                    /* Eq. 13, solid part */
                    mx += om[q] * CX[q];
                    my += om[q] * CY[q];
                }
                /* Eq. 15: B sum_i Omega^s_i c_i is the momentum the fluid gains
                 * in this cell; the particle receives the opposite */
                double fpx = -Bp * mx, fpy = -Bp * my;
                double *ft = s->fterm + (c * ORC_MAX_SLOTS + t) * 3;
                ft[0] = fpx;
                ft[1] = fpy;
                ft[2] = dx * fpy - dy * fpx;                /* Eq. 16 */
            }
            for (int q = 0; q < 9; ++q) s->fs[IDX(s, q, k, i)] = fo[q];
        }
    /* each particle's force and torque: its cells' terms summed in row-major order */
    for (int p = 0; p < s->np; ++p) s->Ffx[p] = s->Ffy[p] = s->Tf[p] = 0.0;
    for (size_t c = 0; c < (size_t)nx * ny; ++c)
        for (int t = 0; t < s->fns[c]; ++t) {
            const int p = s->ids[c * ORC_MAX_SLOTS + t];
            const double *ft = s->fterm + (c * ORC_MAX_SLOTS + t) * 3;
            s->Ffx[p] += ft[0];
            s->Ffy[p] += ft[1];
            s->Tf[p] += ft[2];
        }
}

int orc_step(orc_sim *s, int nsteps)
{
    for (int t = 0; t < nsteps; ++t) {
        if (s->p.dem_on && s->np > 0)
            orc_dem_substeps(s, s->p.N_sub);
        int rc = map_particles(s);
        if (rc) return rc;
        collide(s);
        stream(s);
    }
    return 0;
}

/* ---------------------------------------------------------- readback */
void orc_get_f(const orc_sim *s, double *f)
{
    memcpy(f, s->f, sizeof(double) * 9 * (size_t)s->p.nx * s->p.ny);
}

void orc_set_f(orc_sim *s, const double *f)
{
    memcpy(s->f, f, sizeof(double) * 9 * (size_t)s->p.nx * s->p.ny);
}

void orc_get_macro(const orc_sim *s, double *rho, double *ux, double *uy)
{
    for (int k = 0; k < s->p.ny; ++k)
        for (int i = 0; i < s->p.nx; ++i) {
            double f[9], r, u, v;
            for (int q = 0; q < 9; ++q) f[q] = s->f[IDX(s, q, k, i)];
            moments(f, s->p.Fx, s->p.Fy, &r, &u, &v);
            size_t c = (size_t)k * s->p.nx + i;
            rho[c] = r; ux[c] = u; uy[c] = v;
        }
}

void orc_get_forces(const orc_sim *s, double *F, double *T)
{
    for (int p = 0; p < s->np; ++p) {
        F[2 * p] = s->Ffx[p]; F[2 * p + 1] = s->Ffy[p]; T[p] = s->Tf[p];
    }
}

void orc_set_forces(orc_sim *s, const double *F, const double *T)
{
    for (int p = 0; p < s->np; ++p) {
        s->Ffx[p] = F[2 * p]; s->Ffy[p] = F[2 * p + 1]; s->Tf[p] = T[p];
    }
}

void orc_get_particles(const orc_sim *s, double *x, double *v, double *w)
{
    for (int p = 0; p < s->np; ++p) {
        x[2 * p] = s->px[p]; x[2 * p + 1] = s->py[p];
        v[2 * p] = s->vx[p]; v[2 * p + 1] = s->vy[p];
        w[p] = s->w[p];
    }
}

int orc_cell_map(orc_sim *s, int *count, int *ids, double *eps)
{
    int rc = map_particles(s);
    size_t n = (size_t)s->p.nx * s->p.ny;
    memcpy(count, s->cnt, n * sizeof(int));
    for (size_t c = 0; c < n; ++c)
        for (int t = 0; t < ORC_MAX_SLOTS; ++t) {
            int valid = t < s->cnt[c];
            ids[c * ORC_MAX_SLOTS + t] = valid ? s->ids[c * ORC_MAX_SLOTS + t] : -1;
            eps[c * ORC_MAX_SLOTS + t] = valid ? s->eps[c * ORC_MAX_SLOTS + t] : 0.0;
        }
    return rc;
}

int orc_contacts(const orc_sim *s, int max_pairs, int *pairs)
{
    const int perx = s->p.bc_x == ORC_PERIODIC, pery = s->p.bc_y == ORC_PERIODIC;
    int k = 0;
    for (int a = 0; a < s->np; ++a)
        for (int b = a + 1; b < s->np; ++b) {
            double dx = min_image(s->px[b] - s->px[a], perx, s->p.nx);
            double dy = min_image(s->py[b] - s->py[a], pery, s->p.ny);
            double d2 = dx * dx + dy * dy;
            double R = s->r[a] + s->r[b];
            if (d2 < R * R) {
                if (k < max_pairs) { pairs[2 * k] = a; pairs[2 * k + 1] = b; }
                k++;
            }
        }
    return k;
}

/* Uniform bins of edge `bin` cells over [0,nx) x [0,ny): bin of a particle =
 * (floor(x/bin), floor(y/bin)); ids listed per bin in ascending order. */
int orc_bins(const orc_sim *s, int bin, int *bin_start, int *bin_ids)
{
    int nbx = (s->p.nx + bin - 1) / bin, nby = (s->p.ny + bin - 1) / bin;
    int nb = nbx * nby;
    for (int b = 0; b <= nb; ++b) bin_start[b] = 0;
    int *which = malloc(sizeof(int) * (s->np > 0 ? s->np : 1));
    for (int p = 0; p < s->np; ++p) {
        int bx = (int)floor(s->px[p] / bin), by = (int)floor(s->py[p] / bin);
        if (bx < 0) bx = 0;
        if (bx >= nbx) bx = nbx - 1;
        if (by < 0) by = 0;
        if (by >= nby) by = nby - 1;
        which[p] = by * nbx + bx;
        bin_start[which[p] + 1]++;
    }
    for (int b = 0; b < nb; ++b) bin_start[b + 1] += bin_start[b];
    int *fill = calloc((size_t)nb, sizeof(int));
    for (int p = 0; p < s->np; ++p) {
        int b = which[p];
        bin_ids[bin_start[b] + fill[b]++] = p;
    }
    free(fill);
    free(which);
    return nb;
}

double orc_wall_contact_xi(const orc_sim *s, int p, int wall)
{
    return s->xiw[(size_t)p * 4 + wall];
}

/* ------------------------------------------------------------ adjoint
 * Gradient of the time-averaged drag J = (1/T) sum_{t<T} sum_p F_x,p(t) of T
 * steps taken from the current state, with respect to the inlet velocity, the
 * relaxation time and the particle centres, by reverse-mode differentiation of
 * the steps above (the chain rule through collide and stream in reverse order).
 * Scope: fixed particles (DEM off, v = w = 0, so u_s = 0 in Eq. 12), plain BGK
 * (C_smag = 0), no body force, exact-area solid ratio.  Then the solid term
 * summed over a cell's particles is B (f_{-i} - f^eq_{-i}(rho, u) + w_i rho - f_i)
 * (Eqs. 12-13 with sum_p B_p = B), the cell's drag is B j_x (Eq. 15 with
 * sum_i c_i Omega^s_i = -j), and J depends on the particle positions only through
 * the summed solid ratio E of each cell (Eq. 14). */

/* vertical chord of the disk (centre at the origin, radius r) on the line x = a,
 * clipped to [b0, b1] */
static double chord_len(double a, double b0, double b1, double r)
{
    if (!(fabs(a) < r)) return 0.0;
    double h = sqrt(r * r - a * a);
    double lo = fmax(b0, -h), hi = fmin(b1, h);
    return hi > lo ? hi - lo : 0.0;
}

/* adjoint of stream(): lam holds d J / d f(t+1) on entry (modified), lamg gets
 * d J / d f*(t); fn is f(t+1) (for the inlet density) */
static void stream_adjoint(const orc_sim *s, double *lam, const double *fn, double *lamg, double *g_uin)
{
    const int nx = s->p.nx, ny = s->p.ny;
    if (s->p.bc_x == ORC_INLET_OUTLET) {
        const double ux = s->p.u_in_x, uy = s->p.u_in_y, usq = ux * ux + uy * uy;
        for (int k = 0; k < ny; ++k) {
            /* outlet: f(nx-1) = f^eq(1, u) with u = j / rho of f(nx-2); d f^eq_q / d u =
             * w_q (3 c_q + 9 (c_q . u) c_q - 3 u) and d u / d f_p(nx-2) = (c_p - u) / rho */
            double ro = 0.0, jox = 0.0, joy = 0.0;
            for (int q = 0; q < 9; ++q) {
                const double g = fn[IDX(s, q, k, nx - 2)];
                ro += g;
                jox += CX[q] * g;
                joy += CY[q] * g;
            }
            const double uox = jox / ro, uoy = joy / ro;
            double gx = 0.0, gy = 0.0;
            for (int q = 0; q < 9; ++q) {
                const double cu = CX[q] * uox + CY[q] * uoy, l = lam[IDX(s, q, k, nx - 1)];
                gx += l * W[q] * (3.0 * CX[q] + 9.0 * cu * CX[q] - 3.0 * uox);
                gy += l * W[q] * (3.0 * CY[q] + 9.0 * cu * CY[q] - 3.0 * uoy);
                lam[IDX(s, q, k, nx - 1)] = 0.0;
            }
            for (int q = 0; q < 9; ++q)
                lam[IDX(s, q, k, nx - 2)] += (gx * (CX[q] - uox) + gy * (CY[q] - uoy)) / ro;
            /* inlet: f(0) = f^eq(rho1, u_in), rho1 = sum_q f(1) */
            double rho1 = 0.0;
            for (int q = 0; q < 9; ++q) rho1 += fn[IDX(s, q, k, 1)];
            double lr = 0.0;
            for (int q = 0; q < 9; ++q) {
                double cu = CX[q] * ux + CY[q] * uy, l0 = lam[IDX(s, q, k, 0)];
                lr += l0 * W[q] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                *g_uin += l0 * W[q] * rho1 * (3.0 * CX[q] + 9.0 * cu * CX[q] - 3.0 * ux);
                lam[IDX(s, q, k, 0)] = 0.0;
            }
            for (int q = 0; q < 9; ++q) lam[IDX(s, q, k, 1)] += lr;
        }
    }
    for (int k = 0; k < ny; ++k)
        for (int i = 0; i < nx; ++i)
            for (int q = 0; q < 9; ++q) {
                double g = 0.0;
                int xn = i + CX[q], yn = k + CY[q], wall = 0, gone = 0;
                if (yn < 0 || yn >= ny) {
                    if (s->p.bc_y == ORC_PERIODIC) yn = (yn + ny) % ny;
                    else wall = 1;
                }
                if (!wall && (xn < 0 || xn >= nx)) {
                    if (s->p.bc_x == ORC_PERIODIC) xn = (xn + nx) % nx;
                    else if (s->p.bc_x == ORC_WALL) wall = 1;
                    else gone = 1;
                }
                if (wall) g = lam[IDX(s, OPP[q], k, i)];
                else if (!gone) g = lam[IDX(s, q, yn, xn)];
                lamg[IDX(s, q, k, i)] = g;
            }
}

/* adjoint of collide() at the state f(t) = f: lamg (d J / d f*) -> lam (d J / d f),
 * plus the drag's own dependence on f; accumulates d J / d tau and d J / d E */
static void collide_adjoint(const orc_sim *s, const double *f_all, const double *lamg, double *lam,
                            double inv_T, double *g_tau, double *gE)
{
    const int nx = s->p.nx, ny = s->p.ny;
    const double tau = s->p.tau, t = tau - 0.5;
    for (int k = 0; k < ny; ++k)
        for (int i = 0; i < nx; ++i) {
            double f[9], fe[9], lg[9];
            for (int q = 0; q < 9; ++q) {
                f[q] = f_all[IDX(s, q, k, i)];
                lg[q] = lamg[IDX(s, q, k, i)];
            }
            double rho, ux, uy;
            moments(f, 0.0, 0.0, &rho, &ux, &uy);
            orc_feq(rho, ux, uy, fe);
            double jx = rho * ux, usq = ux * ux + uy * uy;
            size_t c = (size_t)k * nx + i;
            double E = 0.0;
            for (int sl = 0; sl < s->cnt[c]; ++sl) E += s->eps[c * ORC_MAX_SLOTS + sl];
            double e = E < 1.0 ? E : 1.0;
            double B = (s->cnt[c] > 0 && E > 0.0) ? orc_B(e, tau) : 0.0;
            double a = (1.0 - B) / tau;
            double lf[9], mu[9], nu = 0.0;
            for (int q = 0; q < 9; ++q) {
                lf[q] = lg[q] * (1.0 - a - B) + B * lg[OPP[q]] + inv_T * B * CX[q];
                mu[q] = a * lg[q] - B * lg[OPP[q]];
                nu += B * W[q] * lg[q];
            }
            double lr = nu, ljx = 0.0, ljy = 0.0;
            for (int q = 0; q < 9; ++q) {
                double cu = CX[q] * ux + CY[q] * uy;
                lr += mu[q] * W[q] * (1.0 - 4.5 * cu * cu + 1.5 * usq);
                ljx += mu[q] * W[q] * (3.0 * CX[q] + 9.0 * cu * CX[q] - 3.0 * ux);
                ljy += mu[q] * W[q] * (3.0 * CY[q] + 9.0 * cu * CY[q] - 3.0 * uy);
            }
            for (int q = 0; q < 9; ++q)
                lam[IDX(s, q, k, i)] = lf[q] + lr + CX[q] * ljx + CY[q] * ljy;
            double gt = 0.0;
            for (int q = 0; q < 9; ++q) gt += lg[q] * (1.0 - B) * (f[q] - fe[q]) / (tau * tau);
            if (B > 0.0) {
                double lB = inv_T * jx;
                for (int q = 0; q < 9; ++q)
                    lB += lg[q] * ((f[q] - fe[q]) / tau + (f[OPP[q]] - fe[OPP[q]] + W[q] * rho - f[q]));
                double den = (1.0 - e) + t;
                gt += lB * e * (1.0 - e) / (den * den);
                if (E < 1.0) gE[c] += lB * t * (1.0 + t) / (den * den);
            }
            *g_tau += gt;
        }
}

int orc_drag_adjoint(orc_sim *s, int T, double *J, double *dJ_duin, double *dJ_dtau, double *dJ_dx)
{
    if (T < 1 || s->p.dem_on || s->p.C_smag != 0.0 || s->p.Fx != 0.0 || s->p.Fy != 0.0 ||
        s->p.eps_mode != ORC_EPS_EXACT)
        return -3;
    for (int p = 0; p < s->np; ++p)
        if (s->vx[p] != 0.0 || s->vy[p] != 0.0 || s->w[p] != 0.0) return -3;
    const int nx = s->p.nx, ny = s->p.ny;
    const size_t N = (size_t)9 * nx * ny, NC = (size_t)nx * ny;
    int rc = map_particles(s);
    if (rc) return rc;
    /* forward, keeping f(t) of every step */
    double *tape = (double *)malloc(sizeof(double) * N * (size_t)(T + 1));
    if (!tape) return -4;
    double sum = 0.0;
    for (int t = 0; t < T; ++t) {
        memcpy(tape + (size_t)t * N, s->f, sizeof(double) * N);
        collide(s);
        for (int p = 0; p < s->np; ++p) sum += s->Ffx[p];
        stream(s);
    }
    memcpy(tape + (size_t)T * N, s->f, sizeof(double) * N);
    *J = sum / T;
    /* reverse */
    double *lam = (double *)calloc(N, sizeof(double));
    double *lamg = (double *)calloc(N, sizeof(double));
    double *gE = (double *)calloc(NC, sizeof(double));
    double g_uin = 0.0, g_tau = 0.0;
    for (int t = T - 1; t >= 0; --t) {
        stream_adjoint(s, lam, tape + (size_t)(t + 1) * N, lamg, &g_uin);
        collide_adjoint(s, tape + (size_t)t * N, lamg, lam, 1.0 / T, &g_tau, gE);
    }
    *dJ_duin = g_uin;
    *dJ_dtau = g_tau;
    /* d E / d (centre) per covered cell: chord lengths on the cell's edges */
    const int perx = s->p.bc_x == ORC_PERIODIC, pery = s->p.bc_y == ORC_PERIODIC;
    for (int p = 0; p < s->np; ++p) dJ_dx[2 * p] = dJ_dx[2 * p + 1] = 0.0;
    for (int k = 0; k < ny; ++k)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)k * nx + i;
            for (int sl = 0; sl < s->cnt[c]; ++sl) {
                int p = s->ids[c * ORC_MAX_SLOTS + sl];
                double cx = s->px[p], cy = s->py[p], r = s->r[p];
                int ci = (int)floor(cx), cj = (int)floor(cy);
                int ri = rel_index(i, ci, perx, nx), rk = rel_index(k, cj, pery, ny);
                double a0 = (double)ri - (cx - ci), b0 = (double)rk - (cy - cj);
                /* moving the centre by +d moves the cell by -d relative to the disk */
                dJ_dx[2 * p] += gE[c] * (chord_len(a0, b0, b0 + 1.0, r) - chord_len(a0 + 1.0, b0, b0 + 1.0, r));
                dJ_dx[2 * p + 1] += gE[c] * (chord_len(b0, a0, a0 + 1.0, r) - chord_len(b0 + 1.0, a0, a0 + 1.0, r));
            }
        }
    free(tape); free(lam); free(lamg); free(gE);
    return 0;
}
