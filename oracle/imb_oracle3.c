/* imb_oracle3.c -- plain FP64 CPU oracle of the 3D (D3Q19) lattice with immersed spheres.
 *
 * TEST INFRASTRUCTURE (see imb_oracle3.h).  One step, in the paper's order (Sec. 2.4 without
 * the DEM, the spheres being held): the collision of Eqs. 1-2 and 12-14 at every node from
 * f(x, t) with the forces of Eqs. 15-16, then the streaming of Eq. 1's left-hand side with
 * the boundary rules.  Written for clarity, not speed.
 */
#include "imb_oracle3.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q3 19
#define SLOTS3 4

/* Tab. 1: rest, the six face neighbours, the twelve edge neighbours; opposite pairs adjacent */
static const int C3[Q3][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double w3(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static int opp3(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

void orc3_lattice(int *c, double *w) {
    for (int q = 0; q < Q3; ++q) {
        for (int a = 0; a < 3; ++a) c[3 * q + a] = C3[q][a];
        w[q] = w3(q);
    }
}

/* Eq. 2: f^eq_q = w_q rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u) */
void orc3_feq(double rho, double ux, double uy, double uz, double *feq) {
    const double uu = ux * ux + uy * uy + uz * uz;
    for (int q = 0; q < Q3; ++q) {
        const double cu = C3[q][0] * ux + C3[q][1] * uy + C3[q][2] * uz;
        feq[q] = w3(q) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

void orc3_omega_s(const double *f, double rho, double ux, double uy, double uz, double usx, double usy, double usz,
                  double *om) {
    double fe[Q3], fs[Q3];
    orc3_feq(rho, ux, uy, uz, fe);
    orc3_feq(rho, usx, usy, usz, fs);
    for (int q = 0; q < Q3; ++q) om[q] = f[opp3(q)] - fe[opp3(q)] + fs[q] - f[q];
}

double orc3_tau_eff(const double *f, double Fx, double Fy, double Fz, double tau, double C_smag) {
    if (C_smag <= 0.0) return tau;
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < Q3; ++q) {
        rho += f[q];
        for (int d = 0; d < 3; ++d) m[d] += C3[q][d] * f[q];
    }
    const double Fb[3] = {Fx, Fy, Fz};
    double u[3], fe[Q3], P[3][3] = {{0.0}};
    for (int d = 0; d < 3; ++d) u[d] = (m[d] + 0.5 * Fb[d]) / rho;
    orc3_feq(rho, u[0], u[1], u[2], fe);
    for (int q = 0; q < Q3; ++q)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) P[a][b] += C3[q][a] * C3[q][b] * (f[q] - fe[q]);
    double Q = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Q += P[a][b] * P[a][b];
    return 0.5 * (tau + sqrt(tau * tau + 18.0 * sqrt(2.0) * C_smag * C_smag * sqrt(Q) / rho));
}

/* Sec. 2.3: the cell is cut into n x n x n sub-cells; those whose centre lies in the sphere
 * (distance <= R) count.  Offsets are formed from the integer cell offset and the centre's
 * fractional part, every operation rounded separately. */
int orc3_subcell_count(int di, int dj, int dk, double fx, double fy, double fz, double R, int n) {
    const double R2 = R * R;
    int cnt = 0;
    for (int c = 0; c < n; ++c) {
        const double tz = (double)dk + ((double)c + 0.5) / (double)n;
        const double dz = tz - fz;
        for (int b = 0; b < n; ++b) {
            const double ty = (double)dj + ((double)b + 0.5) / (double)n;
            const double dy = ty - fy;
            for (int a = 0; a < n; ++a) {
                const double tx = (double)di + ((double)a + 0.5) / (double)n;
                const double dx = tx - fx;
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 <= R2) ++cnt;
            }
        }
    }
    return cnt;
}

struct orc3_sim {
    orc3_params p;
    size_t ncell;
    double *f, *fs;       /* f(x, t) and the post-collision field */
    int np;
    double *x, *v, *w, *R, *F, *T;
    int *msph, *mcnt;     /* per cell: covering spheres and their sub-cell counts */
};

static size_t cidx(const orc3_sim *s, int i, int j, int k) {
    return ((size_t)k * s->p.ny + (size_t)j) * s->p.nx + (size_t)i;
}

static int wrapi(int a, int L) { return ((a % L) + L) % L; }

/* minimum image of a node-minus-centre component in a periodic axis */
static double min_image(double d, int L) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

static void stream(orc3_sim *s, const double *src, double *dst) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    const size_t nc = s->ncell;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t c = cidx(s, i, j, k);
                for (int q = 0; q < Q3; ++q) {
                    const int jj = j + C3[q][1];
                    if (s->p.wall_y && (jj < 0 || jj >= ny)) {
                        /* halfway bounce-back; a wall moving along x adds the momentum term
                         * -2 w_q rho_w (c_q . u_w) / c_s^2 with rho_w = 1 */
                        const double uw = jj < 0 ? s->p.wall_ux_bot : s->p.wall_ux_top;
                        dst[(size_t)opp3(q) * nc + c] = src[(size_t)q * nc + c] - 6.0 * w3(q) * C3[q][0] * uw;
                        continue;
                    }
                    const int ii = wrapi(i + C3[q][0], nx), kk = wrapi(k + C3[q][2], nz);
                    dst[(size_t)q * nc + cidx(s, ii, wrapi(jj, ny), kk)] = src[(size_t)q * nc + c];
                }
            }
}

orc3_sim *orc3_new(const orc3_params *p) {
    if (p->nx < 3 || p->ny < 3 || p->nz < 3 || !(p->tau > 0.5) || p->n_sub < 1 || !(p->C_smag >= 0.0)) return NULL;
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    s->p = *p;
    s->ncell = (size_t)p->nx * p->ny * p->nz;
    s->f = (double *)calloc(Q3 * s->ncell, sizeof(double));
    s->fs = (double *)calloc(Q3 * s->ncell, sizeof(double));
    s->msph = (int *)malloc(SLOTS3 * s->ncell * sizeof(int));
    s->mcnt = (int *)calloc(SLOTS3 * s->ncell, sizeof(int));
    for (size_t c = 0; c < SLOTS3 * s->ncell; ++c) s->msph[c] = -1;
    double fe[Q3];
    orc3_feq(p->rho0, p->ux0, p->uy0, p->uz0, fe);
    for (int q = 0; q < Q3; ++q)
        for (size_t c = 0; c < s->ncell; ++c) s->fs[(size_t)q * s->ncell + c] = fe[q];
    stream(s, s->fs, s->f);   /* f(x, 0): the streamed equilibrium */
    return s;
}

void orc3_free(orc3_sim *s) {
    if (!s) return;
    free(s->f);
    free(s->fs);
    free(s->msph);
    free(s->mcnt);
    free(s->x);
    free(s->v);
    free(s->w);
    free(s->R);
    free(s->F);
    free(s->T);
    free(s);
}

int orc3_set_spheres(orc3_sim *s, int n, const double *x, const double *v, const double *w, const double *R) {
    const int L[3] = {s->p.nx, s->p.ny, s->p.nz};
    const int per[3] = {1, !s->p.wall_y, 1};
    for (int a = 0; a < n; ++a) {
        if (!(R[a] > 0.0)) return -1;
        for (int d = 0; d < 3; ++d) {
            if (!(x[3 * a + d] >= 0.0 && x[3 * a + d] < L[d])) return -1;
            if (per[d] && 2.0 * (R[a] + 2.0) > L[d]) return -1;   /* one image per cell */
        }
    }
    free(s->x);
    free(s->v);
    free(s->w);
    free(s->R);
    free(s->F);
    free(s->T);
    s->np = n;
    s->x = (double *)malloc(3 * (size_t)(n > 0 ? n : 1) * sizeof(double));
    s->v = (double *)malloc(3 * (size_t)(n > 0 ? n : 1) * sizeof(double));
    s->w = (double *)malloc(3 * (size_t)(n > 0 ? n : 1) * sizeof(double));
    s->R = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    s->F = (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    s->T = (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    memcpy(s->x, x, 3 * (size_t)n * sizeof(double));
    memcpy(s->v, v, 3 * (size_t)n * sizeof(double));
    memcpy(s->w, w, 3 * (size_t)n * sizeof(double));
    memcpy(s->R, R, (size_t)n * sizeof(double));
    for (size_t c = 0; c < SLOTS3 * s->ncell; ++c) {
        s->msph[c] = -1;
        s->mcnt[c] = 0;
    }
    const int nsub = s->p.n_sub;
    for (int a = 0; a < n; ++a) {   /* sphere order = slot order */
        int ci[3];
        double fr[3];
        for (int d = 0; d < 3; ++d) {
            ci[d] = (int)floor(x[3 * a + d]);
            fr[d] = x[3 * a + d] - (double)ci[d];
        }
        const int span = (int)ceil(R[a]) + 1;
        for (int dk = -span; dk <= span; ++dk)
            for (int dj = -span; dj <= span; ++dj)
                for (int di = -span; di <= span; ++di) {
                    const int off[3] = {di, dj, dk};
                    int cc[3], inside = 1;
                    for (int d = 0; d < 3; ++d) {
                        cc[d] = ci[d] + off[d];
                        if (per[d]) cc[d] = wrapi(cc[d], L[d]);
                        else if (cc[d] < 0 || cc[d] >= L[d]) inside = 0;
                    }
                    if (!inside) continue;
                    const int cnt = orc3_subcell_count(di, dj, dk, fr[0], fr[1], fr[2], R[a], nsub);
                    if (cnt == 0) continue;
                    const size_t c = cidx(s, cc[0], cc[1], cc[2]);
                    int k = 0;
                    while (k < SLOTS3 && s->msph[c * SLOTS3 + k] >= 0) ++k;
                    if (k == SLOTS3) return -2;
                    s->msph[c * SLOTS3 + k] = a;
                    s->mcnt[c * SLOTS3 + k] = cnt;
                }
    }
    return 0;
}

int orc3_step(orc3_sim *s, int nsteps) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    const size_t nc = s->ncell;
    const double tau = s->p.tau, Fb[3] = {s->p.Fx, s->p.Fy, s->p.Fz};
    const double nsub3 = (double)s->p.n_sub * s->p.n_sub * s->p.n_sub;
    const int per[3] = {1, !s->p.wall_y, 1};
    const int L[3] = {nx, ny, nz};
    for (int t = 0; t < nsteps; ++t) {
        for (int a = 0; a < 3 * s->np; ++a) s->F[a] = s->T[a] = 0.0;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const size_t c = cidx(s, i, j, k);
                    double f[Q3], fe[Q3], out[Q3];
                    for (int q = 0; q < Q3; ++q) f[q] = s->f[(size_t)q * nc + c];
                    /* Eqs. 3-4 with the Guo half-force shift */
                    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
                    for (int q = 0; q < Q3; ++q) {
                        rho += f[q];
                        for (int d = 0; d < 3; ++d) m[d] += C3[q][d] * f[q];
                    }
                    double u[3];
                    for (int d = 0; d < 3; ++d) u[d] = (m[d] + 0.5 * Fb[d]) / rho;
                    orc3_feq(rho, u[0], u[1], u[2], fe);
                    /* the Smagorinsky relaxation time enters the BGK term, the forcing and B */
                    const double te = orc3_tau_eff(f, Fb[0], Fb[1], Fb[2], tau, s->p.C_smag);
                    /* solid ratio and B (Eq. 14) */
                    double esum = 0.0;
                    for (int k2 = 0; k2 < SLOTS3; ++k2)
                        if (s->msph[c * SLOTS3 + k2] >= 0) esum += s->mcnt[c * SLOTS3 + k2] / nsub3;
                    const double eps = esum < 1.0 ? esum : 1.0;
                    const double B = esum > 0.0 ? eps * (te - 0.5) / ((1.0 - eps) + (te - 0.5)) : 0.0;
                    const double uF = u[0] * Fb[0] + u[1] * Fb[1] + u[2] * Fb[2];
                    for (int q = 0; q < Q3; ++q) {
                        const double cu = C3[q][0] * u[0] + C3[q][1] * u[1] + C3[q][2] * u[2];
                        const double cF = C3[q][0] * Fb[0] + C3[q][1] * Fb[1] + C3[q][2] * Fb[2];
                        const double S = (1.0 - 0.5 / te) * w3(q) * (3.0 * (cF - uF) + 9.0 * cu * cF);
                        out[q] = f[q] + (1.0 - B) * (-(f[q] - fe[q]) / te + S);
                    }
                    if (B > 0.0) {
                        const double node[3] = {i + 0.5, j + 0.5, k + 0.5};
                        for (int k2 = 0; k2 < SLOTS3; ++k2) {
                            const int p = s->msph[c * SLOTS3 + k2];
                            if (p < 0) continue;
                            const double Bp = B * (s->mcnt[c * SLOTS3 + k2] / nsub3) / esum;
                            double r[3], us[3], om[Q3];
                            for (int d = 0; d < 3; ++d) {
                                r[d] = node[d] - s->x[3 * p + d];
                                if (per[d]) r[d] = min_image(r[d], L[d]);
                            }
                            const double *vp = s->v + 3 * p, *wp = s->w + 3 * p;
                            us[0] = vp[0] + wp[1] * r[2] - wp[2] * r[1];   /* u_s = v + w x r */
                            us[1] = vp[1] + wp[2] * r[0] - wp[0] * r[2];
                            us[2] = vp[2] + wp[0] * r[1] - wp[1] * r[0];
                            orc3_omega_s(f, rho, u[0], u[1], u[2], us[0], us[1], us[2], om);
                            double Fp[3] = {0.0, 0.0, 0.0};
                            for (int q = 0; q < Q3; ++q) {
                                out[q] += Bp * om[q];
                                for (int d = 0; d < 3; ++d) Fp[d] -= Bp * om[q] * C3[q][d];   /* Eq. 15 */
                            }
                            for (int d = 0; d < 3; ++d) s->F[3 * p + d] += Fp[d];
                            s->T[3 * p + 0] += r[1] * Fp[2] - r[2] * Fp[1];   /* Eq. 16 */
                            s->T[3 * p + 1] += r[2] * Fp[0] - r[0] * Fp[2];
                            s->T[3 * p + 2] += r[0] * Fp[1] - r[1] * Fp[0];
                        }
                    }
                    for (int q = 0; q < Q3; ++q) s->fs[(size_t)q * nc + c] = out[q];
                }
        stream(s, s->fs, s->f);
    }
    return 0;
}

void orc3_get_f(const orc3_sim *s, double *f) { memcpy(f, s->f, Q3 * s->ncell * sizeof(double)); }
void orc3_set_f(orc3_sim *s, const double *f) { memcpy(s->f, f, Q3 * s->ncell * sizeof(double)); }

void orc3_get_macro(const orc3_sim *s, double *rho, double *ux, double *uy, double *uz) {
    const size_t nc = s->ncell;
    const double Fb[3] = {s->p.Fx, s->p.Fy, s->p.Fz};
    for (size_t c = 0; c < nc; ++c) {
        double r = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q3; ++q) {
            const double fq = s->f[(size_t)q * nc + c];
            r += fq;
            for (int d = 0; d < 3; ++d) m[d] += C3[q][d] * fq;
        }
        rho[c] = r;
        ux[c] = (m[0] + 0.5 * Fb[0]) / r;
        uy[c] = (m[1] + 0.5 * Fb[1]) / r;
        uz[c] = (m[2] + 0.5 * Fb[2]) / r;
    }
}

void orc3_get_forces(const orc3_sim *s, double *F, double *T) {
    memcpy(F, s->F, 3 * (size_t)s->np * sizeof(double));
    memcpy(T, s->T, 3 * (size_t)s->np * sizeof(double));
}

int orc3_cell_map(const orc3_sim *s, int *sphere, int *count) {
    memcpy(sphere, s->msph, SLOTS3 * s->ncell * sizeof(int));
    memcpy(count, s->mcnt, SLOTS3 * s->ncell * sizeof(int));
    return 0;
}
