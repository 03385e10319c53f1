/* imb_oracle3.h -- plain FP64 CPU oracle of the 3D (D3Q19) lattice with immersed spheres.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU leg use it;
 * it shares no code with the CUDA library.
 *
 * The paper's own lattice (Sec. 2.1, Tab. 1): D3Q19 BGK (Eqs. 1-5) with the partially
 * saturated (Noble-Torczynski) collision of Eqs. 12-14, the solid ratio of each cell from
 * its n_sub^3 sub-cells (Sec. 2.3), and the per-sphere force and torque of Eqs. 15-16.
 * Spheres are held in place (they may carry a velocity and a spin that enter u_s).
 * Geometry: cell (i, j, k) is [i, i+1) x [j, j+1) x [k, k+1) with its node at the centre;
 * x and z periodic; y periodic or bounded by halfway bounce-back walls on the domain edges.
 * The body force enters by Guo forcing weighted by 1 - B.  With C_smag > 0 the relaxation time
 * of each node is the Smagorinsky one (tau_eff in the BGK term, the forcing and B).  A cell may
 * hold up to four spheres; B is shared between them by their solid ratios.
 * Populations are [19][nz][ny][nx].
 */
#ifndef IMB_ORACLE3_H
#define IMB_ORACLE3_H

typedef struct {
    int nx, ny, nz;
    double tau;
    int wall_y;               /* 1: walls at y = 0 and y = ny; 0: periodic in y */
    double Fx, Fy, Fz;        /* body force density */
    int n_sub;                /* sub-cells per axis for the solid ratio */
    double rho0, ux0, uy0, uz0;
    double wall_ux_bot, wall_ux_top;   /* x velocity of the walls y = 0 and y = ny */
    double C_smag;                     /* Smagorinsky constant (0: plain BGK) */
} orc3_params;

typedef struct orc3_sim orc3_sim;

/* lattice velocities c[19][3] and weights w[19] (Tab. 1); opposite of q >= 1 is q + 1 for odd q */
void orc3_lattice(int *c, double *w);
void orc3_feq(double rho, double ux, double uy, double uz, double *feq19);
/* Eq. 12 for one particle: Omega^s_q = f_{-q} - feq_{-q}(rho, u) + feq_q(rho, u_s) - f_q */
void orc3_omega_s(const double *f19, double rho, double ux, double uy, double uz, double usx, double usy,
                  double usz, double *om19);
/* Smagorinsky relaxation time of one node (the closure of the 2D path in three dimensions):
 * Pi = sum_q c_q c_q (f_q - f^eq_q), Q = Pi : Pi, tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2
 * sqrt(Q) / rho)) / 2, with u from the moments and the half-force shift */
double orc3_tau_eff(const double *f19, double Fx, double Fy, double Fz, double tau, double C_smag);
/* sub-cell centres of cell offset (di, dj, dk) from the sphere's centre cell that lie in the
 * sphere (fractional centre offset (fx, fy, fz) in [0, 1)); a centre on the surface counts */
int orc3_subcell_count(int di, int dj, int dk, double fx, double fy, double fz, double R, int n);

orc3_sim *orc3_new(const orc3_params *p);
void orc3_free(orc3_sim *s);
int orc3_set_spheres(orc3_sim *s, int n, const double *x, const double *v, const double *w, const double *R);
int orc3_step(orc3_sim *s, int nsteps);
void orc3_get_f(const orc3_sim *s, double *f);
void orc3_set_f(orc3_sim *s, const double *f);
void orc3_get_macro(const orc3_sim *s, double *rho, double *ux, double *uy, double *uz);
void orc3_get_forces(const orc3_sim *s, double *F, double *T);
/* per cell: sub-cells inside each covering sphere; sphere[cell * 4 + k] (-1 unused), count[...] */
int orc3_cell_map(const orc3_sim *s, int *sphere, int *count);

#endif
