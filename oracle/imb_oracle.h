/*
 * imb_oracle.h -- FP64 CPU oracle of the coupled LBM-DEM step with the
 * immersed moving boundary (Yang, Jing, Kwok & Sobral, arXiv 1809.07008).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code, header, table or constant generator with the CUDA library under
 * paper_1809_07008_gb300/ and include/.
 *
 * Lattice: D2Q9 (the 2D member of the DnQm family the paper uses in Sec. 2),
 * directions 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1)
 * 7:(-1,-1) 8:(1,-1); weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
 *
 * Geometry: cell (i,k) = [i,i+1) x [k,k+1), node at its centre; walls on the
 * domain edges (halfway bounce-back).  Populations are stored [q][ny][nx].
 *
 * State exposed by orc_get_f: f(x,t) of Eq. 1, i.e. after streaming and
 * before the collision of step t.
 */
#ifndef IMB_ORACLE_H
#define IMB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_INLET_OUTLET = 2 };
enum { ORC_EPS_EXACT = 0, ORC_EPS_SUBCELL = 1 };
#define ORC_MAX_SLOTS 4

typedef struct {
    int nx, ny;
    double tau, C_smag;
    int bc_x, bc_y;
    double u_in_x, u_in_y;
    double Fx, Fy;           /* body force density on the fluid (Guo forcing) */
    double rho0, ux0, uy0;   /* initial post-collision field f* = f^eq(rho0, u0) */
    int eps_mode, n_sub;
    int dem_on, N_sub;
    double kn, kt, e_rest, ct_ratio, mu, rho_s, gx, gy;
    double wall_u_bot, wall_u_top;   /* x velocity of the walls y = 0 and y = ny (fluid rule only) */
    int contact_model;               /* 0: linear spring-dashpot, 1: simplified Hertz-Mindlin */
    double E_young, nu_poisson;      /* Hertz-Mindlin material (same for particles and walls) */
} orc_params;

typedef struct orc_sim orc_sim;

/* building blocks (each pinned by tests/test_oracle_*.py) */
void   orc_feq(double rho, double ux, double uy, double *feq9);
double orc_B(double eps, double tau);
double orc_tau_eff(const double *f9, double Fx, double Fy, double tau, double C_smag);
double orc_cell_area(double a0, double a1, double b0, double b1, double r);
double orc_eps_subcell(float lox, float loy, float r, int n);
int    orc_covers(float lox, float loy, float r);
void   orc_omega_s(const double *f9, double rho, double ux, double uy, double usx, double usy,
                   double *om9);

/* simulation */
/* host threads of the collide and stream loops (default 1); results do not depend on it */
void     orc_set_threads(int n);
orc_sim *orc_new(const orc_params *p);
void     orc_free(orc_sim *s);
int      orc_set_particles(orc_sim *s, int n, const double *x, const double *v, const double *w,
                           const double *r);
int      orc_step(orc_sim *s, int nsteps);
void     orc_get_f(const orc_sim *s, double *f);
void     orc_set_f(orc_sim *s, const double *f);
void     orc_get_macro(const orc_sim *s, double *rho, double *ux, double *uy);
void     orc_get_forces(const orc_sim *s, double *F, double *T);
void     orc_set_forces(orc_sim *s, const double *F, const double *T);
void     orc_get_particles(const orc_sim *s, double *x, double *v, double *w);
int      orc_cell_map(orc_sim *s, int *count, int *ids, double *eps);
int      orc_contacts(const orc_sim *s, int max_pairs, int *pairs);
int      orc_bins(const orc_sim *s, int bin, int *bin_start, int *bin_ids);
int      orc_dem_substeps(orc_sim *s, int nsub);
double   orc_wall_contact_xi(const orc_sim *s, int p, int wall);

/* Time-averaged drag J = (1/T) sum_{t<T} sum_p F_x,p(t) over T steps from the
 * current state (which advances by T steps) and its gradient with respect to
 * u_in_x, tau and the particle centres (dJ_dx[2p], dJ_dx[2p+1]), by reverse-mode
 * differentiation of the steps.  Scope: DEM off, particles at rest, C_smag = 0,
 * no body force, exact-area solid ratio; returns -3 outside it.  Keeps every
 * state in memory (small cases only). */
int      orc_drag_adjoint(orc_sim *s, int T, double *J, double *dJ_duin, double *dJ_dtau, double *dJ_dx);

#ifdef __cplusplus
}
#endif
#endif
