/*
 * imblbm.h -- C ABI of the GB300 (sm_103a) coupled LBM-DEM step with the
 * immersed moving boundary of Yang, Jing, Kwok & Sobral, "A comprehensive study
 * of coupled LBM-DEM with immersed moving boundary" (arXiv 1809.07008).
 *
 * One time step, imb_step(ctx, 1), follows the coupling cycle of Sec. 2.4
 * (Fig. 4):
 *   1. DEM: N_sub sub-cycles of dt = 1/N_sub (Eq. 17) with the hydrodynamic
 *      force and torque of the previous step held fixed; linear spring-dashpot
 *      contacts (Eqs. 7-9), Newton-Euler motion (Eqs. 10-11), leapfrog Verlet;
 *   2. map the particles on the lattice (Sec. 2.4) -- per-cell solid ratio
 *      (Sec. 2.3, Fig. 3) from the exact disk/cell overlap or from n_sub x n_sub
 *      sub-cells;
 *   3. one fused D2Q9 pull-stream + collide kernel: streaming (Eq. 1 LHS),
 *      moments (Eqs. 3-4), BGK with a Smagorinsky effective relaxation time
 *      (Eq. 1 RHS, Eq. 2, Sec. 3.3), the solid operator (Eq. 12) blended by
 *      B(eps, tau) (Eqs. 13-14), and the per-particle force and torque
 *      (Eqs. 15-16) reduced in the same pass.
 *
 * Lattice units: dx = dt = 1.  Cell (i, k) is [i, i+1) x [k, k+1) with its node
 * at the centre; the domain is [0, nx) x [0, ny); walls lie on the domain edges
 * (halfway bounce-back).  D2Q9 direction order: 0:(0,0) 1:(1,0) 2:(0,1)
 * 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *
 * Sign convention of Eq. 15: the returned force is the force ON the particle,
 * minus the momentum the fluid gains through the solid operator.
 *
 * Ownership: the library allocates and owns all device memory of a context.
 * Every array argument below is a HOST pointer owned by the caller, read or
 * written synchronously before the call returns, unless stated otherwise.
 * All calls return IMB_OK (0) or a negative IMB_E_* code; imb_last_error()
 * then holds a message.  No call aborts the process.
 */
#ifndef IMBLBM_H
#define IMBLBM_H

#ifdef __cplusplus
extern "C" {
#endif

#define IMB_OK 0
#define IMB_E_INVALID_ARG (-1) /* bad size, tau <= 1/2, C_smag < 0, radius, ... */
#define IMB_E_CUDA (-2)        /* a CUDA runtime call failed                    */
#define IMB_E_NOMEM (-3)       /* device allocation failed                      */
#define IMB_E_UNSTABLE (-4)    /* NaN or |u| >= 0.3 (Mach guard, Sec. 2.1)      */
#define IMB_E_OVERFLOW (-5)    /* > 4 particles in a cell, tile or list full    */
#define IMB_E_TIMEOUT (-6)     /* a bounded wait (host or device) ran out       */
#define IMB_E_SKIN (-7)        /* a particle moved > skin/2 in one coupling cycle */
#define IMB_E_STATE (-8)       /* call out of order (e.g. no particles set)     */

enum { IMB_BC_PERIODIC = 0, IMB_BC_WALL = 1, IMB_BC_INLET_OUTLET = 2 };
enum { IMB_STORE_FP32 = 0, IMB_STORE_FP16 = 1, IMB_STORE_BF16 = 2 };
enum { IMB_EPS_EXACT = 0, IMB_EPS_SUBCELL = 1 };
enum { IMB_CONTACT_LINEAR = 0, IMB_CONTACT_HERTZ_MINDLIN = 1 };

/* Parameters of a lattice.  imb_default_params() fills every field. */
typedef struct imb_params {
    int bc_x;            /* PERIODIC, WALL, or INLET_OUTLET: inlet column x = 0 set after each
                            stream to f^eq(rho of column 1, u_in); outlet column x = nx-1 to
                            f^eq(1, u of column nx-2) (reference pressure, zero velocity
                            gradient); the walls y = 0, ny take the corners first        */
    int bc_y;            /* PERIODIC or WALL                                                  */
    double u_in_x, u_in_y; /* inlet velocity for INLET_OUTLET                                  */
    double Fx, Fy;       /* body force density on the fluid (Guo forcing); 0 = none            */
    double rho0, ux0, uy0; /* initial field: the post-collision state is f^eq(rho0, u0)        */
    int storage;         /* IMB_STORE_*: populations stored as f_i - w_i in FP32, FP16 or BF16 */
    int eps_mode;        /* IMB_EPS_EXACT (disk/cell overlap) or IMB_EPS_SUBCELL (Fig. 3b)    */
    int n_sub;           /* sub-cells per axis for IMB_EPS_SUBCELL (paper: 5)                 */
    int dem_on;          /* 1: particles move by DEM; 0: particles are fixed with the given
                            (v, omega) as the solid velocity of Eq. 12                         */
    int N_sub;           /* DEM sub-cycles per LBM step (Eq. 17; paper: 100)                  */
    double kn, kt;       /* normal / tangential spring stiffness (Eqs. 8-9)                    */
    double e_rest;       /* restitution coefficient, sets c_n = 2 zeta sqrt(m* kn)            */
    double ct_ratio;     /* c_t = ct_ratio * c_n                                               */
    double mu;           /* Coulomb friction coefficient (Eq. 9 cap)                           */
    double rho_s;        /* particle density (fluid density is 1)                              */
    double gx, gy;       /* gravity; particles feel (1 - 1/rho_s) g (buoyancy-reduced)         */
    double skin;         /* DEM neighbour-list skin in cells (default 1)                       */
    int timeout_ms;      /* bound on every host wait (default 60000)                           */
    double wall_u_bot, wall_u_top; /* x velocity of the walls y = 0 and y = ny (bc_y = WALL):
                            halfway bounce-back with the moving-wall momentum term (wall
                            density 1); the fluid sees it, DEM wall contacts see walls at
                            rest (default 0, 0)                                                */
    int contact_model;   /* IMB_CONTACT_LINEAR (kn, kt, e_rest, ct_ratio) or
                            IMB_CONTACT_HERTZ_MINDLIN: the simplified Hertz-Mindlin law the paper
                            adopts (Sec. 2.2): with s = sqrt(R* delta), k_n = 4/3 E* s, k_t = 8 G* s,
                            dashpots 2 sqrt(5/6) |beta| sqrt(S m*) (S_n = 2 E* s, S_t = 8 G* s, beta
                            from e_rest); E* = E / (2 (1 - nu^2)), G* = E / (4 (2 - nu)(1 + nu)),
                            walls of the same material; mu caps the tangential force           */
    double E_young, nu_poisson; /* Hertz-Mindlin material (E > 0, 0 <= nu < 1/2)               */
    int work_units;      /* stream-collide work: 0 (default) chooses units of eight rows, one per
                            thread block, when all of them fit on the GPU at once (lattices of
                            up to about 114 tiles of 32 x 32), else tiles handed out to a
                            persistent grid; 1 always the persistent tiles, 2 always the
                            eight-row units.  Same results either way, to rounding of the
                            force sums (each unit keeps its own partials)                      */
    int plain_launches;  /* 0 (default): imb_step / imb_step_async / imb_step_io capture a
                            coupling cycle with the DEM -- and, with kernel timing off, a run
                            of eight lattice steps without it -- as a CUDA graph the first time
                            it runs from a given pair of buffers (again after
                            imb_set_particles) and replay it with one graph launch; 1: every
                            kernel is launched by itself.  Results identical to the bit; launch
                            counts and kernel timing the same either way.  If a capture
                            fails, the context launches its kernels one by one from then on    */
} imb_params;

typedef struct imb_ctx imb_ctx;

/* Defaults: bc_x = PERIODIC, bc_y = WALL, rho0 = 1, u = 0, FP32 storage, exact eps,
 * n_sub = 5, dem_on = 0, N_sub = 100, kn = 1e5, kt = kn/2, e = 0.5, ct_ratio = 0.5,
 * mu = 0.5, rho_s = 2.65, g = 0, skin = 1, timeout 60 s. */
void imb_default_params(imb_params *p);

/* Create a lattice (Sec. 2.1).  nx, ny >= 3; tau > 1/2 (Eq. 5: nu = (tau - 1/2)/3);
 * C_smag >= 0 is the Smagorinsky constant (0 = plain BGK).  p may be NULL (defaults).
 * Allocates two population buffers of 9 planes on the current device and initialises
 * them; each plane is a frame of ny + 2 rows (the ghost rows y = -1 and ny) around the
 * lattice whose ghost cells carry the boundary rules for the pulls of the next step.
 * *out is set on success. */
int imb_init_lattice(imb_ctx **out, int nx, int ny, double tau, double C_smag,
                     const imb_params *p);

/* Set the particles (disks of unit depth), copying n centres x[2n], velocities
 * v[2n], angular velocities omega[n] and radii r[n] (FP64).  Mass rho_s pi r^2,
 * inertia m r^2 / 2.  Resets contact history and hydrodynamic forces.
 * IMB_E_INVALID_ARG if r <= 0, r > 31, a centre lies outside a non-periodic
 * domain, or (dem_on) 2 r_max + skin > 32.  n = 0 removes all particles. */
int imb_set_particles(imb_ctx *ctx, int n, const double *x, const double *v,
                      const double *omega, const double *r);

/* Overwrite positions, velocities and angular velocities of the current particles
 * (same n, radii kept) without touching contact history or forces. */
int imb_set_kinematics(imb_ctx *ctx, const double *x, const double *v, const double *omega);

/* Advance n coupling cycles (Sec. 2.4).  Kernels are queued on the context stream;
 * the call waits (bounded by timeout_ms) for them and checks the device error flags. */
int imb_step(imb_ctx *ctx, int n);

/* One host-coupled round trip: when x_in, v_in and omega_in are given (host arrays of
 * 2n, 2n and n values, as imb_set_kinematics; all three or none) they are uploaded first,
 * then n coupling cycles run, then the force F_out[2n] and torque T_out[n] of the last
 * cycle and the particle state x_out[2n], v_out[2n], omega_out[n] are read back (each
 * output may be NULL).  Everything is queued on the context stream and the call waits
 * once; for pinned host arrays the copies are asynchronous, and when every array given is
 * pinned memory the device can address (cudaHostAlloc'd or mapped), one kernel reads the
 * inputs and one writes the outputs through host memory instead.  Errors as imb_step and
 * imb_set_kinematics.  After IMB_E_TIMEOUT the copies into the output arrays may still be
 * queued: the caller must keep those arrays alive and unused until imb_sync returns
 * IMB_OK or the context is destroyed. */
int imb_step_io(imb_ctx *ctx, int n, const double *x_in, const double *v_in, const double *omega_in,
                double *F_out, double *T_out, double *x_out, double *v_out, double *omega_out);

/* Queue n coupling cycles without waiting and without reading the error flags
 * (imb_sync() does both).  Used for timing. */
int imb_step_async(imb_ctx *ctx, int n);

/* Run only the DEM part of n coupling cycles (n * N_sub sub-cycles) with the
 * current hydrodynamic force and torque held fixed. */
int imb_dem_step(imb_ctx *ctx, int n);

/* Wait (bounded) for queued work and translate the device error flags. */
int imb_sync(imb_ctx *ctx);

/* Populations f_i(x, t) of Eq. 1 -- after streaming, before the collision of the
 * next step -- as 9 * nx * ny doubles, layout [q][y][x] (x fastest, no pitch). */
int imb_get_populations(imb_ctx *ctx, double *f);

/* Macroscopic fields (Eqs. 3-4, 6) from f(x, t): density and velocity (with the
 * half-force shift of Guo forcing), each nx * ny doubles [y][x]. */
int imb_get_macro(imb_ctx *ctx, double *rho, double *ux, double *uy);

/* Hydrodynamic force F[2n] and torque T[n] on each particle (Eqs. 15-16) from the
 * last collision. */
int imb_get_forces(imb_ctx *ctx, double *F, double *T);

/* Overwrite the hydrodynamic force and torque used by the next DEM sub-cycles. */
int imb_set_forces(imb_ctx *ctx, const double *F, const double *T);

/* Particle state x[2n], v[2n], omega[n]. */
int imb_get_particles(imb_ctx *ctx, double *x, double *v, double *omega);

/* Particle-to-lattice map (Sec. 2.4) for the current positions: per cell the
 * number of covering particles count[ny*nx], their ids ids[ny*nx*4] in ascending
 * order (-1 in unused slots) and each one's solid ratio eps[ny*nx*4]. */
int imb_get_cell_map(imb_ctx *ctx, int *count, int *ids, float *eps);

/* Time-averaged drag on disks held at rest, J = (1/T) sum_{t<T} sum_p F_x,p(t) over
 * T steps from the current state (Eq. 15 forces, summed over the disks), and its
 * gradient by reverse-mode differentiation of the steps (the adjoint of the pull
 * streaming, Eq. 1, and of the collision, Eqs. 1-2 and 12-14): dJ_duin (inlet
 * velocity x component; 0 without an inlet), dJ_dtau, and dJ_dx[2n] (each disk
 * centre, through the exact overlap area of every cell it covers).  The forward
 * states are kept every `checkpoint_every` steps and the states in between
 * recomputed one segment at a time (device memory about T / checkpoint_every +
 * checkpoint_every + 4 copies of the populations, allocated for the call and freed
 * after it).  On return the lattice has advanced T steps, as imb_step(ctx, T)
 * would.  Needs DEM off, v = omega = 0, C_smag = 0, no body force, the exact solid
 * ratio and FP32 storage, else IMB_E_INVALID_ARG; IMB_E_NOMEM / IMB_E_CUDA on
 * device failures.  All pointers are host memory owned by the caller. */
int imb_drag_gradient(imb_ctx *ctx, int T, int checkpoint_every, double *J, double *dJ_duin,
                      double *dJ_dtau, double *dJ_dx);

/* The same gradient with binomial checkpointing: `snapshots` + 1 copies of the
 * populations (the start state and `snapshots` more, capped at T - 1) placed by the
 * recursive binomial schedule of imb_binomial_schedule, which recomputes the fewest
 * forward steps that memory allows (about r T for the least r with
 * C(snapshots + 1 + r, r) >= T).  Every step's drag enters J the first time the
 * schedule steps over it; the last step is taken once more to give the final
 * state.  Same requirements, outputs and errors as imb_drag_gradient; snapshots < 0
 * is IMB_E_INVALID_ARG. */
int imb_drag_gradient_binomial(imb_ctx *ctx, int T, int snapshots, double *J, double *dJ_duin,
                               double *dJ_dtau, double *dJ_dx);

/* Operations of the binomial checkpointing schedule (host only, no GPU call): the
 * reversal of T steps with `snapshots` free snapshot slots (1 .. snapshots; slot 0
 * holds the start state).  ops receives pairs (kind, argument): IMB_CK_ADVANCE n
 * (step the working state n times), IMB_CK_STORE k (copy it to slot k),
 * IMB_CK_RESTORE k (copy slot k back), IMB_CK_ADJOINT t (adjoint of step t from the
 * working state, which then holds state t).  At most max_ops pairs are written;
 * *n_ops receives the full count and *n_advances (may be NULL) the forward steps.
 * IMB_E_INVALID_ARG for T < 1, snapshots < 0 or missing outputs. */
#define IMB_CK_ADVANCE 1
#define IMB_CK_STORE 2
#define IMB_CK_RESTORE 3
#define IMB_CK_ADJOINT 4
int imb_binomial_schedule(int T, int snapshots, int *ops, int max_ops, int *n_ops, long long *n_advances);

/* ---- many independent domains (the parameter sweeps of Sec. 3 as one batch) ----
 * Each domain d is an nx[d] x ny[d] lattice, periodic in x and y, at rest at t = 0
 * (rho = 1), driven by the body force (Fx[d], Fy[d]) (Guo forcing), with relaxation
 * time tau[d] and Smagorinsky constant C_smag[d] (0: plain BGK; the closure of the
 * single-lattice path), and n_disks[d] disks held at rest: their centres are
 * disk_xy[2j], disk_xy[2j+1] in the domain's cell units and radii disk_r[j], the
 * disks of domain 0 first, then those of domain 1, and so on.  Populations are
 * stored as f - w in `storage` (IMB_STORE_*).  Every step advances all domains
 * with the collision of Eq. 13 (B of Eq. 14 from the summed exact overlap area of
 * each cell, u_s = 0) and adds each domain's drag (Eq. 15, summed over its disks)
 * to an accumulator.  The library owns the batch; host arrays are copied.
 * Returns IMB_E_INVALID_ARG for a bad size, tau <= 0.5, C_smag < 0, a disk outside its domain
 * or wider than it minus four cells, or disks x (2 ceil(r_max) + 3)^2 beyond one launch of
 * 128-thread blocks (2^31 - 1 blocks); IMB_E_NOMEM / IMB_E_CUDA on device failures
 * (then *out holds a batch to destroy, with the message in imb_batch_last_error). */
typedef struct imb_batch imb_batch;
int imb_batch_create(imb_batch **out, int n_domains, const int *nx, const int *ny, const double *tau,
                     const double *C_smag, const double *Fx, const double *Fy, const int *n_disks,
                     const double *disk_xy, const double *disk_r, int storage);

/* Advance every domain by `steps` steps (two steps at a time as a replayed CUDA graph
 * of two launches) and wait; IMB_E_UNSTABLE when a node went NaN or |u| >= 0.3. */
int imb_batch_run(imb_batch *b, int steps);

/* Time `steps_per_trial` steps of each launch shape (blocks of 128, 256 or
 * 512 threads, where the kernel can launch them; one or two cells per lane along a row) on the batch itself, keep the
 * fastest, and put the state and the drag accumulators back as they were.  Outputs
 * (each may be NULL): the chosen block size, cells per lane and its ms per step. */
int imb_batch_autotune(imb_batch *b, int steps_per_trial, int *block, int *cells_per_lane,
                       double *best_ms_per_step);

/* Set the launch shape by hand: `block` threads per block (128, 256 or 512) and
 * `cells_per_lane` (1 or 2) cells per lane along a row.  The state is unchanged.
 * IMB_E_INVALID_ARG for another value or a block the kernel cannot launch (its
 * registers); the previous shape is then kept. */
int imb_batch_set_launch(imb_batch *b, int block, int cells_per_lane);

/* Mean drag of every domain over the steps run so far: Fx_mean[n_domains],
 * Fy_mean[n_domains] (the force on the domain's disks, summed over them). */
int imb_batch_mean_drag(imb_batch *b, double *Fx_mean, double *Fy_mean);

/* f(x, t) of one domain, [9][ny][nx] in FP64 (as imb_get_populations). */
int imb_batch_get_populations(imb_batch *b, int domain, double *f);

/* Lattice cells of all domains together. */
long long imb_batch_cells(const imb_batch *b);

/* Message of the last failed call on this batch. */
const char *imb_batch_last_error(const imb_batch *b);

/* Free the batch; NULL is ignored. */
void imb_batch_destroy(imb_batch *b);

/* Pairs (a < b) of particles in contact (Eq. 7: overlap > 0) at the current
 * positions, ascending; writes min(max_pairs, total) pairs and *n_pairs = total. */
int imb_get_contacts(imb_ctx *ctx, int max_pairs, int *pairs, int *n_pairs);

/* Uniform bins of 32 x 32 cells: bin_start[nbins + 1] and bin_ids[n] (ascending
 * within each bin), nbins = ceil(nx/32) * ceil(ny/32), bin = by * nbx + bx. */
int imb_get_bins(imb_ctx *ctx, int *bin_start, int *bin_ids);

/* Queue the context's work on an external cudaStream_t of the context's device (e.g.
 * PyTorch's current stream) from the next call on; NULL restores the context's own stream.
 * The caller keeps ownership of the stream and must keep it alive while the context uses it;
 * work already queued stays where it was queued.  IMB_E_INVALID_ARG for a NULL ctx. */
int imb_set_stream(imb_ctx *ctx, void *stream);
/* The stream the context queues its work on (NULL for a NULL ctx). */
void *imb_get_stream(imb_ctx *ctx);

/* Timing of the fused stream-collide: with on != 0, every lattice step from now on records a
 * CUDA event on the context stream before its stream-collide launch and one after the launch
 * of the force gather and ghost cells that completes it (event-record nodes inside the
 * captured cycles).  Either value of on discards the timings not yet read.  IMB_E_INVALID_ARG
 * for a NULL ctx. */
int imb_enable_kernel_timing(imb_ctx *ctx, int on);
/* Waits (bounded) for the context stream, then returns in *ms the summed milliseconds of the
 * timed steps since the last read or enable call and in *launches their number, and restarts
 * the count.  IMB_E_INVALID_ARG for NULL arguments, IMB_E_TIMEOUT or IMB_E_CUDA as imb_sync. */
int imb_kernel_time(imb_ctx *ctx, double *ms, long long *launches);

/* Number of kernels this context has launched (all kinds; the kernels of a captured cycle
 * count once per replay).  0 for a NULL ctx. */
long long imb_launch_count(imb_ctx *ctx);

/* Algorithmic bytes of one stream-collide cell update for this lattice's storage
 * (9 loads + 9 stores of one population: 72 in FP32, 36 in FP16/BF16); 0 for a NULL ctx. */
double imb_bytes_per_cell(imb_ctx *ctx);

/* Particle-to-bin map into caller-owned device buffers, allocating nothing.  The
 * paper has no counterpart: this serves callers that cannot call cudaMalloc (hosts
 * whose device memory belongs to their own pool, real-time loops that must not touch
 * the allocator).
 * d_x: DEVICE pointer to 2n doubles (x, y of each centre, inside [0,nx) x [0,ny));
 * d_bin_start: DEVICE pointer to nbins + 1 ints, nbins = ceil(nx/32) * ceil(ny/32);
 * d_bin_ids: DEVICE pointer to n ints, the particle ids grouped by bin (bin = by * nbx
 * + bx, bx = floor(x/32) clamped to the lattice), ascending within each bin -- the same
 * result as imb_get_bins for the same centres.  stream: a cudaStream_t of the current
 * device, or NULL; the call only queues work on it (a stream of another device returns
 * IMB_E_INVALID_ARG).
 * Scratch (per-bin counts and fill cursors) lives in one fixed device array of
 * 2 * IMB_NOALLOC_MAX_BINS ints inside the library, held by every GPU that loads it
 * until process exit; nbins > IMB_NOALLOC_MAX_BINS returns IMB_E_INVALID_ARG.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress, with that
 * device current), so make that first call before any stream capture; the address is
 * kept for the life of the process, so a cudaDeviceReset of that device makes it stale
 * (do not call this function on a device after resetting it).  Every call
 * shares the array and clears the part it uses; calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller. */
#define IMB_NOALLOC_MAX_BINS 65536
int imb_bin_particles_noalloc(const double *d_x, int n, int nx, int ny, int *d_bin_start,
                              int *d_bin_ids, void *stream);

/* Last error message of ctx (or of the last failed imb_init_lattice when ctx is
 * NULL).  Valid until the next call on the same context. */
const char *imb_last_error(imb_ctx *ctx);

/* Free the context and its device memory.  NULL is accepted. */
void imb_destroy(imb_ctx *ctx);

/* ---- the paper's own lattice: D3Q19 with held spheres (Sec. 2.1, Tab. 1) ----
 * An nx x ny x nz lattice, x and z periodic, y periodic or bounded by halfway
 * bounce-back walls at y = 0 and y = ny (cell (i, j, k) is [i, i+1) x [j, j+1) x
 * [k, k+1), its node at the centre).  BGK collision with Guo forcing for the body
 * force (weighted by 1 - B), the partially saturated collision of Eqs. 12-14 in
 * cells a sphere covers, the solid ratio of a cell being the fraction of its
 * n_sub^3 sub-cell centres inside the sphere (a centre on the surface counts,
 * Sec. 2.3), and per-sphere force and torque (Eqs. 15-16, the force ON the sphere).
 * Spheres are held in place; their velocity and spin enter u_s = v + w x r.  A cell
 * may be covered by two spheres (touching spheres of a packed bed): B of Eq. 14 then
 * comes from their summed solid ratio (at most 1) and is shared between them in
 * proportion to their own ratios, B_p = B eps_p / (eps_1 + eps_2), each sphere's
 * Omega^s weighted by its B_p.  With C_smag > 0 each cell relaxes with the
 * Smagorinsky time tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 |Pi| / rho)) / 2, Pi
 * the non-equilibrium momentum flux, in the BGK term, the forcing and B.  Populations are stored as f_i - w_i, SoA
 * [19][nz][ny][nx], x fastest.  Velocity order: 0 rest; 1-6 (+x, -x, +y, -y, +z,
 * -z); 7-18 (+x+y, -x-y, +x-y, -x+y, +x+z, -x-z, +x-z, -x+z, +y+z, -y-z, +y-z, -y+z). */
typedef struct imb3_ctx imb3_ctx;

typedef struct imb3_params {
    int wall_y;               /* 1: walls at y = 0 and y = ny; 0: periodic in y */
    double Fx, Fy, Fz;        /* body force density on the fluid */
    int n_sub;                /* sub-cells per axis for the solid ratio, 1..10 */
    int storage;              /* IMB_STORE_* */
    double rho0, ux0, uy0, uz0; /* initial state: f* = f^eq(rho0, u0) everywhere */
    int timeout_ms;           /* bound of every host wait */
    double wall_ux_bot, wall_ux_top; /* x velocity of the walls y = 0 and y = ny (moving-wall
                                 bounce-back, wall density 1; default 0, 0) */
    double C_smag;            /* Smagorinsky constant, >= 0 (default 0: plain BGK) */
} imb3_params;

/* Defaults: walls in y at rest, no force, n_sub = 5, FP32, rho0 = 1, at rest, 60 s,
 * C_smag = 0. */
void imb3_default_params(imb3_params *p);

/* Create the lattice (p may be NULL for the defaults).  IMB_E_INVALID_ARG for a size
 * below 3, tau <= 1/2, n_sub outside 1..10, a bad storage code or C_smag < 0; IMB_E_NOMEM /
 * IMB_E_CUDA on device failures (then *out may hold a context to destroy). */
int imb3_init(imb3_ctx **out, int nx, int ny, int nz, double tau, const imb3_params *p);

/* Set n held spheres: centres x[3n] (inside the lattice), velocities v[3n], spins
 * omega[3n], radii R[n] (host arrays, copied); builds the cell map on the GPU.
 * IMB_E_INVALID_ARG for a radius outside (0, 1000], a centre outside, a periodic
 * extent below 2 (R + 2), or n x (2 ceil(R_max) + 3)^3 beyond one launch of 128-thread
 * blocks (2^31 - 1 blocks; the lattice keeps its spheres); IMB_E_OVERFLOW when three
 * spheres cover one cell (the lattice is then left without spheres). */
int imb3_set_spheres(imb3_ctx *c, int n, const double *x, const double *v, const double *omega, const double *R);

/* Advance n steps and wait (bounded).  IMB_E_UNSTABLE on NaN or |u| >= 0.3. */
int imb3_step(imb3_ctx *c, int n);

/* f(x, t) as FP64 [19][nz][ny][nx] (the pull of the stored post-collision field). */
int imb3_get_populations(imb3_ctx *c, double *f);

/* rho and u of f(x, t) (u with the half-force shift), each [nz][ny][nx]. */
int imb3_get_macro(imb3_ctx *c, double *rho, double *ux, double *uy, double *uz);

/* Force F[3n] and torque T[3n] on each sphere from the last step. */
int imb3_get_forces(imb3_ctx *c, double *F, double *T);

/* Per cell, two slots: the covering spheres (lower index first, -1: none) and their
 * sub-cell counts, each [nz][ny][nx][2]. */
int imb3_get_cell_map(imb3_ctx *c, int *sphere, int *count);

/* CUDA-event timing of every stream-collide launch (as imb_enable_kernel_timing):
 * on = 1 records a pair of events around each launch from now on. */
int imb3_enable_kernel_timing(imb3_ctx *c, int on);
/* Waits (bounded), then returns the summed time *ms of the timed launches and their
 * number *launches, and restarts the count.  IMB_E_INVALID_ARG for NULL outputs. */
int imb3_kernel_time(imb3_ctx *c, double *ms, long long *launches);
/* Kernel launches this context has made so far (0 for NULL). */
long long imb3_launch_count(imb3_ctx *c);
/* Algorithmic bytes per cell update: 19 loads + 19 stores of the storage type. */
double imb3_bytes_per_cell(imb3_ctx *c);
/* Message of the last failed call on c (of the last failed imb3_init for NULL); the string
 * belongs to the library and stays valid until the next call on c. */
const char *imb3_last_error(imb3_ctx *c);
/* Waits for the context's work and frees everything it holds; NULL is ignored. */
void imb3_destroy(imb3_ctx *c);

#ifdef __cplusplus
}
#endif
#endif /* IMBLBM_H */
