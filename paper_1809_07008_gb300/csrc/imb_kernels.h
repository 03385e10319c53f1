// imb_kernels.h -- host-side launch wrappers of the CUDA kernels (internal to the
// library; the public interface is include/imblbm.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace imb {

// A launch that, with `early`, may begin while the previous kernel in the stream finishes
// (programmatic dependent launch): the kernel waits for that kernel's completion itself,
// before it touches memory (cudaGridDependencySynchronize at its start), so only the launch
// latency overlaps.
template <typename... P, typename... A>
static cudaError_t launch_dependent(void (*kernel)(P...), int grid, int block, int smem, cudaStream_t s,
                                    bool early, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}

struct PRec;
struct TileCand;
struct GridBarrier;

// Everything the lattice kernels read about the lattice and the particles.
struct LatticeArgs {
    int nx, ny, pitch, bc_x, bc_y;
    // population buffers: 9 planes of plane elements, each a frame of ny + 2 rows of pitch
    // elements around the lattice (ghost rows y = -1 and ny, ghost_x columns left of x = 0 and
    // at least one right of x = nx - 1); node (x, y) of plane q lies at
    // origin + q plane + y pitch + x from the start of the buffer
    size_t plane, origin;
    int ghost_x;
    float tau, omega0;         // relaxation time and 1 / tau
    float smag_coef;           // 18 sqrt(2) C^2 (0 switches the Smagorinsky model off)
    float Fx, Fy;              // body force density (0, 0 = no forcing)
    float u_in_x, u_in_y;
    float uw_bot, uw_top;      // x velocity of the walls y = 0 and y = ny
    int eps_mode, n_sub;
    int nbx, nby;              // bins of 32 x 32 cells
    int np;
    const int *bin_start;      // [nbx*nby + 1]
    const int *bin_ids;        // [np]
    const PRec *prec;          // [np]
    float *eps_tab;            // [np * tab_stride] solid ratios of partially covered cells
    int tab_w, tab_h, tab_stride; // table row width 2 th + 1, half width th, floats per particle
    double *F;                 // [2 np] hydrodynamic force accumulators
    double *T;                 // [np]   hydrodynamic torque accumulators
    unsigned *err;
    unsigned *tile_ctr;        // [2] tiles handed out and blocks finished (zero between launches)
    const int *pbin;           // [np] bin of each particle
    char4 *pivl;               // [np][tab_w] per particle row dk + tab_h: the cells (relative column) the disk
                               // reaches into, [x, y], and covers whole, [z, w] (exact-area mode)
    int *pslot;                // [np][9] tile * TILE_CAND + slot of the particle in the candidate lists of the
                               // 3 x 3 tiles around its bin (row by row), -1 where it is not a candidate
    int tf_units;              // force partials per tile: 1, or SMALL_UPT when each work unit keeps its own
};

// work units per tile of the small-lattice stream-collide (units of eight rows, one per block)
constexpr int SMALL_UPT = 4;

// DEM state and parameters (FP64).
struct DemArgs {
    int np, nx, ny, bc_x, bc_y, N_sub;
    double dt, kn, kt, zeta, ct_ratio, mu, gx_eff, gy_eff, skin;
    int model;                  // 0 linear spring-dashpot, 1 simplified Hertz-Mindlin
    double hm_kn0, hm_sn0, hm_kt0, hm_c0;   // 4/3 E*, 2 E*, 8 G*, 2 sqrt(5/6) |beta|
    double *x, *v, *w;          // primary state [2np], [2np], [np]
    double *x1, *v1, *w1;       // second buffer of the coupled sub-cycle loop
    double *x_start;            // positions at the start of the coupling cycle
    const double *r, *m, *I;
    const double *F, *T;        // hydrodynamic force/torque (frozen during the sub-cycles)
    int *nbr_cnt_old, *nbr_cnt;       // [np]
    int *nbr_id_old, *nbr_id;         // [np * MAX_NBR]
    double *nbr_xi_old, *nbr_xi;      // [np * MAX_NBR]
    double *nbr_cn_old, *nbr_cn;      // [np * MAX_NBR] normal damping of each candidate pair
    double *exc;                      // [np][2] excursion bounds of contact-free motion in the cycle
    int *loud;                        // [np] 1 if p may touch a wall or a candidate within the cycle
    int *iloud;                       // [np] per island root: 1 if any member is loud
    double *wall_xi;                  // [np * 4]
    int *free_ids, *coupled_ids;      // [np]
    int *counters;                    // [0] free, [1] coupled, [2] small islands, [3] big-island
                                      // particles, [4] member-list cursor, [5] medium islands
    int *parent, *label;              // [np] union-find forest and island of each particle
    int *isz, *ifill, *istart;        // per root: island size, fill cursor, start in members
    int *members, *roots, *big_ids;   // [np] island members, roots of small islands, big-island particles
    const int *bin_start, *bin_ids;   // bins of the positions at cycle start
    int *pbin;                        // [np]
    int nbx, nby;
    GridBarrier *barrier;
    unsigned *err;
};

// lattice kernels (imb_lbm.cu)
cudaError_t launch_init_populations(void *f, int storage, const LatticeArgs &a, float rho0, float ux0,
                                    float uy0, cudaStream_t s);
// tile_force: [ntiles][TILE_CAND][3] FP64 partial force / torque sums of each tile's candidates
// the ghost cells of the frame from the edge nodes' populations (after the populations were
// written other than by the stream-collide kernel, which keeps them itself)
cudaError_t launch_fill_ghosts(void *f, int storage, const LatticeArgs &a, cudaStream_t s);
// small: one eight-row unit per block (a.tf_units == SMALL_UPT, tensor maps with boxes of
// tma_box_rows(storage, true) rows)
cudaError_t launch_stream_collide(const void *fin, void *fout, int storage, const LatticeArgs &a,
                                  const CUtensorMap *tmap_narrow, const CUtensorMap *tmap_wide,
                                  const TileCand *tiles, double *tile_force, bool small, cudaStream_t s);
// after a stream-collide launch that wrote f: a.F, a.T of every particle = its tiles' partial
// sums, in a fixed order, and the ghost cells of f
cudaError_t launch_step_tail(void *f, int storage, const LatticeArgs &a, const double *tile_force, cudaStream_t s);
cudaError_t launch_tile_lists(const LatticeArgs &a, TileCand *tiles, cudaStream_t s);
// per particle and row, the reached and fully covered cell intervals (before the tile lists and
// the solid-ratio tables, which read them)
cudaError_t launch_particle_rows(const LatticeArgs &a, cudaStream_t s);
cudaError_t launch_particle_eps(const LatticeArgs &a, cudaStream_t s);
int tma_box_width(int storage, int wide);
int tma_box_rows(int storage, bool small);
// blocks of the stream-collide kernel resident on the current device at once
int stream_collide_resident_blocks(int storage);
cudaError_t launch_gather(const void *fin, int storage, const LatticeArgs &a, double *f_out,
                          double *rho, double *ux, double *uy, cudaStream_t s);
cudaError_t launch_cell_map(const LatticeArgs &a, int *count, int *ids, float *eps, cudaStream_t s);
// drag gradient (imb_adjoint.cu)
cudaError_t launch_drag_sum(const double *F, int np, double *acc, cudaStream_t s);
cudaError_t launch_cell_E(const int *count, const float *eps, size_t ncell, float *E, cudaStream_t s);
cudaError_t launch_adjoint_inlet(float *lam, const float *S1, const LatticeArgs &a, double *g_uin,
                                 cudaStream_t s);
cudaError_t launch_adjoint_step(const float *lam1, const float *S0, float *lam0, const LatticeArgs &a,
                                const float *E, double *gE, float inv_T, double *g_tau, cudaStream_t s);
cudaError_t launch_position_grad(const int *count, const int *ids, const double *gE, const double *x,
                                 const double *r, int nx, int ny, int bc_x, int bc_y, double *dJ_dx,
                                 cudaStream_t s);

// particle kernels (imb_particles.cu)
cudaError_t launch_particle_table(const double *x, const double *r, const double *x_start, int np,
                                  int nx, int ny, int bc_x, int bc_y, double skin_half, int nbx,
                                  int nby, int *bin_count, int *pbin, PRec *prec, const double *v,
                                  const double *w, double *F, double *T, unsigned *err,
                                  cudaStream_t s);
cudaError_t launch_bin_scan(int *bin_count, int *bin_fill, int *bin_start, int nbins, int *bsum,
                            int *dem_counters, cudaStream_t s);
cudaError_t launch_bin_fill(const int *pbin, int np, int *bin_fill, const int *bin_start,
                            int *bin_ids, cudaStream_t s);
cudaError_t launch_dem_neighbours(const DemArgs &d, cudaStream_t s);
cudaError_t launch_dem_coupled(const DemArgs &d, int nblocks, cudaStream_t s);
cudaError_t launch_dem_islands_setup(const DemArgs &d, cudaStream_t s);
// free particles and islands of up to 32 particles, one launch
cudaError_t launch_dem_local(const DemArgs &d, cudaStream_t s);
// device-addressable pinned host arrays (see device_view in the API) <-> the particle arrays
cudaError_t launch_kinematics_in(const double *hx, const double *hv, const double *hw, double *x, double *v, double *w,
                                 int np, cudaStream_t s);
cudaError_t launch_state_out(const double *F, const double *T, const double *x, const double *v, const double *w,
                             double *hF, double *hT, double *hx, double *hv, double *hw, int np, cudaStream_t s);
cudaError_t launch_contacts(const double *x, const double *r, int np, int nx, int ny, int bc_x,
                            int bc_y, const int *bin_start, const int *bin_ids, const int *pbin,
                            int nbx, int nby, int reach, int *pair_cnt, int *pairs, int max_per,
                            cudaStream_t s);
int dem_coupled_blocks();

}  // namespace imb
