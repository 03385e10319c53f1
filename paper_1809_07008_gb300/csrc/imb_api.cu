// imb_api.cu -- host runtime of the GB300 IMB-LBM-DEM library: the C ABI declared
// in include/imblbm.h.  Owns device memory, the stream, the per-step launch
// sequence of the coupling cycle (Sec. 2.4, Fig. 4), bounded waits and the
// translation of device error bits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/imblbm.h"
#include "imb_device.cuh"
#include "imb_kernels.h"

using namespace imb;

// A run of steps captured as a CUDA graph: the instantiated graph, the graph itself (its
// event-record nodes, which time the steps, are re-pointed through it), the launches it holds
// and the buffer indices it leaves.
struct StepGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> ev;
    long long launches = 0;
    int cur_after = 0, nbr_after = 0;
};

// lattice steps without the DEM per graph (even, so the populations come back to their buffer)
constexpr int GRAPH_STEPS = 8;

struct imb_ctx {
    int nx = 0, ny = 0, pitch = 0;
    double tau = 0.0, C_smag = 0.0;
    imb_params p{};
    int device = 0;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    cudaStream_t side = nullptr;                  // solid-ratio tables beside the bins and tile lists
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_rows = nullptr;               // the particles' row intervals are written
    void *fbuf[2] = {nullptr, nullptr};
    int cur = 0;               // buffer holding the latest post-collision populations
    size_t plane = 0, origin = 0, elem = 4;
    int ghost_x = 0;
    // particles
    int np = 0, cap = 0;
    double r_max = 0.0;
    double *x = nullptr, *v = nullptr, *w = nullptr, *r = nullptr, *m = nullptr, *I = nullptr;
    double *F = nullptr, *T = nullptr, *x1 = nullptr, *v1 = nullptr, *w1 = nullptr, *xs = nullptr;
    int *nbr_cnt[2] = {nullptr, nullptr}, *nbr_id[2] = {nullptr, nullptr};
    double *nbr_xi[2] = {nullptr, nullptr};
    double *nbr_cn[2] = {nullptr, nullptr};
    int nbr_cur = 0;
    double *wall_xi = nullptr;
    int *free_ids = nullptr, *coupled_ids = nullptr, *counters = nullptr;
    int *parent = nullptr, *label = nullptr, *isz = nullptr, *ifill = nullptr, *istart = nullptr;
    int *members = nullptr, *roots = nullptr, *big_ids = nullptr;
    int *loud = nullptr, *iloud = nullptr;
    double *exc = nullptr;
    int *pbin = nullptr;
    int *pslot = nullptr;      // [np][9] each particle's slot in the candidate lists of its 3 x 3 tiles
    PRec *prec = nullptr;
    // bins
    int nbx = 0, nby = 0, nbins = 0;
    int *bin_count = nullptr, *bin_fill = nullptr, *bin_start = nullptr, *bin_ids = nullptr;
    int *bin_bsum = nullptr;   // per-block totals of the bin scan
    GridBarrier *barrier = nullptr;
    unsigned *err = nullptr;
    unsigned *tile_ctr = nullptr;
    unsigned *h_err = nullptr;   // pinned host copy of the error word
    TileCand *tiles = nullptr;      // per 32 x 32 tile: particles that can reach it
    double *tile_force = nullptr;   // per tile and candidate: partial force and torque sums
    float *eps_tab = nullptr;       // per particle: solid ratios of its partially covered cells
    size_t eps_tab_cap = 0;
    char4 *pivl = nullptr;          // per particle and row: reached / fully covered cell intervals
    size_t pivl_cap = 0;
    int tab_w = 0, tab_h = 0;
    CUtensorMap tmap[2][2];         // TMA descriptors [buffer][narrow, wide] of the populations
    bool small = false;             // units of eight rows, one per block (all fit on the device at once)
    // steps captured as CUDA graphs (see graph_steps): [0, 8) one coupling cycle with the DEM,
    // by (kernel timing, population buffer, neighbour-list buffer); [8, 12) GRAPH_STEPS lattice
    // steps without it, by (kernel timing, population buffer); off for good after a failed capture
    StepGraph graphs[12];
    bool use_graphs = true;
    bool capturing = false;   // inside graph_steps' capture: timing events become graph nodes
    // parameters derived on the host
    double zeta = 0.0, gx_eff = 0.0, gy_eff = 0.0;
    double hm_kn0 = 0.0, hm_sn0 = 0.0, hm_kt0 = 0.0, hm_c0 = 0.0;   // Hertz-Mindlin constants
    // timing / accounting
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    long long launches = 0;
    std::string msg;
};

static std::string g_init_error;

static int fail(imb_ctx *c, int code, const std::string &m) {
    if (c) c->msg = m;
    else g_init_error = m;
    return code;
}

static int cuda_fail(imb_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? IMB_E_NOMEM : IMB_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename T>
static cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void **)p, n * sizeof(T));
}

static void dfree(void *p) {
    if (p) cudaFree(p);
}

extern "C" void imb_default_params(imb_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->bc_x = IMB_BC_PERIODIC;
    p->bc_y = IMB_BC_WALL;
    p->rho0 = 1.0;
    p->storage = IMB_STORE_FP32;
    p->eps_mode = IMB_EPS_EXACT;
    p->n_sub = 5;
    p->dem_on = 0;
    p->N_sub = 100;
    p->kn = 1.0e5;
    p->kt = 0.5e5;
    p->e_rest = 0.5;
    p->ct_ratio = 0.5;
    p->mu = 0.5;
    p->rho_s = 2.65;
    p->skin = 1.0;
    p->timeout_ms = 60000;
}

static LatticeArgs lattice_args(const imb_ctx *c) {
    LatticeArgs a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.pitch = c->pitch;
    a.bc_x = c->p.bc_x;
    a.bc_y = c->p.bc_y;
    a.plane = c->plane;
    a.origin = c->origin;
    a.ghost_x = c->ghost_x;
    a.tau = (float)c->tau;
    a.omega0 = (float)(1.0 / c->tau);
    a.smag_coef = (float)(18.0 * std::sqrt(2.0) * c->C_smag * c->C_smag);
    a.Fx = (float)c->p.Fx;
    a.Fy = (float)c->p.Fy;
    a.u_in_x = (float)c->p.u_in_x;
    a.u_in_y = (float)c->p.u_in_y;
    a.uw_bot = (float)c->p.wall_u_bot;
    a.uw_top = (float)c->p.wall_u_top;
    a.eps_mode = c->p.eps_mode;
    a.n_sub = c->p.n_sub;
    a.nbx = c->nbx;
    a.nby = c->nby;
    a.np = c->np;
    a.bin_start = c->bin_start;
    a.bin_ids = c->bin_ids;
    a.prec = c->prec;
    a.eps_tab = c->eps_tab;
    a.tab_w = c->tab_w;
    a.tab_h = c->tab_h;
    a.tab_stride = c->tab_w * c->tab_w;
    a.F = c->F;
    a.T = c->T;
    a.err = c->err;
    a.tile_ctr = c->tile_ctr;
    a.pbin = c->pbin;
    a.pslot = c->pslot;
    a.pivl = c->pivl;
    a.tf_units = c->small ? SMALL_UPT : 1;
    return a;
}

static DemArgs dem_args(imb_ctx *c) {
    DemArgs d;
    d.np = c->np;
    d.nx = c->nx;
    d.ny = c->ny;
    d.bc_x = c->p.bc_x;
    d.bc_y = c->p.bc_y;
    d.N_sub = c->p.N_sub;
    d.dt = 1.0 / (double)c->p.N_sub;
    d.kn = c->p.kn;
    d.kt = c->p.kt;
    d.zeta = c->zeta;
    d.model = c->p.contact_model;
    d.hm_kn0 = c->hm_kn0;
    d.hm_sn0 = c->hm_sn0;
    d.hm_kt0 = c->hm_kt0;
    d.hm_c0 = c->hm_c0;
    d.ct_ratio = c->p.ct_ratio;
    d.mu = c->p.mu;
    d.gx_eff = c->gx_eff;
    d.gy_eff = c->gy_eff;
    d.skin = c->p.skin;
    d.x = c->x;
    d.v = c->v;
    d.w = c->w;
    d.x1 = c->x1;
    d.v1 = c->v1;
    d.w1 = c->w1;
    d.x_start = c->xs;
    d.r = c->r;
    d.m = c->m;
    d.I = c->I;
    d.F = c->F;
    d.T = c->T;
    d.nbr_cnt_old = c->nbr_cnt[c->nbr_cur ^ 1];
    d.nbr_cnt = c->nbr_cnt[c->nbr_cur];
    d.nbr_id_old = c->nbr_id[c->nbr_cur ^ 1];
    d.nbr_id = c->nbr_id[c->nbr_cur];
    d.nbr_xi_old = c->nbr_xi[c->nbr_cur ^ 1];
    d.nbr_xi = c->nbr_xi[c->nbr_cur];
    d.nbr_cn_old = c->nbr_cn[c->nbr_cur ^ 1];
    d.nbr_cn = c->nbr_cn[c->nbr_cur];
    d.wall_xi = c->wall_xi;
    d.free_ids = c->free_ids;
    d.coupled_ids = c->coupled_ids;
    d.counters = c->counters;
    d.parent = c->parent;
    d.label = c->label;
    d.isz = c->isz;
    d.ifill = c->ifill;
    d.istart = c->istart;
    d.members = c->members;
    d.roots = c->roots;
    d.exc = c->exc;
    d.loud = c->loud;
    d.iloud = c->iloud;
    d.big_ids = c->big_ids;
    d.bin_start = c->bin_start;
    d.bin_ids = c->bin_ids;
    d.pbin = c->pbin;
    d.nbx = c->nbx;
    d.nby = c->nby;
    d.barrier = c->barrier;
    d.err = c->err;
    return d;
}

static void drop_step_graphs(imb_ctx *c) {
    for (StepGraph &sg : c->graphs) {
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        if (sg.graph) cudaGraphDestroy(sg.graph);
        sg = StepGraph();
    }
}

static void free_particles(imb_ctx *c) {
    drop_step_graphs(c);   // they hold the particle arrays' addresses
    double **dp[] = {&c->x, &c->v, &c->w, &c->r, &c->m, &c->I, &c->F, &c->T,
                     &c->x1, &c->v1, &c->w1, &c->xs, &c->nbr_xi[0], &c->nbr_xi[1], &c->wall_xi,
                     &c->nbr_cn[0], &c->nbr_cn[1], &c->exc};
    for (double **q : dp) { dfree(*q); *q = nullptr; }
    int **ip[] = {&c->nbr_cnt[0], &c->nbr_cnt[1], &c->nbr_id[0], &c->nbr_id[1], &c->free_ids,
                  &c->coupled_ids, &c->pbin, &c->pslot, &c->bin_ids, &c->parent, &c->label, &c->isz, &c->ifill,
                  &c->istart, &c->members, &c->roots, &c->big_ids, &c->loud, &c->iloud};
    for (int **q : ip) { dfree(*q); *q = nullptr; }
    dfree(c->prec);
    c->prec = nullptr;
    c->np = c->cap = 0;
}

extern "C" void imb_destroy(imb_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_particles(c);
    dfree(c->fbuf[0]);
    dfree(c->fbuf[1]);
    dfree(c->bin_count);
    dfree(c->bin_fill);
    dfree(c->bin_start);
    dfree(c->bin_bsum);
    dfree(c->counters);
    dfree(c->barrier);
    dfree(c->err);
    dfree(c->tile_ctr);
    if (c->h_err) cudaFreeHost(c->h_err);
    dfree(c->tiles);
    dfree(c->tile_force);
    dfree(c->eps_tab);
    dfree(c->pivl);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_rows) cudaEventDestroy(c->ev_rows);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

// TMA descriptor of one population buffer: a 3D tensor (x over the padded row,
// y, plane) read in boxes of 32 (narrow) or 32 + halo (wide) x 16 x 1 elements.
static cudaError_t make_tensor_map(imb_ctx *c, void *buf, CUtensorMap *map, int wide) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const CUtensorMapDataType dt = c->p.storage == IMB_STORE_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : c->p.storage == IMB_STORE_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->ny + 2, 9};   // the whole frame
    cuuint64_t strides[2] = {(cuuint64_t)c->pitch * c->elem, (cuuint64_t)c->plane * c->elem};
    cuuint32_t box[3] = {(cuuint32_t)tma_box_width(c->p.storage, wide), (cuuint32_t)tma_box_rows(c->p.storage, c->small),
                         1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, dt, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

extern "C" int imb_init_lattice(imb_ctx **out, int nx, int ny, double tau, double C_smag,
                                const imb_params *pin) {
    if (!out) return fail(nullptr, IMB_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    imb_params p;
    if (pin) p = *pin;
    else imb_default_params(&p);
    if (nx < 3 || ny < 3) return fail(nullptr, IMB_E_INVALID_ARG, "nx and ny must be >= 3");
    if (!(tau > 0.5)) return fail(nullptr, IMB_E_INVALID_ARG, "tau must be > 1/2 (Eq. 5)");
    if (!(C_smag >= 0.0)) return fail(nullptr, IMB_E_INVALID_ARG, "C_smag must be >= 0");
    if (p.bc_x < 0 || p.bc_x > 2 || p.bc_y < 0 || p.bc_y > 1)
        return fail(nullptr, IMB_E_INVALID_ARG, "bad boundary code");
    if (p.storage < 0 || p.storage > 2) return fail(nullptr, IMB_E_INVALID_ARG, "bad storage");
    if (p.eps_mode < 0 || p.eps_mode > 1 || p.n_sub < 1 || p.n_sub > 64)
        return fail(nullptr, IMB_E_INVALID_ARG, "bad solid-ratio mode");
    if (p.N_sub < 1 || !(p.kn > 0.0) || !(p.kt > 0.0) || !(p.e_rest > 0.0) || !(p.e_rest <= 1.0) ||
        !(p.rho_s > 0.0) || !(p.mu >= 0.0) || !(p.skin > 0.0))
        return fail(nullptr, IMB_E_INVALID_ARG, "bad DEM parameters");
    if (p.contact_model < 0 || p.contact_model > 1 ||
        (p.contact_model == IMB_CONTACT_HERTZ_MINDLIN &&
         !(p.E_young > 0.0 && p.nu_poisson >= 0.0 && p.nu_poisson < 0.5)))
        return fail(nullptr, IMB_E_INVALID_ARG, "bad contact model or Hertz-Mindlin material");
    if (p.timeout_ms <= 0) p.timeout_ms = 60000;
    if (p.work_units < 0 || p.work_units > 2) return fail(nullptr, IMB_E_INVALID_ARG, "work_units must be 0, 1 or 2");
    if (p.plain_launches != 0 && p.plain_launches != 1)
        return fail(nullptr, IMB_E_INVALID_ARG, "plain_launches must be 0 or 1");
    if ((long long)nx * ny > (1ll << 31) / 16) return fail(nullptr, IMB_E_INVALID_ARG, "lattice too large");

    imb_ctx *c = new imb_ctx();
    c->nx = nx;
    c->ny = ny;
    c->tau = tau;
    c->C_smag = C_smag;
    c->p = p;
    cudaGetDevice(&c->device);
    c->elem = p.storage == IMB_STORE_FP32 ? 4 : 2;
    // the frame: 128 bytes of ghost columns left of x = 0 (node rows start 128-byte aligned),
    // the ghost column x = nx and padding up to a multiple of 32 elements, ghost rows -1 and ny
    c->ghost_x = 128 / (int)c->elem;
    c->pitch = (c->ghost_x + nx + 1 + 31) / 32 * 32;
    c->plane = (size_t)c->pitch * (ny + 2);
    c->origin = (size_t)c->pitch + c->ghost_x;
    c->nbx = (nx + TILE - 1) / TILE;
    c->nby = (ny + TILE - 1) / TILE;
    c->nbins = c->nbx * c->nby;
    // a lattice whose eight-row units all fit on the device at once takes one per block
    c->use_graphs = p.plain_launches == 0;
    c->small = p.work_units == 2 ||
               (p.work_units == 0 && (long long)c->nbins * SMALL_UPT <= stream_collide_resident_blocks(p.storage));
    const double le = std::log(p.e_rest);
    c->zeta = -le / std::sqrt(M_PI * M_PI + le * le);
    {   // identical materials: E* = E / (2 (1 - nu^2)), G* = E / (4 (2 - nu)(1 + nu))
        const double E = p.E_young, nu = p.nu_poisson;
        const double Es = E / (2.0 * (1.0 - nu * nu));
        const double Gs = E / (4.0 * (2.0 - nu) * (1.0 + nu));
        c->hm_kn0 = 4.0 / 3.0 * Es;
        c->hm_sn0 = 2.0 * Es;
        c->hm_kt0 = 8.0 * Gs;
        c->hm_c0 = 2.0 * std::sqrt(5.0 / 6.0) * c->zeta;
    }
    c->gx_eff = (1.0 - 1.0 / p.rho_s) * p.gx;
    c->gy_eff = (1.0 - 1.0 / p.rho_s) * p.gy;
    auto bail = [&](cudaError_t e, const char *what) {
        g_init_error = std::string(what) + ": " + cudaGetErrorString(e);
        imb_destroy(c);
        return e == cudaErrorMemoryAllocation ? IMB_E_NOMEM : IMB_E_CUDA;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "cudaStreamCreate");
    c->stream = c->own_stream;
    if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_rows, cudaEventDisableTiming)) != cudaSuccess)
        return bail(e, "side stream");
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMalloc(&c->fbuf[b], 9 * c->plane * c->elem)) != cudaSuccess ||
            (e = cudaMemsetAsync(c->fbuf[b], 0, 9 * c->plane * c->elem, c->stream)) != cudaSuccess)
            return bail(e, "population buffers");
    // bin arrays padded to a multiple of 32 entries (the scan moves 16-byte vectors)
    const int nbins_pad = (c->nbins + 31) / 32 * 32;
    if ((e = dalloc(&c->bin_count, nbins_pad)) != cudaSuccess || (e = dalloc(&c->bin_fill, nbins_pad)) != cudaSuccess ||
        (e = dalloc(&c->bin_start, nbins_pad + 32)) != cudaSuccess || (e = dalloc(&c->counters, 8)) != cudaSuccess ||
        (e = dalloc(&c->barrier, 1)) != cudaSuccess || (e = dalloc(&c->err, 1)) != cudaSuccess ||
        (e = dalloc(&c->tile_ctr, 2)) != cudaSuccess || (e = dalloc(&c->tiles, c->nbins)) != cudaSuccess ||
        (e = dalloc(&c->tile_force, (size_t)c->nbins * TILE_CAND * 3 * (c->small ? SMALL_UPT : 1))) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_err, sizeof(unsigned))) != cudaSuccess ||
        (e = dalloc(&c->bin_bsum, c->nbins / 1024 + 1)) != cudaSuccess)
        return bail(e, "bookkeeping buffers");
    cudaMemsetAsync(c->tiles, 0, sizeof(TileCand) * c->nbins, c->stream);
    for (int b = 0; b < 2; ++b)
        for (int wide = 0; wide < 2; ++wide)
            if ((e = make_tensor_map(c, c->fbuf[b], &c->tmap[b][wide], wide)) != cudaSuccess)
                return bail(e, "TMA descriptor");
    cudaMemsetAsync(c->bin_count, 0, sizeof(int) * nbins_pad, c->stream);
    cudaMemsetAsync(c->bin_fill, 0, sizeof(int) * nbins_pad, c->stream);
    cudaMemsetAsync(c->bin_start, 0, sizeof(int) * (nbins_pad + 32), c->stream);
    cudaMemsetAsync(c->counters, 0, sizeof(int) * 8, c->stream);
    cudaMemsetAsync(c->barrier, 0, sizeof(GridBarrier), c->stream);
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream);
    cudaMemsetAsync(c->tile_ctr, 0, 2 * sizeof(unsigned), c->stream);
    LatticeArgs a = lattice_args(c);
    for (int b = 0; b < 2; ++b) {
        if ((e = launch_init_populations(c->fbuf[b], p.storage, a, (float)p.rho0, (float)p.ux0,
                                         (float)p.uy0, c->stream)) != cudaSuccess ||
            (e = launch_fill_ghosts(c->fbuf[b], p.storage, a, c->stream)) != cudaSuccess)
            return bail(e, "init kernel");
        c->launches += 2;
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e, "init sync");
    *out = c;
    return IMB_OK;
}

// rebuild bins and the lattice particle records for the current positions
// (bins_only: the particle records and bins, for a DEM cycle that rebuilds the rest after it)
static int rebuild_table(imb_ctx *c, const double *x_start, bool zero_forces, bool bins_only = false) {
    if (c->np == 0) {
        CK(cudaMemsetAsync(c->tiles, 0, sizeof(TileCand) * c->nbins, c->stream), "clear tile lists");
        return IMB_OK;
    }
    CK(launch_particle_table(c->x, c->r, x_start, c->np, c->nx, c->ny, c->p.bc_x, c->p.bc_y,
                             0.5 * c->p.skin, c->nbx, c->nby, c->bin_count, c->pbin, c->prec, c->v,
                             c->w, zero_forces ? c->F : nullptr, c->T, c->err, c->stream),
       "particle table");
    if (bins_only) {
        CK(launch_bin_scan(c->bin_count, c->bin_fill, c->bin_start, c->nbins, c->bin_bsum, c->counters, c->stream),
           "bin scan");
        CK(launch_bin_fill(c->pbin, c->np, c->bin_fill, c->bin_start, c->bin_ids, c->stream), "bin fill");
        c->launches += 4;   // table, scan (two passes), fill
        return IMB_OK;
    }
    // the rows' cell intervals and the solid-ratio tables need only the particle records: they
    // run on the side stream while the bins are built; the tile lists wait for the intervals,
    // the stream for the tables at the end
    CK(cudaEventRecord(c->ev_fork, c->stream), "fork");
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
    CK(launch_particle_rows(lattice_args(c), c->side), "row intervals");
    CK(cudaEventRecord(c->ev_rows, c->side), "rows");
    CK(launch_particle_eps(lattice_args(c), c->side), "solid-ratio tables");
    CK(cudaEventRecord(c->ev_join, c->side), "join");
    CK(launch_bin_scan(c->bin_count, c->bin_fill, c->bin_start, c->nbins, c->bin_bsum, c->counters, c->stream),
       "bin scan");
    CK(launch_bin_fill(c->pbin, c->np, c->bin_fill, c->bin_start, c->bin_ids, c->stream), "bin fill");
    CK(cudaMemsetAsync(c->pslot, 0xff, 9 * sizeof(int) * (size_t)c->np, c->stream), "clear tile slots");
    CK(cudaStreamWaitEvent(c->stream, c->ev_rows, 0), "rows");
    CK(launch_tile_lists(lattice_args(c), c->tiles, c->stream), "tile lists");
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join");
    c->launches += 7;   // table, scan (two passes), fill, row intervals, tile lists, solid-ratio map
    return IMB_OK;
}

extern "C" int imb_set_particles(imb_ctx *c, int n, const double *x, const double *v,
                                 const double *omega, const double *r) {
    if (!c) return IMB_E_INVALID_ARG;
    if (n < 0 || (n > 0 && (!x || !v || !omega || !r)))
        return fail(c, IMB_E_INVALID_ARG, "bad particle arrays");
    double rmax = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(r[i] > 0.0) || !(r[i] <= 31.0))
            return fail(c, IMB_E_INVALID_ARG, "radius must be in (0, 31]");
        if (!(x[2 * i] >= 0.0 && x[2 * i] < c->nx && x[2 * i + 1] >= 0.0 && x[2 * i + 1] < c->ny))
            return fail(c, IMB_E_INVALID_ARG, "particle centre outside [0,nx) x [0,ny)");
        rmax = std::max(rmax, r[i]);
    }
    if (c->p.dem_on && 2.0 * rmax + c->p.skin > (double)TILE)
        return fail(c, IMB_E_INVALID_ARG, "DEM needs 2 r_max + skin <= 32 cells");
    {   // the tile blocks address the solid-ratio tables with 32-bit offsets
        const long long tw = 2 * ((long long)std::ceil(rmax) + 1) + 1;
        if ((long long)n * tw * tw >= (1ll << 31))
            return fail(c, IMB_E_INVALID_ARG, "n (2 ceil(r_max) + 3)^2 must stay below 2^31 (solid-ratio tables)");
    }
    // a periodic axis must be long enough that a tile sees a single image of a disk
    if (n > 0 && ((c->p.bc_x == IMB_BC_PERIODIC && c->nx < 2.0 * (TILE + rmax + 2.0)) ||
                  (c->p.bc_y == IMB_BC_PERIODIC && c->ny < 2.0 * (TILE + rmax + 2.0))))
        return fail(c, IMB_E_INVALID_ARG, "periodic extent must be at least 2 (32 + r_max + 2) cells");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->stream), "sync");
    drop_step_graphs(c);   // captured with the old count and table shape
    if (n > c->cap) {
        free_particles(c);
        cudaError_t e = cudaSuccess;
        size_t N = (size_t)n;
        double **d2[] = {&c->x, &c->v, &c->F, &c->x1, &c->v1, &c->xs};
        for (double **q : d2) if (e == cudaSuccess) e = dalloc(q, 2 * N);
        double **d1[] = {&c->w, &c->r, &c->m, &c->I, &c->T, &c->w1};
        for (double **q : d1) if (e == cudaSuccess) e = dalloc(q, N);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = dalloc(&c->nbr_cnt[b], N);
            if (e == cudaSuccess) e = dalloc(&c->nbr_id[b], N * MAX_NBR);
            if (e == cudaSuccess) e = dalloc(&c->nbr_xi[b], N * MAX_NBR);
        }
        if (e == cudaSuccess) e = dalloc(&c->wall_xi, 4 * N);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = dalloc(&c->nbr_cn[b], N * MAX_NBR);
        if (e == cudaSuccess) e = dalloc(&c->free_ids, N);
        if (e == cudaSuccess) e = dalloc(&c->coupled_ids, N);
        if (e == cudaSuccess) e = dalloc(&c->pbin, N);
        if (e == cudaSuccess) e = dalloc(&c->pslot, 9 * N);
        if (e == cudaSuccess) e = dalloc(&c->bin_ids, N);
        if (e == cudaSuccess) e = dalloc(&c->prec, N);
        const size_t Np = (N + 31) / 32 * 32;
        int **ia[] = {&c->parent, &c->label, &c->members, &c->roots, &c->big_ids, &c->loud};
        for (int **q : ia) if (e == cudaSuccess) e = dalloc(q, N);
        if (e == cudaSuccess) e = dalloc(&c->isz, Np);
        if (e == cudaSuccess) e = dalloc(&c->ifill, Np);
        if (e == cudaSuccess) e = dalloc(&c->iloud, Np);
        if (e == cudaSuccess) e = dalloc(&c->exc, 2 * N);
        if (e == cudaSuccess) e = dalloc(&c->istart, Np + 32);
        if (e == cudaSuccess) e = cudaMemset(c->isz, 0, 4 * Np);
        if (e == cudaSuccess) e = cudaMemset(c->ifill, 0, 4 * Np);
        if (e != cudaSuccess) {
            free_particles(c);
            return cuda_fail(c, e, "particle buffers");
        }
        c->cap = n;
    }
    c->np = n;
    c->r_max = rmax;
    {
        const int th = (int)std::ceil(rmax) + 1, tw = 2 * th + 1;
        const size_t need = (size_t)std::max(n, 1) * tw * tw;
        if (need > c->eps_tab_cap) {
            dfree(c->eps_tab);
            c->eps_tab = nullptr;
            c->eps_tab_cap = 0;
            cudaError_t e = dalloc(&c->eps_tab, need);
            if (e != cudaSuccess) return cuda_fail(c, e, "solid-ratio table");
            c->eps_tab_cap = need;
        }
        const size_t need_rows = (size_t)std::max(n, 1) * tw;
        if (need_rows > c->pivl_cap) {
            dfree(c->pivl);
            c->pivl = nullptr;
            c->pivl_cap = 0;
            cudaError_t e = dalloc(&c->pivl, need_rows);
            if (e != cudaSuccess) return cuda_fail(c, e, "row intervals");
            c->pivl_cap = need_rows;
        }
        c->tab_h = th;
        c->tab_w = tw;
    }
    if (n > 0) {
        std::vector<double> m(n), I(n);
        for (int i = 0; i < n; ++i) {
            m[i] = c->p.rho_s * M_PI * r[i] * r[i];   // disk of unit depth
            I[i] = 0.5 * m[i] * r[i] * r[i];
        }
        CK(cudaMemcpy(c->x, x, 16 * (size_t)n, cudaMemcpyHostToDevice), "copy x");
        CK(cudaMemcpy(c->v, v, 16 * (size_t)n, cudaMemcpyHostToDevice), "copy v");
        CK(cudaMemcpy(c->w, omega, 8 * (size_t)n, cudaMemcpyHostToDevice), "copy omega");
        CK(cudaMemcpy(c->r, r, 8 * (size_t)n, cudaMemcpyHostToDevice), "copy r");
        CK(cudaMemcpy(c->m, m.data(), 8 * (size_t)n, cudaMemcpyHostToDevice), "copy m");
        CK(cudaMemcpy(c->I, I.data(), 8 * (size_t)n, cudaMemcpyHostToDevice), "copy I");
        for (int b = 0; b < 2; ++b) CK(cudaMemset(c->nbr_cnt[b], 0, 4 * (size_t)n), "reset history");
        CK(cudaMemset(c->wall_xi, 0, 32 * (size_t)n), "reset wall history");
        CK(cudaMemset(c->F, 0, 16 * (size_t)n), "reset forces");
        CK(cudaMemset(c->T, 0, 8 * (size_t)n), "reset torques");
    }
    CK(cudaMemset(c->counters, 0, 32), "reset counters");
    int rc = rebuild_table(c, nullptr, false);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream), "sync");
    return IMB_OK;
}

// Every centre (x[2i], x[2i+1]) inside [0, nx) x [0, ny), NaN failing: a branch-free pass (the
// check sits between two host-coupled steps, before the next step's first launch)
static bool centres_inside(const double *x, int n, int nx, int ny) {
    const double X = (double)nx, Y = (double)ny;
    int ok = 1;
    for (int i = 0; i < n; ++i) {
        const double a = x[2 * i], b = x[2 * i + 1];
        ok &= (int)(a >= 0.0) & (int)(a < X) & (int)(b >= 0.0) & (int)(b < Y);
    }
    return ok != 0;
}

// The device address of a pinned host array the device can address (page-locked and mapped,
// as cudaHostAlloc / cudaHostRegister give under unified addressing), else NULL.
template <typename T>
static T *device_view(T *p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error an unknown pointer leaves
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? static_cast<T *>(at.devicePointer) : nullptr;
}

extern "C" int imb_set_kinematics(imb_ctx *c, const double *x, const double *v, const double *omega) {
    if (!c) return IMB_E_INVALID_ARG;
    if (c->np == 0) return IMB_OK;
    if (!x || !v || !omega) return fail(c, IMB_E_INVALID_ARG, "bad kinematics arrays");
    if (!centres_inside(x, c->np, c->nx, c->ny))
        return fail(c, IMB_E_INVALID_ARG, "particle centre outside [0,nx) x [0,ny)");
    const double *dx = device_view(x), *dv = device_view(v), *dw = device_view(omega);
    if (dx && dv && dw) {   // one launch reads the three arrays from host memory
        CK(launch_kinematics_in(dx, dv, dw, c->x, c->v, c->w, c->np, c->stream), "upload kinematics");
        c->launches++;
    } else {
        CK(cudaMemcpyAsync(c->x, x, 16 * (size_t)c->np, cudaMemcpyHostToDevice, c->stream), "copy x");
        CK(cudaMemcpyAsync(c->v, v, 16 * (size_t)c->np, cudaMemcpyHostToDevice, c->stream), "copy v");
        CK(cudaMemcpyAsync(c->w, omega, 8 * (size_t)c->np, cudaMemcpyHostToDevice, c->stream), "copy omega");
    }
    // with the DEM on, the next coupling cycle starts from the bins and rebuilds the map after
    // moving the particles, so the tile lists and solid-ratio tables would go unused
    return rebuild_table(c, nullptr, false, c->p.dem_on != 0);
}

// ------------------------------------------------------------- stepping
static int dem_cycle(imb_ctx *c, bool zero_forces) {
    DemArgs d = dem_args(c);
    CK(launch_dem_neighbours(d, c->stream), "dem neighbours");
    CK(launch_dem_islands_setup(d, c->stream), "dem islands");
    CK(launch_dem_local(d, c->stream), "dem free particles and islands");
    CK(launch_dem_coupled(d, dem_coupled_blocks(), c->stream), "dem coupled");
    c->launches += 7;   // neighbours, link, label, alloc, fill, free particles and islands, coupled
    c->nbr_cur ^= 1;
    return rebuild_table(c, c->xs, zero_forces);
}

static int lattice_step(imb_ctx *c) {
    // every particle's force and torque are written whole by the force gather below
    LatticeArgs a = lattice_args(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        while (c->events.size() < c->ev_used + 2) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e), "cudaEventCreate");
            c->events.push_back(e);
        }
        e0 = c->events[c->ev_used];
        e1 = c->events[c->ev_used + 1];
        c->ev_used += 2;
        // (an event-record node of its own when the steps are captured)
        CK(cudaEventRecordWithFlags(e0, c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault),
           "event record");
    }
    CK(launch_stream_collide(c->fbuf[c->cur], c->fbuf[c->cur ^ 1], c->p.storage, a, &c->tmap[c->cur][0],
                             &c->tmap[c->cur][1], c->tiles, c->tile_force, c->small, c->stream),
       "stream-collide");
    CK(launch_step_tail(c->fbuf[c->cur ^ 1], c->p.storage, a, c->tile_force, c->stream), "forces and ghosts");
    c->launches += 2;
    if (c->timing)
        CK(cudaEventRecordWithFlags(e1, c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault),
           "event record");
    c->cur ^= 1;
    return IMB_OK;
}

// Steps from a CUDA graph: `dem` one coupling cycle with the DEM (DEM, particle map,
// stream-collide, tail, ~25 kernels), else GRAPH_STEPS lattice steps.  Captured on first use for
// the current buffers, then replayed with one launch, so that the kernels reach the GPU without a
// host launch each.  With kernel timing on, the events that bracket each stream-collide and its
// tail are event-record nodes, pointed at the context's next events before every replay.  A
// stream that is already capturing is left alone, and a capture that fails turns graphs off:
// the steps then run as launches.
static int graph_steps(imb_ctx *c, bool dem, bool &done) {
    done = false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!c->use_graphs || cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return IMB_OK;
    const int steps = dem ? 1 : GRAPH_STEPS, nev = c->timing ? 2 * steps : 0;
    StepGraph &sg = c->graphs[dem ? 4 * (int)c->timing + 2 * c->cur + c->nbr_cur : 8 + 2 * (int)c->timing + c->cur];
    while (c->events.size() < c->ev_used + nev) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e), "cudaEventCreate");
        c->events.push_back(e);
    }
    if (!sg.exec) {
        const int cur0 = c->cur, nbr0 = c->nbr_cur;
        const long long l0 = c->launches;
        const size_t ev0 = c->ev_used;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->use_graphs = false;
            return IMB_OK;
        }
        c->capturing = true;
        int rc = dem ? dem_cycle(c, true) : IMB_OK;
        for (int t = 0; t < steps && !rc; ++t) rc = lattice_step(c);
        c->capturing = false;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        sg.cur_after = c->cur;
        sg.nbr_after = c->nbr_cur;
        sg.launches = c->launches - l0;
        c->cur = cur0;   // the capture ran nothing
        c->nbr_cur = nbr0;
        c->launches = l0;
        c->ev_used = ev0;
        bool ok = !rc && e == cudaSuccess && g;
        sg.ev.assign(nev, nullptr);
        if (ok && nev) {   // the nodes that record the events, in the order the steps record them
            size_t nn = 0;
            ok = cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess;
            std::vector<cudaGraphNode_t> nodes(nn);
            ok = ok && cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess;
            for (size_t i = 0; ok && i < nn; ++i) {
                cudaGraphNodeType t;
                cudaEvent_t ev = nullptr;
                if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) ok = false;
                else if (t == cudaGraphNodeTypeEventRecord && cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) == cudaSuccess)
                    for (int h = 0; h < nev; ++h)
                        if (ev == c->events[ev0 + h]) sg.ev[h] = nodes[i];
            }
            for (int h = 0; h < nev; ++h) ok = ok && sg.ev[h];
        }
        cudaGraphExec_t x = nullptr;
        ok = ok && cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
        if (!ok) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            c->msg.clear();
            sg = StepGraph();
            c->use_graphs = false;
            return IMB_OK;
        }
        sg.graph = g;   // kept: the event nodes are the graph's
        sg.exec = x;
    }
    for (int h = 0; h < nev; ++h)
        CK(cudaGraphExecEventRecordNodeSetEvent(sg.exec, sg.ev[h], c->events[c->ev_used + h]), "timing events");
    c->ev_used += nev;
    CK(cudaGraphLaunch(sg.exec, c->stream), "step graph");
    c->launches += sg.launches;
    c->cur = sg.cur_after;
    c->nbr_cur = sg.nbr_after;
    done = true;
    return IMB_OK;
}

static int queue_steps(imb_ctx *c, int n) {
    if (!c) return IMB_E_INVALID_ARG;
    if (n < 0) return fail(c, IMB_E_INVALID_ARG, "n must be >= 0");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const bool dem = c->p.dem_on && c->np > 0;
    for (int t = 0; t < n;) {
        // (timed lattice steps stay launches: the events between steps cost more in a graph)
        if (dem || (n - t >= GRAPH_STEPS && !c->timing)) {
            bool done = false;
            int rc = graph_steps(c, dem, done);
            if (rc) return rc;
            if (done) {
                t += dem ? 1 : GRAPH_STEPS;
                continue;
            }
        }
        if (dem) {
            int rc = dem_cycle(c, true);
            if (rc) return rc;
        }
        int rc = lattice_step(c);
        if (rc) return rc;
        ++t;
    }
    return IMB_OK;
}

// Wait for the stream with a deadline: poll without sleeping for the first 2 ms (the usual
// wait of a coupling cycle), then with 20 us sleeps.
static int bounded_wait(imb_ctx *c) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return IMB_OK;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "stream");
        const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if (us > 1000LL * c->p.timeout_ms) return fail(c, IMB_E_TIMEOUT, "timed out waiting for the GPU");
        if (us > 2000) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" int imb_sync(imb_ctx *c) {
    if (!c) return IMB_E_INVALID_ARG;
    // the error word travels with the stream's work, into pinned host memory
    CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "read error flags");
    int rc = bounded_wait(c);
    if (rc) return rc;
    const unsigned bits = *c->h_err;
    if (!bits) return IMB_OK;
    CK(cudaMemset(c->err, 0, sizeof(unsigned)), "clear error flags");
    if (bits & ERR_UNSTABLE) return fail(c, IMB_E_UNSTABLE, "NaN or |u| >= 0.3 (Mach guard)");
    if (bits & ERR_CELL_SLOTS) return fail(c, IMB_E_OVERFLOW, "more than 4 particles cover one cell");
    if (bits & ERR_TILE_LIST) return fail(c, IMB_E_OVERFLOW, "more than 32 particles touch one tile");
    if (bits & ERR_NEIGHBOURS) return fail(c, IMB_E_OVERFLOW, "DEM neighbour list full (16)");
    if (bits & ERR_BARRIER) return fail(c, IMB_E_TIMEOUT, "DEM grid barrier timed out");
    if (bits & ERR_TMA) return fail(c, IMB_E_TIMEOUT, "wait on a stream-collide tile copy timed out");
    if (bits & ERR_SKIN) return fail(c, IMB_E_SKIN, "a particle moved more than skin/2 in one step");
    if (bits & ERR_LIST) return fail(c, IMB_E_STATE, "a per-cycle DEM particle list overflowed");
    return fail(c, IMB_E_CUDA, "unknown device error flag");
}

extern "C" int imb_step_async(imb_ctx *c, int n) { return queue_steps(c, n); }

extern "C" int imb_step(imb_ctx *c, int n) {
    int rc = queue_steps(c, n);
    if (rc) return rc;
    return imb_sync(c);
}

extern "C" int imb_step_io(imb_ctx *c, int n, const double *x_in, const double *v_in, const double *omega_in,
                           double *F_out, double *T_out, double *x_out, double *v_out, double *omega_out) {
    if (!c) return IMB_E_INVALID_ARG;
    const bool in = x_in || v_in || omega_in;
    if (in && !(x_in && v_in && omega_in)) return fail(c, IMB_E_INVALID_ARG, "give x_in, v_in and omega_in together");
    int rc;
    if (in && (rc = imb_set_kinematics(c, x_in, v_in, omega_in))) return rc;
    if ((rc = queue_steps(c, n))) return rc;
    const size_t np = (size_t)c->np;
    double *outs[5] = {F_out, T_out, x_out, v_out, omega_out}, *dev[5];
    bool mapped = true;
    for (int k = 0; k < 5; ++k) {
        dev[k] = device_view(outs[k]);
        if (outs[k] && !dev[k]) mapped = false;
    }
    if (np && mapped) {   // one launch writes every output into host memory
        CK(launch_state_out(c->F, c->T, c->x, c->v, c->w, dev[0], dev[1], dev[2], dev[3], dev[4], c->np, c->stream),
           "read back");
        c->launches++;
    } else if (np) {
        if (F_out) CK(cudaMemcpyAsync(F_out, c->F, 16 * np, cudaMemcpyDeviceToHost, c->stream), "copy F");
        if (T_out) CK(cudaMemcpyAsync(T_out, c->T, 8 * np, cudaMemcpyDeviceToHost, c->stream), "copy T");
        if (x_out) CK(cudaMemcpyAsync(x_out, c->x, 16 * np, cudaMemcpyDeviceToHost, c->stream), "copy x");
        if (v_out) CK(cudaMemcpyAsync(v_out, c->v, 16 * np, cudaMemcpyDeviceToHost, c->stream), "copy v");
        if (omega_out) CK(cudaMemcpyAsync(omega_out, c->w, 8 * np, cudaMemcpyDeviceToHost, c->stream), "copy w");
    }
    return imb_sync(c);
}

extern "C" int imb_dem_step(imb_ctx *c, int n) {
    if (!c) return IMB_E_INVALID_ARG;
    if (n < 0) return fail(c, IMB_E_INVALID_ARG, "n must be >= 0");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    for (int t = 0; t < n && c->np > 0; ++t) {
        int rc = dem_cycle(c, false);
        if (rc) return rc;
    }
    return imb_sync(c);
}

// ------------------------------------------------------------- readback
template <typename T>
struct DevTmp {
    T *p = nullptr;
    ~DevTmp() { if (p) cudaFree(p); }
};

extern "C" int imb_get_populations(imb_ctx *c, double *f) {
    if (!c || !f) return IMB_E_INVALID_ARG;
    int rc = imb_sync(c);
    if (rc) return rc;
    size_t n = (size_t)9 * c->nx * c->ny;
    DevTmp<double> t;
    CK(dalloc(&t.p, n), "readback buffer");
    LatticeArgs a = lattice_args(c);
    CK(launch_gather(c->fbuf[c->cur], c->p.storage, a, t.p, nullptr, nullptr, nullptr, c->stream), "gather");
    c->launches++;
    CK(cudaMemcpyAsync(f, t.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy f");
    return imb_sync(c);
}

extern "C" int imb_get_macro(imb_ctx *c, double *rho, double *ux, double *uy) {
    if (!c || !rho || !ux || !uy) return IMB_E_INVALID_ARG;
    int rc = imb_sync(c);
    if (rc) return rc;
    size_t n = (size_t)c->nx * c->ny;
    DevTmp<double> t;
    CK(dalloc(&t.p, 3 * n), "readback buffer");
    LatticeArgs a = lattice_args(c);
    CK(launch_gather(c->fbuf[c->cur], c->p.storage, a, nullptr, t.p, t.p + n, t.p + 2 * n, c->stream), "gather");
    c->launches++;
    CK(cudaMemcpyAsync(rho, t.p, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy rho");
    CK(cudaMemcpyAsync(ux, t.p + n, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy ux");
    CK(cudaMemcpyAsync(uy, t.p + 2 * n, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy uy");
    return imb_sync(c);
}

extern "C" int imb_get_forces(imb_ctx *c, double *F, double *T) {
    if (!c || (c->np && (!F || !T))) return IMB_E_INVALID_ARG;
    if (c->np == 0) return IMB_OK;
    CK(cudaMemcpyAsync(F, c->F, 16 * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream), "copy F");
    CK(cudaMemcpyAsync(T, c->T, 8 * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream), "copy T");
    return imb_sync(c);
}

extern "C" int imb_set_forces(imb_ctx *c, const double *F, const double *T) {
    if (!c || (c->np && (!F || !T))) return IMB_E_INVALID_ARG;
    if (c->np == 0) return IMB_OK;
    CK(cudaMemcpyAsync(c->F, F, 16 * (size_t)c->np, cudaMemcpyHostToDevice, c->stream), "copy F");
    CK(cudaMemcpyAsync(c->T, T, 8 * (size_t)c->np, cudaMemcpyHostToDevice, c->stream), "copy T");
    return imb_sync(c);
}

extern "C" int imb_get_particles(imb_ctx *c, double *x, double *v, double *omega) {
    if (!c || (c->np && (!x || !v || !omega))) return IMB_E_INVALID_ARG;
    if (c->np == 0) return IMB_OK;
    CK(cudaMemcpyAsync(x, c->x, 16 * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream), "copy x");
    CK(cudaMemcpyAsync(v, c->v, 16 * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream), "copy v");
    CK(cudaMemcpyAsync(omega, c->w, 8 * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream), "copy w");
    return imb_sync(c);
}

extern "C" int imb_get_cell_map(imb_ctx *c, int *count, int *ids, float *eps) {
    if (!c || !count || !ids || !eps) return IMB_E_INVALID_ARG;
    int rc = imb_sync(c);
    if (rc) return rc;
    size_t n = (size_t)c->nx * c->ny;
    DevTmp<int> tc, ti;
    DevTmp<float> te;
    CK(dalloc(&tc.p, n), "readback buffer");
    CK(dalloc(&ti.p, n * MAX_SLOTS), "readback buffer");
    CK(dalloc(&te.p, n * MAX_SLOTS), "readback buffer");
    if (c->np == 0) {
        std::fill(count, count + n, 0);
        std::fill(ids, ids + n * MAX_SLOTS, -1);
        std::fill(eps, eps + n * MAX_SLOTS, 0.0f);
        return IMB_OK;
    }
    LatticeArgs a = lattice_args(c);
    CK(launch_cell_map(a, tc.p, ti.p, te.p, c->stream), "cell map");
    c->launches++;
    CK(cudaMemcpyAsync(count, tc.p, n * 4, cudaMemcpyDeviceToHost, c->stream), "copy count");
    CK(cudaMemcpyAsync(ids, ti.p, n * 4 * MAX_SLOTS, cudaMemcpyDeviceToHost, c->stream), "copy ids");
    CK(cudaMemcpyAsync(eps, te.p, n * 4 * MAX_SLOTS, cudaMemcpyDeviceToHost, c->stream), "copy eps");
    return imb_sync(c);
}

extern "C" int imb_get_contacts(imb_ctx *c, int max_pairs, int *pairs, int *n_pairs) {
    if (!c || !n_pairs || max_pairs < 0 || (max_pairs > 0 && !pairs)) return IMB_E_INVALID_ARG;
    *n_pairs = 0;
    if (c->np == 0) return IMB_OK;
    int rc = imb_sync(c);
    if (rc) return rc;
    const int max_per = 32;
    const int reach = (int)std::ceil(2.0 * c->r_max / TILE);
    DevTmp<int> tc, tp;
    CK(dalloc(&tc.p, c->np), "contacts buffer");
    CK(dalloc(&tp.p, (size_t)c->np * max_per), "contacts buffer");
    CK(launch_contacts(c->x, c->r, c->np, c->nx, c->ny, c->p.bc_x, c->p.bc_y, c->bin_start, c->bin_ids,
                       c->pbin, c->nbx, c->nby, reach, tc.p, tp.p, max_per, c->stream),
       "contacts");
    c->launches++;
    std::vector<int> cnt(c->np), lst((size_t)c->np * max_per);
    CK(cudaMemcpyAsync(cnt.data(), tc.p, 4 * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaMemcpyAsync(lst.data(), tp.p, 4 * lst.size(), cudaMemcpyDeviceToHost, c->stream), "copy");
    rc = imb_sync(c);
    if (rc) return rc;
    std::vector<std::pair<int, int>> all;
    for (int a = 0; a < c->np; ++a) {
        if (cnt[a] > max_per) return fail(c, IMB_E_OVERFLOW, "more than 32 contacts of one particle");
        for (int k = 0; k < cnt[a]; ++k) all.emplace_back(a, lst[(size_t)a * max_per + k]);
    }
    std::sort(all.begin(), all.end());
    *n_pairs = (int)all.size();
    for (int k = 0; k < (int)all.size() && k < max_pairs; ++k) {
        pairs[2 * k] = all[k].first;
        pairs[2 * k + 1] = all[k].second;
    }
    return IMB_OK;
}

extern "C" int imb_get_bins(imb_ctx *c, int *bin_start, int *bin_ids) {
    if (!c || !bin_start || (c->np && !bin_ids)) return IMB_E_INVALID_ARG;
    int rc = imb_sync(c);
    if (rc) return rc;
    CK(cudaMemcpy(bin_start, c->bin_start, 4 * (size_t)(c->nbins + 1), cudaMemcpyDeviceToHost), "copy");
    if (c->np == 0) return IMB_OK;
    CK(cudaMemcpy(bin_ids, c->bin_ids, 4 * (size_t)c->np, cudaMemcpyDeviceToHost), "copy");
    for (int b = 0; b < c->nbins; ++b) std::sort(bin_ids + bin_start[b], bin_ids + bin_start[b + 1]);
    return IMB_OK;
}

// ---------------------------------------------------------------- misc
extern "C" int imb_set_stream(imb_ctx *c, void *stream) {
    if (!c) return IMB_E_INVALID_ARG;
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    return IMB_OK;
}

extern "C" void *imb_get_stream(imb_ctx *c) { return c ? (void *)c->stream : nullptr; }

extern "C" int imb_enable_kernel_timing(imb_ctx *c, int on) {
    if (!c) return IMB_E_INVALID_ARG;
    c->timing = on != 0;
    c->ev_used = 0;
    return IMB_OK;
}

extern "C" int imb_kernel_time(imb_ctx *c, double *ms, long long *launches) {
    if (!c || !ms || !launches) return IMB_E_INVALID_ARG;
    int rc = bounded_wait(c);
    if (rc) return rc;
    double tot = 0.0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, c->events[k], c->events[k + 1]), "event elapsed");
        tot += t;
    }
    *ms = tot;
    *launches = (long long)(c->ev_used / 2);
    c->ev_used = 0;
    return IMB_OK;
}

extern "C" long long imb_launch_count(imb_ctx *c) { return c ? c->launches : 0; }

extern "C" double imb_bytes_per_cell(imb_ctx *c) { return c ? 18.0 * (double)c->elem : 0.0; }

extern "C" const char *imb_last_error(imb_ctx *c) {
    return c ? c->msg.c_str() : g_init_error.c_str();
}

// ------------------------------------------------------------------ drag gradient
// Reverse-mode gradient of the time-averaged drag J = (1/T) sum_t sum_p F_x,p(t) of T steps
// (Eq. 15 forces) with respect to the inlet velocity, tau and the disk centres.  The adjoint
// of step t needs the post-collision field the step starts from ("state t"); how the states
// are kept is the checkpointing scheme: uniform (every K-th state, a segment recomputed at a
// time) or binomial (a fixed number of snapshots placed by the recursive binomial schedule).
namespace {

struct GradBufs {
    size_t ncell = 0, state = 0, sb = 0;   // cells, floats per state, bytes per state
    DevTmp<float> lam, Eb, fin;
    DevTmp<double> acc, gE, gx, Fsave;
    DevTmp<int> cnt, ids;
    DevTmp<float> epsb;
    float *lam1 = nullptr, *lam0 = nullptr;   // d J / d f(t+1), d J / d f(t)
    float inv_T = 0.0f;
};

int grad_prepare(imb_ctx *c, int T, GradBufs &g) {
    if (c->p.dem_on || c->C_smag != 0.0 || c->p.Fx != 0.0 || c->p.Fy != 0.0 || c->p.eps_mode != IMB_EPS_EXACT ||
        c->p.storage != IMB_STORE_FP32 || c->p.wall_u_bot != 0.0 || c->p.wall_u_top != 0.0)
        return fail(c, IMB_E_INVALID_ARG, "drag gradient needs DEM off, C_smag = 0, no body force, exact solid "
                                          "ratio, FP32 storage and walls at rest");
    int rc = imb_sync(c);
    if (rc) return rc;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const int np = c->np;
    if (np > 0) {   // disks at rest
        std::vector<double> hv(2 * (size_t)np), hw(np);
        CK(cudaMemcpy(hv.data(), c->v, 16 * (size_t)np, cudaMemcpyDeviceToHost), "read v");
        CK(cudaMemcpy(hw.data(), c->w, 8 * (size_t)np, cudaMemcpyDeviceToHost), "read w");
        for (int i = 0; i < np; ++i)
            if (hv[2 * i] != 0.0 || hv[2 * i + 1] != 0.0 || hw[i] != 0.0)
                return fail(c, IMB_E_INVALID_ARG, "drag gradient needs disks at rest");
    }
    g.ncell = (size_t)c->nx * c->ny;
    g.state = 9 * c->plane;
    g.sb = g.state * sizeof(float);
    g.inv_T = 1.0f / (float)T;
    CK(dalloc(&g.lam.p, 2 * g.state), "adjoint buffers");
    CK(dalloc(&g.fin.p, g.state), "final state");
    CK(dalloc(&g.Eb.p, g.ncell), "solid ratio");
    CK(dalloc(&g.gE.p, g.ncell), "solid-ratio gradient");
    CK(dalloc(&g.acc.p, 4), "accumulators");
    CK(dalloc(&g.gx.p, 2 * (size_t)std::max(np, 1)), "position gradient");
    CK(dalloc(&g.Fsave.p, 3 * (size_t)std::max(np, 1)), "force copy");
    CK(dalloc(&g.cnt.p, g.ncell), "cell map");
    CK(dalloc(&g.ids.p, g.ncell * MAX_SLOTS), "cell map");
    CK(dalloc(&g.epsb.p, g.ncell * MAX_SLOTS), "cell map");
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(g.acc.p, 0, 4 * sizeof(double), s), "clear");
    CK(cudaMemsetAsync(g.gE.p, 0, g.ncell * sizeof(double), s), "clear");
    CK(cudaMemsetAsync(g.gx.p, 0, 2 * (size_t)std::max(np, 1) * sizeof(double), s), "clear");
    CK(cudaMemsetAsync(g.lam.p, 0, 2 * g.sb, s), "clear");
    CK(cudaMemsetAsync(g.Eb.p, 0, g.ncell * sizeof(float), s), "clear");
    g.lam1 = g.lam.p;
    g.lam0 = g.lam.p + g.state;
    if (np > 0) {
        LatticeArgs a = lattice_args(c);
        CK(launch_cell_map(a, g.cnt.p, g.ids.p, g.epsb.p, s), "cell map");
        CK(launch_cell_E(g.cnt.p, g.epsb.p, g.ncell, g.Eb.p, s), "solid ratio");
        c->launches += 2;
    }
    return IMB_OK;
}

// one forward step whose drag enters J
int grad_forward_step(imb_ctx *c, GradBufs &g) {
    int rc = lattice_step(c);
    if (rc) return rc;
    if (c->np > 0) {
        CK(launch_drag_sum(c->F, c->np, g.acc.p, c->stream), "drag");
        c->launches++;
    }
    return IMB_OK;
}

// the state after the T steps and its forces, kept for the end of the call
int grad_keep_final(imb_ctx *c, GradBufs &g) {
    cudaStream_t s = c->stream;
    CK(cudaMemcpyAsync(g.fin.p, c->fbuf[c->cur], g.sb, cudaMemcpyDeviceToDevice, s), "final state");
    if (c->np > 0) {
        CK(cudaMemcpyAsync(g.Fsave.p, c->F, 16 * (size_t)c->np, cudaMemcpyDeviceToDevice, s), "forces");
        CK(cudaMemcpyAsync(g.Fsave.p + 2 * (size_t)c->np, c->T, 8 * (size_t)c->np, cudaMemcpyDeviceToDevice, s),
           "torques");
    }
    return IMB_OK;
}

// Adjoint of step t from state t (S0): d J / d f(t+1) -> d J / d f(t), plus the tau and
// solid-ratio terms; then, for t >= 1, the transpose of the inlet/outlet rule that produced
// f(t) from state t (it adds the inlet-velocity term), so that the next unit starts from the
// full d J / d f(t).
int grad_unit(imb_ctx *c, GradBufs &g, int t, const float *S0) {
    LatticeArgs a = lattice_args(c);
    cudaStream_t s = c->stream;
    CK(launch_adjoint_step(g.lam1, S0, g.lam0, a, g.Eb.p, g.gE.p, g.inv_T, g.acc.p + 1, s), "adjoint step");
    c->launches++;
    std::swap(g.lam1, g.lam0);
    if (t >= 1 && c->p.bc_x == IMB_BC_INLET_OUTLET) {
        CK(launch_adjoint_inlet(g.lam1, S0, a, g.acc.p + 2, s), "adjoint inlet");
        c->launches++;
    }
    return IMB_OK;
}

int grad_finish(imb_ctx *c, GradBufs &g, int T, double *J, double *dJ_duin, double *dJ_dtau, double *dJ_dx) {
    cudaStream_t s = c->stream;
    const int np = c->np;
    CK(cudaMemcpyAsync(c->fbuf[c->cur], g.fin.p, g.sb, cudaMemcpyDeviceToDevice, s), "restore final state");
    if (np > 0) {
        CK(cudaMemcpyAsync(c->F, g.Fsave.p, 16 * (size_t)np, cudaMemcpyDeviceToDevice, s), "forces");
        CK(cudaMemcpyAsync(c->T, g.Fsave.p + 2 * (size_t)np, 8 * (size_t)np, cudaMemcpyDeviceToDevice, s), "torques");
        CK(launch_position_grad(g.cnt.p, g.ids.p, g.gE.p, c->x, c->r, c->nx, c->ny, c->p.bc_x, c->p.bc_y, g.gx.p, s),
           "position gradient");
        c->launches++;
    }
    double h[4];
    CK(cudaMemcpyAsync(h, g.acc.p, sizeof(h), cudaMemcpyDeviceToHost, s), "accumulators");
    if (np > 0) CK(cudaMemcpyAsync(dJ_dx, g.gx.p, 16 * (size_t)np, cudaMemcpyDeviceToHost, s), "gradient");
    int rc = imb_sync(c);
    if (rc) return rc;
    *J = h[0] / T;
    *dJ_dtau = h[1];
    *dJ_duin = h[2];
    return IMB_OK;
}

// ---- binomial checkpointing schedule (Griewank's recursive reversal) ----
// C(s + r, s), saturated far above any step count
long long binom_beta(int s, int r) {
    if (r < 0) return 0;
    long double v = 1.0L;
    for (int k = 1; k <= s; ++k) {
        v = v * (long double)(r + k) / (long double)k;
        if (v > 4.0e18L) return (long long)4e18;
    }
    return (long long)(v + 0.5L);
}

struct Sched {
    std::vector<int> ops;   // (kind, argument) pairs
    long long advances = 0;
    int cur = 0;            // time of the state in the working buffer
    std::vector<int> slot_t, free_slots;
    void emit(int k, int v) {
        ops.push_back(k);
        ops.push_back(v);
    }
    void restore(int slot) {
        if (cur != slot_t[slot]) {
            emit(IMB_CK_RESTORE, slot);
            cur = slot_t[slot];
        }
    }
    void advance(int n) {
        emit(IMB_CK_ADVANCE, n);
        cur += n;
        advances += n;
    }
    // adjoints of steps b-1 .. a; state a is in `slot`, s snapshots are free
    void reverse(int a, int b, int s, int slot) {
        const int l = b - a;
        if (l == 1) {
            restore(slot);
            emit(IMB_CK_ADJOINT, a);
            return;
        }
        if (s == 0) {   // no snapshot left: recompute every state from state a
            for (int t = b - 1; t >= a; --t) {
                restore(slot);
                if (t > a) advance(t - a);
                emit(IMB_CK_ADJOINT, t);
            }
            return;
        }
        // repetition number r: the least with C(s + 1 + r, r) >= l; then a first snapshot j
        // steps on, the left part [a, a + j) reversed with the same snapshots, the right part
        // with one fewer, both within their repetition budgets (r - 1 and r)
        int r = 0;
        while (binom_beta(s + 1, r) < l) ++r;
        long long j = std::max(binom_beta(s + 1, r - 2), (long long)l - binom_beta(s, r));
        j = std::max(1LL, std::min(j, (long long)l - 1));
        restore(slot);
        advance((int)j);
        const int sl = free_slots.back();
        free_slots.pop_back();
        slot_t[sl] = cur;
        emit(IMB_CK_STORE, sl);
        reverse(a + (int)j, b, s - 1, sl);
        free_slots.push_back(sl);
        reverse(a, a + (int)j, s, slot);
    }
};

void binomial_schedule(int T, int snapshots, Sched &sc) {
    const int s = std::max(0, std::min(snapshots, T - 1));
    sc.slot_t.assign(s + 1, -1);
    for (int k = s; k >= 1; --k) sc.free_slots.push_back(k);
    sc.slot_t[0] = 0;
    sc.emit(IMB_CK_STORE, 0);
    sc.reverse(0, T, s, 0);
}

}  // namespace

extern "C" int imb_binomial_schedule(int T, int snapshots, int *ops, int max_ops, int *n_ops,
                                     long long *n_advances) {
    if (T < 1 || snapshots < 0 || max_ops < 0 || (max_ops > 0 && !ops) || !n_ops) return IMB_E_INVALID_ARG;
    Sched sc;
    binomial_schedule(T, snapshots, sc);
    const int n = (int)(sc.ops.size() / 2);
    for (int k = 0; k < std::min(n, max_ops); ++k) {
        ops[2 * k] = sc.ops[2 * k];
        ops[2 * k + 1] = sc.ops[2 * k + 1];
    }
    *n_ops = n;
    if (n_advances) *n_advances = sc.advances;
    return IMB_OK;
}

extern "C" int imb_drag_gradient(imb_ctx *c, int T, int checkpoint_every, double *J, double *dJ_duin,
                                 double *dJ_dtau, double *dJ_dx) {
    if (!c || !J || !dJ_duin || !dJ_dtau || (c->np > 0 && !dJ_dx)) return IMB_E_INVALID_ARG;
    if (T < 1 || checkpoint_every < 1) return fail(c, IMB_E_INVALID_ARG, "T and checkpoint_every must be >= 1");
    GradBufs g;
    int rc = grad_prepare(c, T, g);
    if (rc) return rc;
    const int K = checkpoint_every, nck = (T + K - 1) / K;
    const size_t state = g.state, sb = g.sb;
    DevTmp<float> ck, seg;
    CK(dalloc(&ck.p, state * nck), "checkpoints");
    CK(dalloc(&seg.p, state * (size_t)std::min(K, T)), "segment states");
    cudaStream_t s = c->stream;
    // forward: every K-th state kept, the drag of every step summed
    for (int t = 0; t < T; ++t) {
        if (t % K == 0)
            CK(cudaMemcpyAsync(ck.p + state * (t / K), c->fbuf[c->cur], sb, cudaMemcpyDeviceToDevice, s), "checkpoint");
        if ((rc = grad_forward_step(c, g))) return rc;
    }
    if ((rc = grad_keep_final(c, g))) return rc;
    // backward, one checkpoint segment at a time: recompute its states, then walk back
    for (int j = nck - 1; j >= 0; --j) {
        const int t0 = j * K, t1 = std::min(T, t0 + K);
        CK(cudaMemcpyAsync(c->fbuf[c->cur], ck.p + state * j, sb, cudaMemcpyDeviceToDevice, s), "restore");
        for (int t = t0; t < t1; ++t) {
            CK(cudaMemcpyAsync(seg.p + state * (t - t0), c->fbuf[c->cur], sb, cudaMemcpyDeviceToDevice, s), "segment");
            if (t + 1 < t1 && (rc = lattice_step(c))) return rc;
        }
        for (int t = t1 - 1; t >= t0; --t)
            if ((rc = grad_unit(c, g, t, seg.p + state * (t - t0)))) return rc;
    }
    return grad_finish(c, g, T, J, dJ_duin, dJ_dtau, dJ_dx);
}

extern "C" int imb_drag_gradient_binomial(imb_ctx *c, int T, int snapshots, double *J, double *dJ_duin,
                                          double *dJ_dtau, double *dJ_dx) {
    if (!c || !J || !dJ_duin || !dJ_dtau || (c->np > 0 && !dJ_dx)) return IMB_E_INVALID_ARG;
    if (T < 1 || snapshots < 0) return fail(c, IMB_E_INVALID_ARG, "T must be >= 1 and snapshots >= 0");
    GradBufs g;
    int rc = grad_prepare(c, T, g);
    if (rc) return rc;
    Sched sc;
    binomial_schedule(T, snapshots, sc);
    const size_t state = g.state, sb = g.sb;
    DevTmp<float> snap;
    CK(dalloc(&snap.p, state * sc.slot_t.size()), "snapshots");
    std::vector<int> slot_t(sc.slot_t.size(), -1);
    cudaStream_t s = c->stream;
    int cur_t = 0, done = 0;   // time of the working state; steps whose drag is in J
    for (size_t k = 0; k < sc.ops.size(); k += 2) {
        const int kind = sc.ops[k], v = sc.ops[k + 1];
        if (kind == IMB_CK_ADVANCE) {
            for (int n = 0; n < v; ++n, ++cur_t) {
                if (cur_t == done) {   // first pass over this step: its drag enters J
                    if ((rc = grad_forward_step(c, g))) return rc;
                    ++done;
                } else if ((rc = lattice_step(c))) {
                    return rc;
                }
            }
        } else if (kind == IMB_CK_STORE) {
            CK(cudaMemcpyAsync(snap.p + state * v, c->fbuf[c->cur], sb, cudaMemcpyDeviceToDevice, s), "snapshot");
            slot_t[v] = cur_t;
        } else if (kind == IMB_CK_RESTORE) {
            CK(cudaMemcpyAsync(c->fbuf[c->cur], snap.p + state * v, sb, cudaMemcpyDeviceToDevice, s), "restore");
            cur_t = slot_t[v];
        } else {   // IMB_CK_ADJOINT of step v from the working state
            if (v != cur_t) return fail(c, IMB_E_CUDA, "internal: checkpoint schedule out of order");
            if (v == T - 1) {   // the first adjoint: the last forward step completes J and the final state
                if (done != T - 1) return fail(c, IMB_E_CUDA, "internal: checkpoint schedule skipped a step");
                if ((rc = grad_forward_step(c, g))) return rc;
                ++done;
                if ((rc = grad_keep_final(c, g))) return rc;
                c->cur ^= 1;   // the step wrote the other buffer: state T - 1 is still in this one
            }
            if ((rc = grad_unit(c, g, v, (const float *)c->fbuf[c->cur]))) return rc;
        }
    }
    return grad_finish(c, g, T, J, dJ_duin, dJ_dtau, dJ_dx);
}
