// imb_particles.cu -- particle kernels of the GB300 IMB-LBM-DEM library.
//
//   k_particle_table  after every DEM update: bin of each particle (32 x 32 cells),
//                     the FP32 record read by the lattice kernels, the skin check,
//                     and zeroing of the hydrodynamic force accumulators;
//   k_bin_scan        exclusive scan of the bin counts (one block);
//   k_bin_fill        scatter of particle ids into their bins;
//   k_dem_neighbours  sorted neighbour candidates within r_a + r_b + skin, carrying
//                     the tangential spring of each pair over, and the split of the
//                     particles into free (no candidate) and coupled ones;
//   k_dem_local       the N_sub sub-cycles (Eq. 17) of the free particles (in registers)
//                     and of the islands of up to 32 particles (a warp each, or eight
//                     islands of up to four to a warp, in shared memory), in one launch;
//   k_dem_coupled     the N_sub sub-cycles of the coupled particles, one bounded grid
//                     barrier per sub-cycle (cooperative launch);
//   k_contacts        pairs in contact (Eq. 7) for readback.
//
// DEM arithmetic is FP64.  This file is compiled with --fmad=false so that every
// multiply and add is rounded separately; with the contact partners summed in
// ascending id order, particle trajectories then reproduce a plain sequential
// FP64 evaluation of Eqs. 7-11 exactly.
#include "imb_device.cuh"
#include "imb_kernels.h"

namespace imb {

// ------------------------------------------------------------- binning
__device__ __forceinline__ double min_image(double d, bool periodic, int L) {
    if (periodic) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

__device__ __forceinline__ int bin_of(double px, double py, int nbx, int nby) {
    int bx = (int)floor(px / (double)TILE), by = (int)floor(py / (double)TILE);
    bx = bx < 0 ? 0 : (bx >= nbx ? nbx - 1 : bx);
    by = by < 0 ? 0 : (by >= nby ? nby - 1 : by);
    return by * nbx + bx;
}

__global__ void k_particle_table(const double *__restrict__ x, const double *__restrict__ r,
                                 const double *__restrict__ x_start, int np, int nx, int ny, int bc_x,
                                 int bc_y, double skin_half, int nbx, int nby, int *bin_count, int *pbin,
                                 PRec *prec, const double *__restrict__ v, const double *__restrict__ w,
                                 double *F, double *T, unsigned *err) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double px = x[2 * p], py = x[2 * p + 1];
    const int b = bin_of(px, py, nbx, nby);
    pbin[p] = b;
    atomicAdd(&bin_count[b], 1);
    PRec P;
    P.ci = (int)floor(px);
    P.cj = (int)floor(py);
    P.fx = __double2float_rn(px - (double)P.ci);
    P.fy = __double2float_rn(py - (double)P.cj);
    P.r = __double2float_rn(r[p]);
    P.vx = __double2float_rn(v[2 * p]);
    P.vy = __double2float_rn(v[2 * p + 1]);
    P.w = __double2float_rn(w[p]);
    prec[p] = P;
    if (x_start) {
        const double dx = min_image(px - x_start[2 * p], bc_x == BC_PERIODIC, nx);
        const double dy = min_image(py - x_start[2 * p + 1], bc_y == BC_PERIODIC, ny);
        if (dx * dx + dy * dy > skin_half * skin_half) set_err(err, ERR_SKIN);
    }
    if (F) {
        F[2 * p] = 0.0;
        F[2 * p + 1] = 0.0;
        T[p] = 0.0;
    }
}

// Exclusive scan of the bin counts by one block: each thread owns 32 consecutive
// bins (eight 16-byte loads in flight), the block scans the per-thread sums.  Also
// resets the counts and fill cursors (and the DEM list counters) for reuse.  The
// bin arrays are padded to a multiple of 32 entries.
// Exclusive scan of the bin counts in two passes over blocks of SCAN_BINS bins: each
// block scans its bins and records their total, then adds the totals of the blocks
// before it.  Both passes also clear the counters that the next binning accumulates.
constexpr int SCAN_BINS = 1024;   // 256 threads x 4 bins

__device__ __forceinline__ int block_exclusive_scan(int v, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    total = wsum[nw - 1];
    return (warp ? wsum[warp - 1] : 0) + incl - v;
}

__global__ void __launch_bounds__(256) k_bin_scan_local(int *count, int *start, int nbins, int *bsum,
                                                        int *dem_counters) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    __shared__ int wsum[8];
    const int b0 = blockIdx.x * SCAN_BINS + threadIdx.x * 4;
    int4 v = make_int4(0, 0, 0, 0);
    if (b0 < nbins) v = *reinterpret_cast<const int4 *>(count + b0);   // counts padded to 32
    int total;
    int run = block_exclusive_scan(v.x + v.y + v.z + v.w, wsum, total);
    if (b0 < nbins) {
        int4 o;
        o.x = run; run += v.x;
        o.y = run; run += v.y;
        o.z = run; run += v.z;
        o.w = run;
        *reinterpret_cast<int4 *>(start + b0) = o;
        *reinterpret_cast<int4 *>(count + b0) = make_int4(0, 0, 0, 0);
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
    if (blockIdx.x == 0 && threadIdx.x < 6 && dem_counters) dem_counters[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(256) k_bin_scan_add(int *fill, int *start, int nbins, const int *bsum) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    __shared__ int s_off;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {   // totals of the blocks before this one
        int acc = 0;
        for (int i = lane; i < (int)blockIdx.x; i += 32) acc += bsum[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_off = acc;
    }
    __syncthreads();
    const int off = s_off;
    const int b0 = blockIdx.x * SCAN_BINS + threadIdx.x * 4;
    if (b0 < nbins) {
        int4 *p = reinterpret_cast<int4 *>(start + b0);
        int4 o = *p;
        o.x += off; o.y += off; o.z += off; o.w += off;
        *p = o;
        *reinterpret_cast<int4 *>(fill + b0) = make_int4(0, 0, 0, 0);
    }
    __syncthreads();
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) start[nbins] = off + bsum[blockIdx.x];
}

__global__ void k_bin_fill(const int *__restrict__ pbin, int np, int *fill, const int *__restrict__ start,
                           int *ids) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int b = pbin[p];
    ids[start[b] + atomicAdd(&fill[b], 1)] = p;
}

// ----------------------------------------------------------------- DEM
// Spring-dashpot contact seen from particle a (Eqs. 7-9): n from a to the partner,
// t = z x n, (dvx, dvy) partner minus a, rot = w_a r_a + w_b r_b, R* and m* the pair's
// reduced radius and mass.  Linear law (cn of the pair precomputed) or the simplified
// Hertz-Mindlin law of Sec. 2.2 (stiffness and dashpots from s = sqrt(R* delta)).
// Returns the force on a and the tangential force magnitude.
// Normal damping of a pair of reduced mass m* (set from the restitution coefficient).
__device__ __forceinline__ double damping_cn(const DemArgs &d, double mstar) {
    return 2.0 * d.zeta * sqrt(mstar * d.kn);
}

__device__ __forceinline__ void contact_law_cn(const DemArgs &d, double nxv, double nyv, double delta,
                                               double dvx, double dvy, double rot, double cn_lin,
                                               double Rstar, double mstar, double &xi, double &fx,
                                               double &fy, double &Ft) {
    const double tx = -nyv, ty = nxv;
    const double vn = dvx * nxv + dvy * nyv;
    const double vt = (dvx * tx + dvy * ty) - rot;
    double kn, kt, cn, ct;
    if (d.model == 1) {
        const double sq = sqrt(Rstar * delta);
        kn = d.hm_kn0 * sq;
        kt = d.hm_kt0 * sq;
        cn = d.hm_c0 * sqrt(d.hm_sn0 * sq * mstar);
        ct = d.hm_c0 * sqrt(d.hm_kt0 * sq * mstar);
    } else {
        kn = d.kn;
        kt = d.kt;
        cn = cn_lin;
        ct = d.ct_ratio * cn;
    }
    xi = xi + vt * d.dt;                     // incremental tangential spring (Eq. 9)
    const double Fn = kn * delta - cn * vn;  // Eq. 8, repulsive when positive
    double F_t = kt * xi + ct * vt;          // Eq. 9
    const double lim = d.mu * fabs(Fn);      // Coulomb cap
    if (fabs(F_t) > lim) {
        F_t = copysign(lim, F_t);
        xi = copysign(lim / kt, xi);
    }
    fx = -Fn * nxv + F_t * tx;
    fy = -Fn * nyv + F_t * ty;
    Ft = F_t;
}

__device__ __forceinline__ void contact_law(const DemArgs &d, double nxv, double nyv, double delta,
                                            double dvx, double dvy, double rot, double Rstar, double mstar,
                                            double &xi, double &fx, double &fy, double &Ft) {
    contact_law_cn(d, nxv, nyv, delta, dvx, dvy, rot, d.model == 1 ? 0.0 : damping_cn(d, mstar), Rstar, mstar,
                   xi, fx, fy, Ft);
}

// Force on particle p of its candidate q in slot j (seen from p), with the pair's tangential
// spring xi; the pair's damping constant is cached in the neighbour list.  Returns false (and
// releases the spring) without overlap.
__device__ __forceinline__ bool pair_force_xi(const DemArgs &d, const int p, const int j, const int q, double &xi,
                                              const double px, const double py, const double w, const double qx,
                                              const double qy, const double qvx, const double qvy, const double qw,
                                              const double vx, const double vy, double &fx, double &fy,
                                              double &Ft) {
    const bool perx = d.bc_x == BC_PERIODIC, pery = d.bc_y == BC_PERIODIC;
    const double rp = d.r[p];
    const double dx = min_image(qx - px, perx, d.nx);
    const double dy = min_image(qy - py, pery, d.ny);
    const double d2 = dx * dx + dy * dy;
    const double R = rp + d.r[q];
    if (!(d2 < R * R)) {  // Eq. 7: no overlap, the spring is released
        xi = 0.0;
        return false;
    }
    const double dist = sqrt(d2);
    const double nxv = dx / dist, nyv = dy / dist;
    const double rot = w * rp + qw * d.r[q];
    double Rstar = 0.0, mstar = 0.0;
    if (d.model == 1) {
        Rstar = rp * d.r[q] / (rp + d.r[q]);
        mstar = d.m[p] * d.m[q] / (d.m[p] + d.m[q]);
    }
    contact_law_cn(d, nxv, nyv, R - dist, qvx - vx, qvy - vy, rot, d.nbr_cn[p * MAX_NBR + j], Rstar, mstar, xi,
                   fx, fy, Ft);
    return true;
}

// The same for candidate slot j, its spring in the neighbour list.
__device__ __forceinline__ bool pair_force(const DemArgs &d, const int p, const int j, const double px,
                                           const double py, const double w, const double qx, const double qy,
                                           const double qvx, const double qvy, const double qw,
                                           const double vx, const double vy, double &fx, double &fy,
                                           double &Ft) {
    return pair_force_xi(d, p, j, d.nbr_id[p * MAX_NBR + j], d.nbr_xi[p * MAX_NBR + j], px, py, w, qx, qy, qvx,
                         qvy, qw, vx, vy, fx, fy, Ft);
}

// Walls on the domain edges of non-periodic axes, an immovable partner (m* = m).  Returns
// whether any wall touches.
__device__ __forceinline__ bool wall_contacts(const DemArgs &d, int p, double px, double py, double vx,
                                              double vy, double w, double rp, double mp, double *xiw,
                                              double &Fcx, double &Fcy, double &Tc) {
    bool touched = false;
#pragma unroll
    for (int wl = 0; wl < 4; ++wl) {
        const bool active = wl < 2 ? d.bc_x == BC_WALL : d.bc_y == BC_WALL;
        if (!active) continue;
        double dist, nxv, nyv;
        if (wl == 0) { dist = px; nxv = -1.0; nyv = 0.0; }
        else if (wl == 1) { dist = (double)d.nx - px; nxv = 1.0; nyv = 0.0; }
        else if (wl == 2) { dist = py; nxv = 0.0; nyv = -1.0; }
        else { dist = (double)d.ny - py; nxv = 0.0; nyv = 1.0; }
        if (!(dist < rp)) {
            xiw[wl] = 0.0;
            continue;
        }
        double fx, fy, Ft;
        contact_law(d, nxv, nyv, rp - dist, -vx, -vy, w * rp, rp, mp, xiw[wl], fx, fy, Ft);
        Fcx += fx;
        Fcy += fy;
        Tc += rp * Ft;
        touched = true;
    }
    return touched;
}

// The drift of the leapfrog update (Eq. 11), wrapped on periodic axes.
__device__ __forceinline__ void drift(const DemArgs &d, double &px, double &py, double vx, double vy) {
    px = px + vx * d.dt;
    py = py + vy * d.dt;
    if (d.bc_x == BC_PERIODIC) {
        if (px >= d.nx) px -= d.nx;
        else if (px < 0.0) px += d.nx;
    }
    if (d.bc_y == BC_PERIODIC) {
        if (py >= d.ny) py -= d.ny;
        else if (py < 0.0) py += d.ny;
    }
}

// Eqs. 10-11, leapfrog kick-drift.
__device__ __forceinline__ void integrate(const DemArgs &d, int p, double Fcx, double Fcy, double Tc,
                                          double &px, double &py, double &vx, double &vy, double &w) {
    const double ax = (Fcx + d.F[2 * p]) / d.m[p] + d.gx_eff;
    const double ay = (Fcy + d.F[2 * p + 1]) / d.m[p] + d.gy_eff;
    const double al = (Tc + d.T[p]) / d.I[p];
    vx = vx + ax * d.dt;
    vy = vy + ay * d.dt;
    w = w + al * d.dt;
    drift(d, px, py, vx, vy);
}

// The velocity increments a dt of a sub-cycle without contacts: integrate()'s operations on
// zero contact sums (0 + F), evaluated once per coupling cycle since F, T, m, I are fixed.
struct Kick {
    double dvx, dvy, dw;
};

__device__ __forceinline__ Kick free_kick(const DemArgs &d, int p) {
    const double ax = (0.0 + d.F[2 * p]) / d.m[p] + d.gx_eff;
    const double ay = (0.0 + d.F[2 * p + 1]) / d.m[p] + d.gy_eff;
    const double al = (0.0 + d.T[p]) / d.I[p];
    return {ax * d.dt, ay * d.dt, al * d.dt};
}

// integrate() when nothing touched in the sub-cycle, to the bit.
__device__ __forceinline__ void coast(const DemArgs &d, const Kick &k, double &px, double &py, double &vx,
                                      double &vy, double &w) {
    vx = vx + k.dvx;
    vy = vy + k.dvy;
    w = w + k.dw;
    drift(d, px, py, vx, vy);
}

// Motion of particle p over one coupling cycle when it touches nothing: the accelerations
// are evaluated once, with exactly the operations integrate() uses on zero contact sums.
struct FreeMotion {
    double ax, ay, al;   // accelerations
    double ex, ey;       // bounds on |x(t) - x(0)| per axis within the cycle
};

__device__ __forceinline__ FreeMotion free_motion(const DemArgs &d, int p, double vx, double vy) {
    FreeMotion f;
    f.ax = (0.0 + d.F[2 * p]) / d.m[p] + d.gx_eff;
    f.ay = (0.0 + d.F[2 * p + 1]) / d.m[p] + d.gy_eff;
    f.al = (0.0 + d.T[p]) / d.I[p];
    // constant a over N sub-cycles of dt = 1/N: after k of them the drift is
    // v k dt + a dt^2 k (k + 1) / 2, so |dx| <= |v| + |a| (N + 1) / (2N) <= |v| + |a|;
    // the margin covers the rounding of the updates
    f.ex = fabs(vx) + fabs(f.ax) + 1e-6;
    f.ey = fabs(vy) + fabs(f.ay) + 1e-6;
    return f;
}

// No wall within reach and no periodic crossing during the cycle.
__device__ __forceinline__ bool free_of_edges(const DemArgs &d, const FreeMotion &f, double px, double py,
                                              double rp) {
    return (d.bc_x != BC_WALL || (px - rp > f.ex && ((double)d.nx - px) - rp > f.ex)) &&
           (d.bc_y != BC_WALL || (py - rp > f.ey && ((double)d.ny - py) - rp > f.ey)) &&
           (d.bc_x != BC_PERIODIC || (px > f.ex && px < (double)d.nx - f.ex)) &&
           (d.bc_y != BC_PERIODIC || (py > f.ey && py < (double)d.ny - f.ey));
}

// The N_sub sub-cycles of a particle that touches nothing: the updates of integrate().
__device__ __forceinline__ void free_run(const DemArgs &d, const FreeMotion &f, double &px, double &py,
                                         double &vx, double &vy, double &w) {
    // the velocity increments a dt round to the same value every sub-cycle
    const double dvx = f.ax * d.dt, dvy = f.ay * d.dt, dw = f.al * d.dt;
    for (int s = 0; s < d.N_sub; ++s) {
        vx = vx + dvx;
        vy = vy + dvy;
        w = w + dw;
        px = px + vx * d.dt;
        py = py + vy * d.dt;
    }
}

// Candidate pair (p, q) cannot overlap within the cycle if both move freely: the gap
// exceeds the sum of their excursion bounds.
__device__ __forceinline__ bool pair_apart(const DemArgs &d, double px, double py, double rp, double exp_,
                                           double eyp, double qx, double qy, double rq, double exq,
                                           double eyq) {
    const double dx = min_image(qx - px, d.bc_x == BC_PERIODIC, d.nx);
    const double dy = min_image(qy - py, d.bc_y == BC_PERIODIC, d.ny);
    const double M = rp + rq + (exp_ + exq) + (eyp + eyq);
    return dx * dx + dy * dy > M * M;
}

// Candidate lists, one warp per particle: lanes 0-8 take the 3 x 3 bins around the
// particle's bin, then every lane tests candidates from the flattened bins (pairs within
// r_p + r_q + skin), the hits are ranked by id (the list is in ascending id order), and
// each kept pair carries its tangential spring and damping constant over from the
// previous list.
// append particle p to a per-cycle list of capacity np (the counts are reset by the bin scan
// of every rebuild); a full list is reported, not overrun
__device__ __forceinline__ void list_append(int *list, int *count, int np, int p, unsigned *err) {
    const int k = atomicAdd(count, 1);
    if (k < np) list[k] = p;
    else set_err(err, ERR_LIST);
}

constexpr int NB_WARPS = 4;
constexpr int NB_HITS = 64;   // hits a warp can hold before the overflow is reported

__global__ void __launch_bounds__(32 * NB_WARPS) k_dem_neighbours(const DemArgs d) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    __shared__ int s_hit[NB_WARPS][NB_HITS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = blockIdx.x * NB_WARPS + warp;
    if (p >= d.np) return;
    const unsigned FULLM = 0xffffffffu;
    const bool perx = d.bc_x == BC_PERIODIC, pery = d.bc_y == BC_PERIODIC;
    const double px = d.x[2 * p], py = d.x[2 * p + 1], rp = d.r[p];
    if (lane == 0) {
        d.x_start[2 * p] = px;
        d.x_start[2 * p + 1] = py;
    }
    const int b = d.pbin[p];
    const int bx = b % d.nbx, by = b / d.nbx;
    int bb = -1;
    if (lane < 9) {
        int ix = bx + lane % 3 - 1, iy = by + lane / 3 - 1;
        bool ok = true;
        if (ix < 0 || ix >= d.nbx) {
            if (perx) ix = (ix + d.nbx) % d.nbx;
            else ok = false;
        }
        if (iy < 0 || iy >= d.nby) {
            if (pery) iy = (iy + d.nby) % d.nby;
            else ok = false;
        }
        if (ok) bb = iy * d.nbx + ix;
    }
    const unsigned same = __match_any_sync(FULLM, bb);   // a bin met twice on a tiny periodic lattice
    if (bb >= 0 && __ffs(same) - 1 != lane) bb = -1;
    int beg = 0, cnt = 0;
    if (bb >= 0) {
        beg = d.bin_start[bb];
        cnt = d.bin_start[bb + 1] - beg;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULLM, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULLM, incl, 31);
    const int excl = incl - cnt;
    int nh = 0;
    for (int base = 0; base < total; base += 32) {
        const int k = base + lane;
        int q = -1;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int e = __shfl_sync(FULLM, excl, j), c = __shfl_sync(FULLM, cnt, j);
            const int g = __shfl_sync(FULLM, beg, j);
            if (k >= e && k < e + c) q = d.bin_ids[g + k - e];
        }
        bool hit = false;
        if (q >= 0 && q != p) {
            const double dx = min_image(d.x[2 * q] - px, perx, d.nx);
            const double dy = min_image(d.x[2 * q + 1] - py, pery, d.ny);
            const double R = rp + d.r[q] + d.skin;
            hit = dx * dx + dy * dy < R * R;
        }
        const unsigned hb = __ballot_sync(FULLM, hit);
        const int pos = nh + __popc(hb & ((1u << lane) - 1u));
        if (hit && pos < NB_HITS) s_hit[warp][pos] = q;
        nh += __popc(hb);
    }
    __syncwarp();
    if (nh > MAX_NBR) {
        if (lane == 0) set_err(d.err, ERR_NEIGHBOURS);
    }
    const int nkeep = min(nh, NB_HITS);
    const int n = min(nh, MAX_NBR);
    const int nold = d.nbr_cnt_old[p];
    for (int j = lane; j < nkeep; j += 32) {
        const int q = s_hit[warp][j];
        int rank = 0;
        for (int i = 0; i < nkeep; ++i) rank += s_hit[warp][i] < q;
        if (rank >= MAX_NBR) continue;
        double xi = 0.0, cn = -1.0;
        for (int k = 0; k < nold; ++k)
            if (d.nbr_id_old[p * MAX_NBR + k] == q) {
                xi = d.nbr_xi_old[p * MAX_NBR + k];
                cn = d.nbr_cn_old[p * MAX_NBR + k];
            }
        if (cn < 0.0) {   // a new candidate pair: its damping constant, once
            const double mq = d.m[q], mp = d.m[p];
            cn = damping_cn(d, mp * mq / (mp + mq));
        }
        d.nbr_id[p * MAX_NBR + rank] = q;
        d.nbr_xi[p * MAX_NBR + rank] = xi;
        d.nbr_cn[p * MAX_NBR + rank] = cn;
    }
    if (lane == 0) {
        d.nbr_cnt[p] = n;
        d.parent[p] = p;
        d.isz[p] = 0;
        d.ifill[p] = 0;
        d.iloud[p] = 0;
        if (n > 0) {
            const FreeMotion f = free_motion(d, p, d.v[2 * p], d.v[2 * p + 1]);
            d.exc[2 * p] = f.ex;
            d.exc[2 * p + 1] = f.ey;
            d.loud[p] = !free_of_edges(d, f, px, py, rp);
        }
        if (n == 0) list_append(d.free_ids, &d.counters[0], d.np, p, d.err);
        else list_append(d.coupled_ids, &d.counters[1], d.np, p, d.err);
    }
}

// Free particles, one per thread: blocks blk of nblk.
__device__ __forceinline__ void dem_free(const DemArgs &d, const int blk, const int nblk) {
    const int nfree = d.counters[0];
    for (int c = blk * blockDim.x + threadIdx.x; c < nfree; c += nblk * blockDim.x) {
        const int p = d.free_ids[c];
        double px = d.x[2 * p], py = d.x[2 * p + 1], vx = d.v[2 * p], vy = d.v[2 * p + 1], w = d.w[p];
        const double rp = d.r[p], mp = d.m[p];
        double xiw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) xiw[k] = d.wall_xi[4 * p + k];
        // candidate partners of a quiet island stay out of reach: their springs are released
        for (int j = 0, nn = d.nbr_cnt[p]; j < nn; ++j) d.nbr_xi[p * MAX_NBR + j] = 0.0;
        const FreeMotion f = free_motion(d, p, vx, vy);
        const Kick kick = free_kick(d, p);
        if (free_of_edges(d, f, px, py, rp)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) xiw[k] = 0.0;
            free_run(d, f, px, py, vx, vy, w);
        } else {
            const bool walls = d.bc_x == BC_WALL || d.bc_y == BC_WALL;
            for (int s = 0; s < d.N_sub; ++s) {
                bool touching = false;
                if (walls)
                    touching = (d.bc_x == BC_WALL && (px < rp || (double)d.nx - px < rp)) ||
                               (d.bc_y == BC_WALL && (py < rp || (double)d.ny - py < rp));
                if (touching) {
                    double Fcx = 0.0, Fcy = 0.0, Tc = 0.0;
                    wall_contacts(d, p, px, py, vx, vy, w, rp, mp, xiw, Fcx, Fcy, Tc);
                    integrate(d, p, Fcx, Fcy, Tc, px, py, vx, vy, w);
                } else {
                    // a released wall spring (wall_contacts would zero it)
#pragma unroll
                    for (int k = 0; k < 4; ++k) xiw[k] = 0.0;
                    coast(d, kick, px, py, vx, vy, w);
                }
            }
        }
        d.x[2 * p] = px;
        d.x[2 * p + 1] = py;
        d.v[2 * p] = vx;
        d.v[2 * p + 1] = vy;
        d.w[p] = w;
#pragma unroll
        for (int k = 0; k < 4; ++k) d.wall_xi[4 * p + k] = xiw[k];
    }
}

// One sub-cycle of particle p (Eqs. 7-11): contact forces from the candidate list in
// ascending id order, then the walls, then the leapfrog update.  nb(j, q, ...) yields
// the state of the j-th candidate q at the start of the sub-cycle.
template <typename NB>
__device__ __forceinline__ void particle_substep(const DemArgs &d, const int p, const Kick &kick, double &px,
                                                 double &py, double &vx, double &vy, double &w, NB &&nb) {
    const double rp = d.r[p], mp = d.m[p];
    double Fcx = 0.0, Fcy = 0.0, Tc = 0.0;
    bool touched = false;
    const int n = d.nbr_cnt[p];
    for (int j = 0; j < n; ++j) {
        double qx, qy, qvx, qvy, qw;
        nb(j, d.nbr_id[p * MAX_NBR + j], qx, qy, qvx, qvy, qw);
        double fx, fy, Ft;
        if (!pair_force(d, p, j, px, py, w, qx, qy, qvx, qvy, qw, vx, vy, fx, fy, Ft)) continue;
        Fcx += fx;
        Fcy += fy;
        Tc += rp * Ft;
        touched = true;
    }
    touched |= wall_contacts(d, p, px, py, vx, vy, w, rp, mp, &d.wall_xi[4 * p], Fcx, Fcy, Tc);
    if (touched) integrate(d, p, Fcx, Fcy, Tc, px, py, vx, vy, w);
    else coast(d, kick, px, py, vx, vy, w);
}

// Particles of islands larger than a warp: all blocks step them together, one bounded
// grid barrier per sub-cycle (cooperative launch), state exchanged through L2.
__global__ void k_dem_coupled(const DemArgs d) {
    const int ncpl = d.counters[3];
    const int nb_active = min((int)gridDim.x, (ncpl + (int)blockDim.x - 1) / (int)blockDim.x);
    if (ncpl == 0 || (int)blockIdx.x >= nb_active) return;
    const int stride = nb_active * blockDim.x;
    const int c0 = blockIdx.x * blockDim.x + threadIdx.x;
    const Kick k0 = c0 < ncpl ? free_kick(d, d.big_ids[c0]) : Kick{0.0, 0.0, 0.0};   // usually its only particle
    for (int s = 0; s < d.N_sub; ++s) {
        const double *xc = (s & 1) ? d.x1 : d.x;
        const double *vc = (s & 1) ? d.v1 : d.v;
        const double *wc = (s & 1) ? d.w1 : d.w;
        double *xn = (s & 1) ? d.x : d.x1;
        double *vn = (s & 1) ? d.v : d.v1;
        double *wn = (s & 1) ? d.w : d.w1;
        for (int c = c0; c < ncpl; c += stride) {
            const int p = d.big_ids[c];
            double px = __ldcg(&xc[2 * p]), py = __ldcg(&xc[2 * p + 1]);
            double vx = __ldcg(&vc[2 * p]), vy = __ldcg(&vc[2 * p + 1]), w = __ldcg(&wc[p]);
            particle_substep(d, p, c == c0 ? k0 : free_kick(d, p), px, py, vx, vy, w,
                             [&](int, int q, double &qx, double &qy, double &qvx, double &qvy, double &qw) {
                                 qx = __ldcg(&xc[2 * q]);
                                 qy = __ldcg(&xc[2 * q + 1]);
                                 qvx = __ldcg(&vc[2 * q]);
                                 qvy = __ldcg(&vc[2 * q + 1]);
                                 qw = __ldcg(&wc[q]);
                             });
            __stcg(&xn[2 * p], px);
            __stcg(&xn[2 * p + 1], py);
            __stcg(&vn[2 * p], vx);
            __stcg(&vn[2 * p + 1], vy);
            __stcg(&wn[p], w);
        }
        if (nb_active > 1) {
            if (!grid_barrier(d.barrier, (unsigned)nb_active, d.err)) return;
        } else {
            __syncthreads();
        }
    }
    if (d.N_sub & 1) {  // the last sub-cycle wrote the second buffer
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncpl; c += stride) {
            const int p = d.big_ids[c];
            d.x[2 * p] = __ldcg(&d.x1[2 * p]);
            d.x[2 * p + 1] = __ldcg(&d.x1[2 * p + 1]);
            d.v[2 * p] = __ldcg(&d.v1[2 * p]);
            d.v[2 * p + 1] = __ldcg(&d.v1[2 * p + 1]);
            d.w[p] = __ldcg(&d.w1[p]);
        }
    }
}

// ------------------------------------------------------------ islands
// Particles that can touch during a coupling cycle form the connected components
// ("islands") of the candidate graph; islands evolve independently.  Lock-free
// union-find: roots hook under the smaller index, finds halve paths.
__device__ __forceinline__ int uf_find(int *parent, int x) {
    volatile int *par = parent;
    for (;;) {
        const int p = par[x];
        if (p == x) return x;
        const int g = par[p];
        if (g == p) return p;
        par[x] = g;
        x = g;
    }
}

__global__ void k_uf_link(const DemArgs d) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    const int ncpl = d.counters[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncpl; c += gridDim.x * blockDim.x) {
        const int p = d.coupled_ids[c];
        const int n = d.nbr_cnt[p];
        const double px = d.x[2 * p], py = d.x[2 * p + 1], rp = d.r[p];
        const double exp_ = d.exc[2 * p], eyp = d.exc[2 * p + 1];
        int loud = d.loud[p];
        for (int j = 0; j < n; ++j) {
            const int q = d.nbr_id[p * MAX_NBR + j];
            loud |= !pair_apart(d, px, py, rp, exp_, eyp, d.x[2 * q], d.x[2 * q + 1], d.r[q], d.exc[2 * q],
                                d.exc[2 * q + 1]);
            if (q < p) continue;
            int a = p, b = q;
            for (;;) {
                a = uf_find(d.parent, a);
                b = uf_find(d.parent, b);
                if (a == b) break;
                if (a < b) { const int t = a; a = b; b = t; }
                if (atomicCAS(&d.parent[a], a, b) == a) break;
            }
        }
        d.loud[p] = loud;
    }
}

__global__ void k_uf_label(const DemArgs d) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    const int ncpl = d.counters[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncpl; c += gridDim.x * blockDim.x) {
        const int p = d.coupled_ids[c];
        const int r = uf_find(d.parent, p);
        d.label[p] = r;
        atomicAdd(&d.isz[r], 1);
        if (d.loud[p]) atomicOr(&d.iloud[r], 1);
    }
}

constexpr int ISL_SMALL = 4;           // islands up to this size share a warp, 8 to a warp
constexpr int ISL_WARPS = 4;
constexpr int ISL_PAIRS = 96;          // pairs evaluated a lane each, beyond that particle by particle

// Roots reserve a contiguous range of the member list for their island.
__global__ void k_island_alloc(const DemArgs d) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    const int ncpl = d.counters[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncpl; c += gridDim.x * blockDim.x) {
        const int p = d.coupled_ids[c];
        if (d.label[p] == p) d.istart[p] = atomicAdd(&d.counters[4], d.isz[p]);
    }
}

__global__ void k_island_fill(const DemArgs d) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    const int ncpl = d.counters[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncpl; c += gridDim.x * blockDim.x) {
        const int p = d.coupled_ids[c];
        const int r = d.label[p];
        if (!d.iloud[r]) {   // nothing in the island can touch within the cycle: free particles
            list_append(d.free_ids, &d.counters[0], d.np, p, d.err);
            continue;
        }
        const int size = d.isz[r];
        d.members[d.istart[r] + atomicAdd(&d.ifill[r], 1)] = p;
        if (size <= ISL_SMALL) {
            if (p == r) d.roots[atomicAdd(&d.counters[2], 1)] = r;
        } else if (size <= 32) {
            if (p == r) d.roots[d.np - 1 - atomicAdd(&d.counters[5], 1)] = r;   // filled from the end
        } else {
            d.big_ids[atomicAdd(&d.counters[3], 1)] = p;
        }
    }
}

// The islands a warp steps together: lane l holds particle id[l] (or -1), its candidates are
// members of its own island, and all N_sub sub-cycles run with the state in shared memory
// (double-buffered).  A sub-cycle is one round of pair forces, each candidate pair once with a
// lane of its own, then one round of particle updates, lane l summing its pairs in slot order
// -- the order of a sequential evaluation -- and adding the walls.  A pair's force on its
// second particle is the negated force on its first, to the bit: every operation of Eqs. 7-9
// is odd or even under the exchange of the two particles (n -> -n, t -> -t, the relative
// velocity -> its negative, sums and products of the two radii and masses unchanged) and IEEE
// rounding to nearest is symmetric, so the two tangential springs stay equal as well.  Every
// FP64 instruction costs a warp the same whatever its active lanes, so a sub-cycle's cost is
// the instructions of its two rounds.
constexpr int SMALL_PER_WARP = 32 / ISL_SMALL;

struct WarpIslands {
    double st[2][5][32];                 // x, y, vx, vy, w
    double f[3][ISL_PAIRS];              // fx, fy, Ft on the pair's first particle
    double xi[ISL_PAIRS];                // the pair's tangential spring
    int id[32];
    unsigned char nn[32];                // candidates of lane l
    unsigned char nl[32][MAX_NBR];       // lane of candidate j
    unsigned char slot[32][MAX_NBR];     // pair of candidate j, bit 7 set on the pair's second particle
    unsigned char pi[ISL_PAIRS], pj[ISL_PAIRS], pr[ISL_PAIRS], on[ISL_PAIRS];
};

// p: this lane's particle or -1; [g0, g0 + gn): the lanes of its island.
__device__ __forceinline__ void warp_islands(const DemArgs &d, WarpIslands &w, const int p, const int g0,
                                             const int gn) {
    const int lane = threadIdx.x & 31;
    const bool act = p >= 0;
    const int nn = act ? d.nbr_cnt[p] : 0;
    w.id[lane] = p;
    w.nn[lane] = (unsigned char)nn;
    __syncwarp();
    int own = 0;   // pairs this lane leads: its candidates on higher lanes
    if (act) {
        for (int j = 0; j < nn; ++j) {
            const int q = d.nbr_id[p * MAX_NBR + j];
            int l = g0;
            while (l < g0 + gn - 1 && w.id[l] != q) ++l;   // q is in the same island
            w.nl[lane][j] = (unsigned char)l;
            w.slot[lane][j] = 255;   // set below by the pair's leading lane
            own += l > lane;
        }
        w.st[0][0][lane] = d.x[2 * p];
        w.st[0][1][lane] = d.x[2 * p + 1];
        w.st[0][2][lane] = d.v[2 * p];
        w.st[0][3][lane] = d.v[2 * p + 1];
        w.st[0][4][lane] = d.w[p];
    }
    int off = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += t;
    }
    const int npairs = __shfl_sync(0xffffffffu, off, 31);
    off -= own;
    __syncwarp();
    if (act && npairs <= ISL_PAIRS) {
        int k = off;
        for (int j = 0; j < nn; ++j) {
            const int l = w.nl[lane][j];
            if (l <= lane) continue;
            int jr = 0;
            while (jr < w.nn[l] && w.nl[l][jr] != lane) ++jr;
            w.pi[k] = (unsigned char)lane;
            w.pj[k] = (unsigned char)j;
            w.pr[k] = (unsigned char)(jr < w.nn[l] ? jr : 0);
            w.slot[lane][j] = (unsigned char)k;
            if (jr < w.nn[l]) w.slot[l][jr] = (unsigned char)(k | 128);
            w.xi[k] = d.nbr_xi[p * MAX_NBR + j];   // equal to the partner's spring of the pair
            ++k;
        }
    }
    __syncwarp();
    // pairs evaluated a lane each only when every candidate slot of the warp names a pair (the
    // candidate lists are symmetric and stay within the island), else particle by particle
    bool ok = npairs <= ISL_PAIRS;
    for (int j = 0; ok && j < nn; ++j) ok = (w.slot[lane][j] & 127) < npairs && w.nl[lane][j] != lane;
    const bool pairwise = __all_sync(0xffffffffu, ok);
    const Kick kick = act ? free_kick(d, p) : Kick{0.0, 0.0, 0.0};
    const double rp = act ? d.r[p] : 0.0, mp = act ? d.m[p] : 0.0;
    double xiw[4];   // wall springs, in registers on the pair-parallel path
#pragma unroll
    for (int q = 0; q < 4; ++q) xiw[q] = act ? d.wall_xi[4 * p + q] : 0.0;
    __syncwarp();
    for (int s = 0; s < d.N_sub; ++s) {
        const int cur = s & 1;
        const double(*st)[32] = w.st[cur];
        if (pairwise) {
            for (int k = lane; k < npairs; k += 32) {
                const int i = w.pi[k], j = w.pj[k], l = w.nl[i][j];
                double xi = w.xi[k];
                double fx = 0.0, fy = 0.0, Ft = 0.0;
                w.on[k] = pair_force_xi(d, w.id[i], j, w.id[l], xi, st[0][i], st[1][i], st[4][i], st[0][l],
                                        st[1][l], st[2][l], st[3][l], st[4][l], st[2][i], st[3][i], fx, fy, Ft);
                w.xi[k] = xi;
                w.f[0][k] = fx;
                w.f[1][k] = fy;
                w.f[2][k] = Ft;
            }
            __syncwarp();
        }
        if (act) {
            double px = st[0][lane], py = st[1][lane], vx = st[2][lane], vy = st[3][lane], om = st[4][lane];
            if (pairwise) {
                double Fcx = 0.0, Fcy = 0.0, Tc = 0.0;
                bool touched = false;
                for (int j = 0; j < nn; ++j) {
                    const int e = w.slot[lane][j], k = e & 127;
                    if (!w.on[k]) continue;
                    if (e & 128) {
                        Fcx += -w.f[0][k];
                        Fcy += -w.f[1][k];
                    } else {
                        Fcx += w.f[0][k];
                        Fcy += w.f[1][k];
                    }
                    Tc += rp * w.f[2][k];
                    touched = true;
                }
                touched |= wall_contacts(d, p, px, py, vx, vy, om, rp, mp, xiw, Fcx, Fcy, Tc);
                if (touched) integrate(d, p, Fcx, Fcy, Tc, px, py, vx, vy, om);
                else coast(d, kick, px, py, vx, vy, om);
            } else {
                particle_substep(d, p, kick, px, py, vx, vy, om,
                                 [&](int j, int, double &qx, double &qy, double &qvx, double &qvy, double &qw) {
                                     const int l = w.nl[lane][j];
                                     qx = st[0][l];
                                     qy = st[1][l];
                                     qvx = st[2][l];
                                     qvy = st[3][l];
                                     qw = st[4][l];
                                 });
            }
            w.st[cur ^ 1][0][lane] = px;
            w.st[cur ^ 1][1][lane] = py;
            w.st[cur ^ 1][2][lane] = vx;
            w.st[cur ^ 1][3][lane] = vy;
            w.st[cur ^ 1][4][lane] = om;
        }
        __syncwarp();
    }
    if (act) {
        const int fin = d.N_sub & 1;
        d.x[2 * p] = w.st[fin][0][lane];
        d.x[2 * p + 1] = w.st[fin][1][lane];
        d.v[2 * p] = w.st[fin][2][lane];
        d.v[2 * p + 1] = w.st[fin][3][lane];
        d.w[p] = w.st[fin][4][lane];
        if (pairwise) {   // the springs back into both particles' lists
#pragma unroll
            for (int q = 0; q < 4; ++q) d.wall_xi[4 * p + q] = xiw[q];
            for (int j = 0; j < nn; ++j) {
                const int e = w.slot[lane][j];
                d.nbr_xi[p * MAX_NBR + j] = w.xi[e & 127];
            }
        }
    }
    __syncwarp();
}

// Islands of up to ISL_SMALL particles, SMALL_PER_WARP to a warp in lane groups of
// ISL_SMALL: block blk of the role.
__device__ __forceinline__ void dem_small_islands(const DemArgs &d, const int blk, WarpIslands (&sm)[ISL_WARPS]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / ISL_SMALL, k = lane % ISL_SMALL;
    const int nisl = d.counters[2];
    const int i = (blk * ISL_WARPS + warp) * SMALL_PER_WARP + grp;
    if ((blk * ISL_WARPS + warp) * SMALL_PER_WARP >= nisl) return;   // whole warp idle
    int p = -1, n = 0;
    if (i < nisl) {
        const int r = d.roots[i];
        n = d.isz[r];
        if (k < n) p = d.members[d.istart[r] + k];
    }
    warp_islands(d, sm[warp], p, grp * ISL_SMALL, n);
}

// Islands of five to 32 particles, one per warp: block blk of nblk.
__device__ __forceinline__ void dem_islands(const DemArgs &d, const int blk, const int nblk,
                                            WarpIslands (&sm)[ISL_WARPS]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nisl = d.counters[5];
    for (int i = blk * ISL_WARPS + warp; i < nisl; i += nblk * ISL_WARPS) {
        const int r = d.roots[d.np - 1 - i];
        const int n = d.isz[r];
        warp_islands(d, sm[warp], lane < n ? d.members[d.istart[r] + lane] : -1, 0, n);
    }
}

// The particles of one coupling cycle that need no grid barrier -- free particles, islands
// of up to four, islands of five to 32 -- in one launch: the roles take consecutive block
// ranges in that order and run side by side (the three sets of particles are disjoint), so
// an island's chain of N_sub sub-cycles, bound by the latency of its FP64 instructions,
// overlaps the free particles' FP64 throughput and the other islands' chains.
constexpr int LOCAL_THREADS = 32 * ISL_WARPS;

__global__ void __launch_bounds__(LOCAL_THREADS) k_dem_local(const DemArgs d, int nb_islands, int nb_small) {
    cudaGridDependencySynchronize();   // launched as a dependent of the kernel before it
    __shared__ WarpIslands sm[ISL_WARPS];
    const int b = blockIdx.x, nb_free = (int)gridDim.x - nb_islands - nb_small;
    if (b < nb_free) dem_free(d, b, nb_free);
    else if (b < nb_free + nb_small) dem_small_islands(d, b - nb_free, sm);
    else dem_islands(d, b - nb_free - nb_small, nb_islands, sm);
}

__global__ void k_contacts(const double *__restrict__ x, const double *__restrict__ r, int np, int nx,
                           int ny, int bc_x, int bc_y, const int *__restrict__ bin_start,
                           const int *__restrict__ bin_ids, const int *__restrict__ pbin, int nbx,
                           int nby, int reach, int *pair_cnt, int *pairs, int max_per) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= np) return;
    const bool perx = bc_x == BC_PERIODIC, pery = bc_y == BC_PERIODIC;
    const int b = pbin[a];
    const int bx = b % nbx, by = b / nbx;
    int n = 0;
    const int wx = min(2 * reach + 1, nbx), wy = min(2 * reach + 1, nby);
    for (int oy = 0; oy < wy; ++oy)
        for (int ox = 0; ox < wx; ++ox) {
            int ix = bx - reach + ox, iy = by - reach + oy;
            if (perx) ix = ((ix % nbx) + nbx) % nbx;
            else if (ix < 0 || ix >= nbx) continue;
            if (pery) iy = ((iy % nby) + nby) % nby;
            else if (iy < 0 || iy >= nby) continue;
            const int bb = iy * nbx + ix;
            for (int k = bin_start[bb]; k < bin_start[bb + 1]; ++k) {
                const int q = bin_ids[k];
                if (q <= a) continue;
                const double dx = min_image(x[2 * q] - x[2 * a], perx, nx);
                const double dy = min_image(x[2 * q + 1] - x[2 * a + 1], pery, ny);
                const double R = r[a] + r[q];
                if (dx * dx + dy * dy < R * R) {
                    if (n < max_per) pairs[a * max_per + n] = q;
                    ++n;
                }
            }
        }
    pair_cnt[a] = n;
}

// ------------------------------------------------------------ launchers
static inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

cudaError_t launch_particle_table(const double *x, const double *r, const double *x_start, int np,
                                  int nx, int ny, int bc_x, int bc_y, double skin_half, int nbx,
                                  int nby, int *bin_count, int *pbin, PRec *prec, const double *v,
                                  const double *w, double *F, double *T, unsigned *err,
                                  cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    return launch_dependent(k_particle_table, blocks_for(np, 128), 128, 0, s, true, x, r, x_start, np, nx, ny, bc_x,
                            bc_y, skin_half, nbx, nby, bin_count, pbin, prec, v, w, F, T, err);
}

cudaError_t launch_bin_scan(int *bin_count, int *bin_fill, int *bin_start, int nbins, int *bsum,
                            int *dem_counters, cudaStream_t s) {
    const int nb = (nbins + SCAN_BINS - 1) / SCAN_BINS;
    cudaError_t e = launch_dependent(k_bin_scan_local, nb, 256, 0, s, true, bin_count, bin_start, nbins, bsum,
                                     dem_counters);
    if (e != cudaSuccess) return e;
    return launch_dependent(k_bin_scan_add, nb, 256, 0, s, true, bin_fill, bin_start, nbins, (const int *)bsum);
}

cudaError_t launch_bin_fill(const int *pbin, int np, int *bin_fill, const int *bin_start,
                            int *bin_ids, cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    return launch_dependent(k_bin_fill, blocks_for(np, 128), 128, 0, s, true, pbin, np, bin_fill, bin_start, bin_ids);
}

cudaError_t launch_dem_neighbours(const DemArgs &d, cudaStream_t s) {
    if (d.np == 0) return cudaSuccess;
    return launch_dependent(k_dem_neighbours, blocks_for(d.np, NB_WARPS), 32 * NB_WARPS, 0, s, true, d);
}


static int g_coupled_blocks = 0;

int dem_coupled_blocks() {
    if (g_coupled_blocks == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_coupled_blocks = sms > 0 ? sms : 1;
    }
    return g_coupled_blocks;
}

cudaError_t launch_dem_coupled(const DemArgs &d, int nblocks, cudaStream_t s) {
    if (d.np == 0) return cudaSuccess;
    DemArgs copy = d;
    void *args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void *)k_dem_coupled, dim3(nblocks), dim3(32), args, 0, s);
}

cudaError_t launch_dem_islands_setup(const DemArgs &d, cudaStream_t s) {
    if (d.np == 0) return cudaSuccess;
    const int g = blocks_for(d.np, 128);
    cudaError_t e = cudaSuccess;
    for (auto k : {k_uf_link, k_uf_label, k_island_alloc, k_island_fill})
        if (e == cudaSuccess) e = launch_dependent(k, g, 128, 0, s, true, d);
    return e;
}

cudaError_t launch_dem_local(const DemArgs &d, cudaStream_t s) {
    if (d.np == 0) return cudaSuccess;
    // enough warps for every island at once: at most np/5 islands of five or more, at most
    // np/2 of two or more
    const int nb_islands = blocks_for(d.np / 5 + 1, ISL_WARPS);
    const int nb_small = blocks_for(blocks_for(d.np / 2 + 1, SMALL_PER_WARP), ISL_WARPS);
    const int nb_free = blocks_for(d.np, LOCAL_THREADS);
    return launch_dependent(k_dem_local, nb_islands + nb_small + nb_free, LOCAL_THREADS, 0, s, true, d, nb_islands,
                            nb_small);
}

// Host round trips through pinned host memory that the device can address (NVLink-C2C or PCIe
// mapped pages): one launch moves the particles' kinematics in, one the forces and state out,
// instead of a DMA copy per array.
__global__ void k_kinematics_in(const double *__restrict__ hx, const double *__restrict__ hv,
                                const double *__restrict__ hw, double *x, double *v, double *w, int np) {
    cudaGridDependencySynchronize();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    x[2 * p] = hx[2 * p];
    x[2 * p + 1] = hx[2 * p + 1];
    v[2 * p] = hv[2 * p];
    v[2 * p + 1] = hv[2 * p + 1];
    w[p] = hw[p];
}

__global__ void k_state_out(const double *__restrict__ F, const double *__restrict__ T, const double *__restrict__ x,
                            const double *__restrict__ v, const double *__restrict__ w, double *hF, double *hT,
                            double *hx, double *hv, double *hw, int np) {
    cudaGridDependencySynchronize();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    if (hF) {
        hF[2 * p] = F[2 * p];
        hF[2 * p + 1] = F[2 * p + 1];
    }
    if (hT) hT[p] = T[p];
    if (hx) {
        hx[2 * p] = x[2 * p];
        hx[2 * p + 1] = x[2 * p + 1];
    }
    if (hv) {
        hv[2 * p] = v[2 * p];
        hv[2 * p + 1] = v[2 * p + 1];
    }
    if (hw) hw[p] = w[p];
}

cudaError_t launch_kinematics_in(const double *hx, const double *hv, const double *hw, double *x, double *v, double *w,
                                 int np, cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    return launch_dependent(k_kinematics_in, blocks_for(np, 128), 128, 0, s, true, hx, hv, hw, x, v, w, np);
}

cudaError_t launch_state_out(const double *F, const double *T, const double *x, const double *v, const double *w,
                             double *hF, double *hT, double *hx, double *hv, double *hw, int np, cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    return launch_dependent(k_state_out, blocks_for(np, 128), 128, 0, s, true, F, T, x, v, w, hF, hT, hx, hv, hw, np);
}

cudaError_t launch_contacts(const double *x, const double *r, int np, int nx, int ny, int bc_x,
                            int bc_y, const int *bin_start, const int *bin_ids, const int *pbin,
                            int nbx, int nby, int reach, int *pair_cnt, int *pairs, int max_per,
                            cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    k_contacts<<<blocks_for(np, 128), 128, 0, s>>>(x, r, np, nx, ny, bc_x, bc_y, bin_start, bin_ids,
                                                   pbin, nbx, nby, reach, pair_cnt, pairs, max_per);
    return cudaGetLastError();
}

}  // namespace imb
