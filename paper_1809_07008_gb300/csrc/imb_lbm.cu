// imb_lbm.cu -- lattice kernels of the GB300 IMB-LBM-DEM library.
//
//   k_stream_collide  one fused pass per time step: D2Q9 pull streaming (Eq. 1 LHS)
//                     with periodic / halfway bounce-back / inlet-outlet boundaries,
//                     moments (Eqs. 3-4), BGK with Smagorinsky tau_eff (Eqs. 1-2,
//                     Sec. 3.3), solid ratio per cell (Sec. 2.3), weighting B (Eq. 14),
//                     solid operator (Eq. 12) and blend (Eq. 13), and the per-particle
//                     force and torque (Eqs. 15-16) reduced warp -> block -> FP64
//                     atomics.  Populations are stored as f_i - w_i (SoA planes).
//   k_gather          the same pull without collision: f(x, t) and the fields.
//   k_cell_map        the particle-to-lattice bookkeeping of the same tiles.
//   k_init            f* = f^eq(rho0, u0) in both buffers.
//
// A block owns one 32 x 32 tile, which is also one bin of the particle grid, so
// the particles that can reach the tile sit in the 3 x 3 surrounding bins.
#include <type_traits>

#include "imb_device.cuh"
#include "imb_kernels.h"

namespace imb {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLOCK = 256;            // 8 warps; warp w handles rows w, w+8, w+16, w+24
constexpr int WARPS = BLOCK / 32;

// ---------------------------------------------------------------- pulls
template <typename S>
__device__ __forceinline__ void pull_generic(const S *__restrict__ fin, const LatticeArgs &a, int x,
                                             int y, float (&d)[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        int xs = x - cx_of(q), ys = y - cy_of(q);
        const size_t self_opp = (size_t)opp_of(q) * a.plane + (size_t)y * a.pitch + x;
        if (ys < 0 || ys >= a.ny) {
            if (a.bc_y == BC_PERIODIC) {
                ys = ys < 0 ? ys + a.ny : ys - a.ny;
            } else {  // halfway bounce-back: what left (x,y) towards the wall comes back
                d[q] = Store<S>::ld(fin + self_opp);
                continue;
            }
        }
        if (xs < 0 || xs >= a.nx) {
            if (a.bc_x == BC_PERIODIC) {
                xs = xs < 0 ? xs + a.nx : xs - a.nx;
            } else if (a.bc_x == BC_WALL) {
                d[q] = Store<S>::ld(fin + self_opp);
                continue;
            } else {  // inlet / outlet column, rebuilt by pull_cell
                d[q] = 0.0f;
                continue;
            }
        }
        d[q] = Store<S>::ld(fin + (size_t)q * a.plane + (size_t)ys * a.pitch + xs);
    }
}

// shifted equilibrium f^eq_q - w_q = w_q (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2))   (Eq. 2)
__device__ __forceinline__ void equilibrium_shifted(float drho, float rho, float ux, float uy,
                                                    float (&d)[9]) {
    const float usq = ux * ux + uy * uy;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float cu = (float)cx_of(q) * ux + (float)cy_of(q) * uy;
        d[q] = w_of(q) * (drho + rho * (cu * (3.0f + 4.5f * cu) - 1.5f * usq));
    }
}

template <typename S>
__device__ __forceinline__ void pull_cell(const S *__restrict__ fin, const LatticeArgs &a, int x,
                                          int y, float (&d)[9]) {
    if (a.bc_x == BC_INLET_OUTLET && (x == 0 || x == a.nx - 1)) {
        // inlet: f^eq(rho of column 1, u_in); outlet: copy of column nx-2 (zero gradient)
        pull_generic(fin, a, x == 0 ? 1 : a.nx - 2, y, d);
        if (x == 0) {
            float drho = 0.0f;
#pragma unroll
            for (int q = 0; q < 9; ++q) drho += d[q];
            equilibrium_shifted(drho, 1.0f + drho, a.u_in_x, a.u_in_y, d);
        }
        return;
    }
    pull_generic(fin, a, x, y, d);
}

template <typename S>
__device__ __forceinline__ void pull_interior(const S *__restrict__ fin, const LatticeArgs &a, int x,
                                              int y, float (&d)[9]) {
    const S *base = fin + (size_t)y * a.pitch + x;
#pragma unroll
    for (int q = 0; q < 9; ++q)
        d[q] = Store<S>::ld(base + (size_t)q * a.plane - (ptrdiff_t)cy_of(q) * a.pitch - cx_of(q));
}

// ------------------------------------------------------ tile prologue
struct TileShared {
    PRec p[TILE_CAND];
    int id[TILE_CAND];
    unsigned rowbits[TILE_CAND];
    unsigned rowmask[TILE];
    int bexcl[9], bstart[9], bcnt[9];
    int nc;
};

// 1D distance from a particle centre (tile centre minus centre cell = dc, fractional
// offset frac) to the span of a tile, the minimum over the periodic images.
__device__ __forceinline__ float tile_gap1(int dc, float frac) {
    float lo = (float)(dc - TILE / 2) - frac, hi = lo + (float)TILE;
    return lo > 0.0f ? lo : (hi < 0.0f ? -hi : 0.0f);
}
__device__ __forceinline__ float tile_gap(int dc, float frac, int L, bool periodic) {
    float g = tile_gap1(dc, frac);
    if (periodic) g = fminf(g, fminf(tile_gap1(dc + L, frac), tile_gap1(dc - L, frac)));
    return g;
}

// Collect (ascending id) the particles whose disk can reach into tile (bx, by), and
// per tile row a bit mask of the candidates whose y-extent meets that row.
__device__ void tile_candidates(const LatticeArgs &a, int bx, int by, TileShared &sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool perx = a.bc_x == BC_PERIODIC, pery = a.bc_y == BC_PERIODIC;
    if (warp == 0) {
        int bidx = -1;
        if (lane < 9) {
            int ix = bx + (lane % 3) - 1, iy = by + (lane / 3) - 1;
            bool ok = true;
            if (ix < 0 || ix >= a.nbx) {
                if (perx) ix = (ix + a.nbx) % a.nbx; else ok = false;
            }
            if (iy < 0 || iy >= a.nby) {
                if (pery) iy = (iy + a.nby) % a.nby; else ok = false;
            }
            if (ok) bidx = iy * a.nbx + ix;
        }
        for (int j = 0; j < 9; ++j) {  // a bin reached twice through a periodic wrap counts once
            int bj = __shfl_sync(FULL, bidx, j);
            if (j < lane && bj == bidx) bidx = -1;
        }
        int start = 0, cnt = 0;
        if (bidx >= 0) {
            start = a.bin_start[bidx];
            cnt = a.bin_start[bidx + 1] - start;
        }
        int pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULL, pre, o);
            if (lane >= o) pre += t;
        }
        const int total = __shfl_sync(FULL, pre, 31);
        if (lane < 9) {
            sh.bexcl[lane] = pre - cnt;
            sh.bstart[lane] = start;
            sh.bcnt[lane] = cnt;
        }
        __syncwarp();
        const int xc = bx * TILE + TILE / 2, yc = by * TILE + TILE / 2;
        int nc = 0;
        for (int base = 0; base < total; base += 32) {
            const int k = base + lane;
            bool take = false;
            int pid = -1;
            PRec P;
            if (k < total) {
                int j = 0;
                while (j < 8 && k >= sh.bexcl[j] + sh.bcnt[j]) ++j;
                pid = a.bin_ids[sh.bstart[j] + k - sh.bexcl[j]];
                P = a.prec[pid];
                // nearest point of the whole tile within r (+ margin), over the periodic
                // images: a necessary condition for the disk to reach any of its cells
                const float gx = tile_gap(wrap_rel(xc - P.ci, a.nx, perx), P.fx, a.nx, perx);
                const float gy = tile_gap(wrap_rel(yc - P.cj, a.ny, pery), P.fy, a.ny, pery);
                const float rr = P.r + 0.5f;
                take = gx * gx + gy * gy < rr * rr;
            }
            unsigned bal = __ballot_sync(FULL, take);
            int pos = nc + __popc(bal & ((1u << lane) - 1u));
            if (take) {
                if (pos < TILE_CAND) {
                    sh.id[pos] = pid;
                    sh.p[pos] = P;
                } else {
                    set_err(a.err, ERR_TILE_LIST);
                }
            }
            nc += __popc(bal);
        }
        nc = nc < TILE_CAND ? nc : TILE_CAND;
        __syncwarp();
        // order the candidates by particle id (deterministic whatever the bin order)
        int myid = lane < nc ? sh.id[lane] : 0x7fffffff;
        PRec myp;
        if (lane < nc) myp = sh.p[lane];
        int rank = 0;
        for (int t = 0; t < nc; ++t) rank += sh.id[t] < myid;
        __syncwarp();
        if (lane < nc) {
            sh.id[rank] = myid;
            sh.p[rank] = myp;
        }
        if (lane == 0) sh.nc = nc;
    }
    __syncthreads();
    const int nc = sh.nc;
    const int y = by * TILE + lane;
    for (int s = warp; s < nc; s += WARPS) {
        const PRec P = sh.p[s];
        bool rel = false;
        if (y < a.ny) {
            // necessary for coverage of any cell of row y: dy_near^2 < r^2 (same rounding as covers)
            int dk = wrap_rel(y - P.cj, a.ny, pery);
            float loy = __fsub_rn((float)dk, P.fy);
            float hiy = __fadd_rn(loy, 1.0f);
            float dy = loy > 0.0f ? loy : (hiy < 0.0f ? hiy : 0.0f);
            rel = __fmul_rn(dy, dy) < __fmul_rn(P.r, P.r);
        }
        unsigned bits = __ballot_sync(FULL, rel);
        if (lane == 0) sh.rowbits[s] = bits;
    }
    __syncthreads();
    if (threadIdx.x < TILE) {
        unsigned m = 0;
        for (int s = 0; s < nc; ++s) m |= ((sh.rowbits[s] >> threadIdx.x) & 1u) << s;
        sh.rowmask[threadIdx.x] = m;
    }
    __syncthreads();
}

// ------------------------------------------------- fused stream-collide
template <typename S>
__global__ void __launch_bounds__(BLOCK)
k_stream_collide(const S *__restrict__ fin, S *__restrict__ fout, const LatticeArgs a) {
    __shared__ TileShared sh;
    __shared__ float s_part[WARPS][TILE_CAND][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = blockIdx.x, by = blockIdx.y;
    const int x0 = bx * TILE, y0 = by * TILE;
    int nc = 0;
    if (a.np > 0) {
        tile_candidates(a, bx, by, sh);
        nc = sh.nc;
        for (int i = threadIdx.x; i < WARPS * TILE_CAND * 3; i += BLOCK) (&s_part[0][0][0])[i] = 0.0f;
        __syncthreads();
    }
    const bool perx = a.bc_x == BC_PERIODIC, pery = a.bc_y == BC_PERIODIC;
    const bool interior = x0 >= 1 && x0 + TILE <= a.nx - 1 && y0 >= 1 && y0 + TILE <= a.ny - 1;
    const bool forced = a.Fx != 0.0f || a.Fy != 0.0f;
    const bool smag = a.smag_coef > 0.0f;
    const int x = x0 + lane;
    const bool xin = x < a.nx;
    bool unstable = false;

    for (int rr = 0; rr < TILE / WARPS; ++rr) {
        const int y = y0 + warp + WARPS * rr;
        if (y >= a.ny) break;
        float d[9];
        if (xin) {
            if (interior) pull_interior(fin, a, x, y, d);
            else pull_cell(fin, a, x, y, d);
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) d[q] = 0.0f;
        }
        // ---- moments (Eqs. 3-4, Guo half-force shift)
        float drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        const float rho = 1.0f + drho;
        float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
        if (forced) {
            jx = fmaf(0.5f, a.Fx, jx);
            jy = fmaf(0.5f, a.Fy, jy);
        }
        const float inv = 1.0f / rho;
        const float ux = jx * inv, uy = jy * inv;
        const float usq = ux * ux + uy * uy;
        if (xin && !(usq < 0.09f)) unstable = true;       // Mach guard, also catches NaN
        // ---- non-equilibrium parts (Eq. 2)
        float n[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float cu = (float)cx_of(q) * ux + (float)cy_of(q) * uy;
            n[q] = d[q] - w_of(q) * (drho + rho * (cu * (3.0f + 4.5f * cu) - 1.5f * usq));
        }
        // ---- Smagorinsky effective relaxation time (Hou et al. 1996 closure)
        float te = a.tau;
        if (smag) {
            const float pxx = (n[1] + n[3]) + (n[5] + n[6]) + (n[7] + n[8]);
            const float pyy = (n[2] + n[4]) + (n[5] + n[6]) + (n[7] + n[8]);
            const float pxy = (n[5] - n[6]) + (n[7] - n[8]);
            const float Q = pxx * pxx + pyy * pyy + 2.0f * pxy * pxy;
            te = 0.5f * (a.tau + sqrtf(a.tau * a.tau + a.smag_coef * sqrtf(Q) * inv));
        }
        const float omega = 1.0f / te;
        // ---- immersed moving boundary: solid ratio, B, solid velocity moments
        float B = 0.0f;
        float m1x = 0.0f, m1y = 0.0f, m2xx = 0.0f, m2xy = 0.0f, m2yy = 0.0f;
        int c0 = -1, c1 = -1, c2 = -1, c3 = -1;
        float fx0 = 0.f, fy0 = 0.f, t0 = 0.f, fx1 = 0.f, fy1 = 0.f, t1 = 0.f;
        float fx2 = 0.f, fy2 = 0.f, t2 = 0.f, fx3 = 0.f, fy3 = 0.f, t3 = 0.f;
        const unsigned mask = nc ? sh.rowmask[y - y0] : 0u;
        if (mask) {
            int ns = 0;
            float esum = 0.0f, e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
            unsigned m = mask;
            while (m) {
                const int s = __ffs(m) - 1;
                m &= m - 1u;
                if (!xin) continue;
                const PRec P = sh.p[s];
                const int di = wrap_rel(x - P.ci, a.nx, perx), dk = wrap_rel(y - P.cj, a.ny, pery);
                const float lox = __fsub_rn((float)di, P.fx), loy = __fsub_rn((float)dk, P.fy);
                if (!covers(lox, loy, P.r)) continue;
                const float e = a.eps_mode == EPS_EXACT ? cell_disk_area(lox, loy, P.r)
                                                        : cell_subcell_ratio(lox, loy, P.r, a.n_sub);
                if (ns == 0) { c0 = s; e0 = e; }
                else if (ns == 1) { c1 = s; e1 = e; }
                else if (ns == 2) { c2 = s; e2 = e; }
                else if (ns == 3) { c3 = s; e3 = e; }
                else { set_err(a.err, ERR_CELL_SLOTS); continue; }
                ++ns;
                esum += e;
            }
            if (ns > 0 && esum > 0.0f) {
                const float eps = fminf(esum, 1.0f);
                const float tm = te - 0.5f;
                B = eps * tm / ((1.0f - eps) + tm);                 // Eq. 14
                const float Bs = B / esum;
#pragma unroll
                for (int k = 0; k < MAX_SLOTS; ++k) {
                    const int ck = k == 0 ? c0 : (k == 1 ? c1 : (k == 2 ? c2 : c3));
                    const float ek = k == 0 ? e0 : (k == 1 ? e1 : (k == 2 ? e2 : e3));
                    if (ck < 0) continue;
                    const PRec P = sh.p[ck];
                    const int di = wrap_rel(x - P.ci, a.nx, perx), dk = wrap_rel(y - P.cj, a.ny, pery);
                    const float rx = __fsub_rn((float)di, P.fx) + 0.5f;   // node minus centre
                    const float ry = __fsub_rn((float)dk, P.fy) + 0.5f;
                    const float usx = P.vx - P.w * ry, usy = P.vy + P.w * rx; // u_s = v + w z x r
                    const float Bp = Bs * ek;
                    m1x += Bp * usx;
                    m1y += Bp * usy;
                    m2xx += Bp * usx * usx;
                    m2xy += Bp * usx * usy;
                    m2yy += Bp * usy * usy;
                    // Eq. 15 per cell: -Bp sum_i Omega^s_i c_i = Bp (rho u - rho u_s - F)
                    const float fxk = Bp * (jx - rho * usx - a.Fx);
                    const float fyk = Bp * (jy - rho * usy - a.Fy);
                    const float tk = rx * fyk - ry * fxk;              // Eq. 16 (z)
                    if (k == 0) { fx0 = fxk; fy0 = fyk; t0 = tk; }
                    else if (k == 1) { fx1 = fxk; fy1 = fyk; t1 = tk; }
                    else if (k == 2) { fx2 = fxk; fy2 = fyk; t2 = tk; }
                    else { fx3 = fxk; fy3 = fyk; t3 = tk; }
                }
            }
        }
        // ---- collision and store (Eq. 13): fluid part weighted 1 - B, solid part by B
        if (xin) {
            const float fl = 1.0f - B;
            const float sf = 1.0f - 0.5f * omega;
            S *outp = fout + (size_t)y * a.pitch + x;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float cxq = (float)cx_of(q), cyq = (float)cy_of(q);
                float upd = -omega * n[q];
                if (forced) {  // Guo forcing term
                    const float cu = cxq * ux + cyq * uy;
                    const float S_q = w_of(q) * (3.0f * ((cxq - ux) * a.Fx + (cyq - uy) * a.Fy) +
                                                 9.0f * cu * (cxq * a.Fx + cyq * a.Fy));
                    upd = fmaf(sf, S_q, upd);
                }
                upd *= fl;
                if (B > 0.0f) {
                    // Eq. 12 summed over the covering particles:
                    // sum_p B_p Omega^s_p = B (n_{-q} - n_q) + sum_p B_p (f^eq_q(u_s,p) - f^eq_q(u))
                    const float cu = cxq * ux + cyq * uy;
                    const float cm1 = cxq * m1x + cyq * m1y;
                    const float cm2c = cxq * cxq * m2xx + 2.0f * cxq * cyq * m2xy + cyq * cyq * m2yy;
                    const float dfeq = rho * w_of(q) *
                                       (3.0f * (cm1 - B * cu) + 4.5f * (cm2c - B * cu * cu) -
                                        1.5f * ((m2xx + m2yy) - B * usq));
                    upd += B * (n[opp_of(q)] - n[q]) + dfeq;
                }
                Store<S>::st(outp + (size_t)q * a.plane, d[q] + upd);
            }
        }
        // ---- per-particle force / torque: warp reduction per candidate of this row
        if (mask) {
            unsigned m = mask;
            while (m) {
                const int s = __ffs(m) - 1;
                m &= m - 1u;
                const bool mine = c0 == s || c1 == s || c2 == s || c3 == s;
                if (!__any_sync(FULL, mine && B > 0.0f)) continue;
                float vx = (c0 == s ? fx0 : 0.f) + (c1 == s ? fx1 : 0.f) + (c2 == s ? fx2 : 0.f) +
                           (c3 == s ? fx3 : 0.f);
                float vy = (c0 == s ? fy0 : 0.f) + (c1 == s ? fy1 : 0.f) + (c2 == s ? fy2 : 0.f) +
                           (c3 == s ? fy3 : 0.f);
                float vt = (c0 == s ? t0 : 0.f) + (c1 == s ? t1 : 0.f) + (c2 == s ? t2 : 0.f) +
                           (c3 == s ? t3 : 0.f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vx += __shfl_xor_sync(FULL, vx, o);
                    vy += __shfl_xor_sync(FULL, vy, o);
                    vt += __shfl_xor_sync(FULL, vt, o);
                }
                if (lane == 0) {
                    s_part[warp][s][0] += vx;
                    s_part[warp][s][1] += vy;
                    s_part[warp][s][2] += vt;
                }
            }
        }
    }
    if (__any_sync(FULL, unstable) && lane == 0) set_err(a.err, ERR_UNSTABLE);
    if (nc) {
        __syncthreads();
        for (int t = threadIdx.x; t < nc * 3; t += BLOCK) {
            const int s = t / 3, c = t - 3 * s;
            double acc = 0.0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) acc += (double)s_part[w][s][c];
            if (acc != 0.0) {
                const int id = sh.id[s];
                if (c < 2) atomicAdd(&a.F[2 * id + c], acc);
                else atomicAdd(&a.T[id], acc);
            }
        }
    }
}

// ------------------------------------------------------------- gather
template <typename S>
__global__ void k_gather(const S *__restrict__ fin, const LatticeArgs a, double *f_out, double *rho_out,
                         double *ux_out, double *uy_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    float d[9];
    pull_cell(fin, a, x, y, d);
    const size_t c = (size_t)y * a.nx + x, nn = (size_t)a.nx * a.ny;
    double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double f = (double)w_of(q) + (double)d[q];
        if (f_out) f_out[q * nn + c] = f;
        r += f;
        jx += cx_of(q) * f;
        jy += cy_of(q) * f;
    }
    if (rho_out) {
        rho_out[c] = r;
        ux_out[c] = (jx + 0.5 * (double)a.Fx) / r;
        uy_out[c] = (jy + 0.5 * (double)a.Fy) / r;
    }
}

// ------------------------------------------------------------ cell map
__global__ void __launch_bounds__(BLOCK) k_cell_map(const LatticeArgs a, int *count, int *ids, float *eps) {
    __shared__ TileShared sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = blockIdx.x, by = blockIdx.y;
    tile_candidates(a, bx, by, sh);
    const int nc = sh.nc;
    const bool perx = a.bc_x == BC_PERIODIC, pery = a.bc_y == BC_PERIODIC;
    const int x = bx * TILE + lane;
    for (int rr = 0; rr < TILE / WARPS; ++rr) {
        const int y = by * TILE + warp + WARPS * rr;
        if (y >= a.ny || x >= a.nx) continue;
        const size_t c = (size_t)y * a.nx + x;
        unsigned m = nc ? sh.rowmask[y - by * TILE] : 0u;
        int ns = 0;
        while (m) {
            const int s = __ffs(m) - 1;
            m &= m - 1u;
            const PRec P = sh.p[s];
            const int di = wrap_rel(x - P.ci, a.nx, perx), dk = wrap_rel(y - P.cj, a.ny, pery);
            const float lox = __fsub_rn((float)di, P.fx), loy = __fsub_rn((float)dk, P.fy);
            if (!covers(lox, loy, P.r)) continue;
            if (ns < MAX_SLOTS) {
                ids[c * MAX_SLOTS + ns] = sh.id[s];
                eps[c * MAX_SLOTS + ns] = a.eps_mode == EPS_EXACT
                                              ? cell_disk_area(lox, loy, P.r)
                                              : cell_subcell_ratio(lox, loy, P.r, a.n_sub);
            } else {
                set_err(a.err, ERR_CELL_SLOTS);
            }
            ++ns;
        }
        count[c] = ns < MAX_SLOTS ? ns : MAX_SLOTS;
        for (int k = ns; k < MAX_SLOTS; ++k) {
            ids[c * MAX_SLOTS + k] = -1;
            eps[c * MAX_SLOTS + k] = 0.0f;
        }
    }
}

// ---------------------------------------------------------------- init
template <typename S>
__global__ void k_init(S *f, const LatticeArgs a, float rho0, float ux0, float uy0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.pitch || y >= a.ny) return;
    float d[9];
    equilibrium_shifted(rho0 - 1.0f, rho0, ux0, uy0, d);
#pragma unroll
    for (int q = 0; q < 9; ++q)
        Store<S>::st(f + (size_t)q * a.plane + (size_t)y * a.pitch + x, x < a.nx ? d[q] : 0.0f);
}

// ------------------------------------------------------------ launchers
template <typename F>
static cudaError_t by_storage(int storage, F &&fn) {
    switch (storage) {
    case 0: return fn((float *)nullptr);
    case 1: return fn((__half *)nullptr);
    case 2: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_populations(void *f, int storage, const LatticeArgs &a, float rho0, float ux0,
                                    float uy0, cudaStream_t s) {
    return by_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        dim3 grid((a.pitch + 255) / 256, a.ny);
        k_init<S><<<grid, 256, 0, s>>>((S *)f, a, rho0, ux0, uy0);
        return cudaGetLastError();
    });
}

cudaError_t launch_stream_collide(const void *fin, void *fout, int storage, const LatticeArgs &a,
                                  cudaStream_t s) {
    return by_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        dim3 grid((a.nx + TILE - 1) / TILE, (a.ny + TILE - 1) / TILE);
        k_stream_collide<S><<<grid, BLOCK, 0, s>>>((const S *)fin, (S *)fout, a);
        return cudaGetLastError();
    });
}

cudaError_t launch_gather(const void *fin, int storage, const LatticeArgs &a, double *f_out,
                          double *rho, double *ux, double *uy, cudaStream_t s) {
    return by_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        dim3 grid((a.nx + 127) / 128, a.ny);
        k_gather<S><<<grid, 128, 0, s>>>((const S *)fin, a, f_out, rho, ux, uy);
        return cudaGetLastError();
    });
}

cudaError_t launch_cell_map(const LatticeArgs &a, int *count, int *ids, float *eps, cudaStream_t s) {
    dim3 grid((a.nx + TILE - 1) / TILE, (a.ny + TILE - 1) / TILE);
    k_cell_map<<<grid, BLOCK, 0, s>>>(a, count, ids, eps);
    return cudaGetLastError();
}

}  // namespace imb
