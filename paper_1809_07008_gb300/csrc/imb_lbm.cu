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
#include <algorithm>
#include <type_traits>
#include <utility>

#include "imb_device.cuh"
#include "imb_kernels.h"
#include "imb_pull.cuh"
#include "imb_node.cuh"

namespace imb {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLOCK = 256;            // 8 warps; warp w handles rows w, w+8, w+16, w+24
constexpr int WARPS = BLOCK / 32;

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

// Collect (ascending id, into sh.id / sh.p) the particles whose disk can reach into
// tile (bx, by).  Executed by one full warp; returns the count (warp-uniform).
__device__ int gather_tile_candidates(const LatticeArgs &a, int bx, int by, TileShared &sh) {
    const int lane = threadIdx.x & 31;
    const bool perx = a.bc_x == BC_PERIODIC, pery = a.bc_y == BC_PERIODIC;
    {
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
        __syncwarp();
        return nc;
    }
}

// gather_tile_candidates by warp 0, then per tile row a bit mask of the candidates
// whose y-extent meets that row (whole block).
__device__ void tile_candidates(const LatticeArgs &a, int bx, int by, TileShared &sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool pery = a.bc_y == BC_PERIODIC;
    if (warp == 0) {
        const int n = gather_tile_candidates(a, bx, by, sh);
        if (lane == 0) sh.nc = n;
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
// Immersed moving boundary on one row of a warp (Sec. 2.3).  Bit s of `cm` is set when
// tile candidate s reaches into the lane's node, `rowc` is the union of cm over the warp
// (non-zero: the caller tests it), e0 the solid ratio of the lane's first candidate
// (fetched by the caller ahead of the row).  Total solid ratio -> B (Eq. 14) -> per-particle
// weights B_p = B eps_p / sum eps -> solid-velocity moments.  The per-particle force and
// torque terms of the node (Eqs. 15-16) go to the lane's register sums fa / fb when the
// candidate is ka / kb (the first two candidates of the warp's rows in the unit); those of
// any further candidate are summed over the warp's lanes at once (fixed shuffle tree) and
// added to the warp's column of the tile's partials acc_w[(3 s + c) * WARPS].
// solid ratio of tile candidate s at node (xl, yy) from the particle's table (a cell the disk
// covers in part, or any covered cell in the cell-decomposition mode)
__device__ __forceinline__ float cand_table_eps(const int *__restrict__ eoff, int s, int xl, int yy,
                                                const LatticeArgs &a) {
    return __ldg(a.eps_tab + (eoff[s] + yy * a.tab_w + xl));
}

// Solid ratio of a node that candidate s is known to reach into (covers() true): 1 when the
// cell is fully covered in exact-area mode, else the value k_particle_eps stored for it.
__device__ __forceinline__ float cand_slot_eps(const PRec *__restrict__ cand, const int *__restrict__ eoff,
                                               int s, int xl, int yy, const LatticeArgs &a) {
    const PRec &P = cand[s];
    if (a.eps_mode == EPS_EXACT &&
        fully_covered(__fsub_rn((float)(xl - P.ci), P.fx), __fsub_rn((float)(yy - P.cj), P.fy), P.r))
        return 1.0f;
    return cand_table_eps(eoff, s, xl, yy, a);
}

// force and torque terms of one node and particle (Eq. 15 per cell: -Bp sum_i Omega^s_i c_i =
// Bp (rho u - rho u_s - F); Eq. 16, z component), with the particle's solid-velocity moments
template <bool FORCED>
__device__ __forceinline__ void node_particle(const NodeState &c, const PRec &P, const int di, const int dk,
                                              const float Bp, const LatticeArgs &a, SolidMoments &sm,
                                              float &vx, float &vy, float &vt) {
    const float rx = __fsub_rn((float)di, P.fx) + 0.5f;   // node minus centre
    const float ry = __fsub_rn((float)dk, P.fy) + 0.5f;
    const float usx = P.vx - P.w * ry, usy = P.vy + P.w * rx; // u_s = v + w z x r
    sm.m1x += Bp * usx;
    sm.m1y += Bp * usy;
    sm.m2xx += Bp * usx * usx;
    sm.m2xy += Bp * usx * usy;
    sm.m2yy += Bp * usy * usy;
    vx = Bp * (c.jx - c.rho * usx - (FORCED ? a.Fx : 0.0f));
    vy = Bp * (c.jy - c.rho * usy - (FORCED ? a.Fy : 0.0f));
    vt = rx * vy - ry * vx;
}

// add one row's force terms of candidate s: to the lane's register sums when s is ka or kb,
// else summed over the warp's lanes at once (fixed shuffle tree) into the warp's column of
// the tile's partials
__device__ __forceinline__ void add_terms(const int s, float vx, float vy, float vt, const int ka, const int kb,
                                          float (&fa)[3], float (&fb)[3], float *__restrict__ acc_w) {
    if (s == ka) {
        fa[0] += vx;
        fa[1] += vy;
        fa[2] += vt;
    } else if (s == kb) {
        fb[0] += vx;
        fb[1] += vy;
        fb[2] += vt;
    } else {   // a third candidate in the warp's rows of the unit
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {   // butterfly: every lane ends with the same sums
            vx += __shfl_xor_sync(FULL, vx, o);
            vy += __shfl_xor_sync(FULL, vy, o);
            vt += __shfl_xor_sync(FULL, vt, o);
        }
        const int lane = threadIdx.x & 31;
        if (lane < 3) acc_w[(3 * s + lane) * WARPS] += lane == 0 ? vx : (lane == 1 ? vy : vt);
    }
}

template <bool FORCED>
__device__ __forceinline__ void row_imb(const NodeState &c, const int xl, const int yy, const unsigned cm,
                                        const unsigned rowc, const float e0, const PRec *__restrict__ cand,
                                        const int *__restrict__ eoff, const int ka, const int kb,
                                        float (&fa)[3], float (&fb)[3], float *__restrict__ acc_w,
                                        const LatticeArgs &a, SolidMoments &sm) {
    sm.B = sm.m1x = sm.m1y = sm.m2xx = sm.m2xy = sm.m2yy = 0.0f;
    const float tm = c.te - 0.5f;
    if (!(rowc & (rowc - 1u))) {
        // one candidate s in the row: a lane's node is covered by s alone or not at all (e0 = 0,
        // hence B = B_p = 0 and no terms)
        const int s = __ffs(rowc) - 1;
        const float eps = fminf(e0, 1.0f);
        sm.B = e0 > 0.0f ? __fdividef(eps * tm, (1.0f - eps) + tm) : 0.0f;   // Eq. 14
        const float Bp = sm.B;   // B_p = B eps_p / sum eps with a single particle
        const PRec &P = cand[s];
        float vx, vy, vt;
        node_particle<FORCED>(c, P, xl - P.ci, yy - P.cj, Bp, a, sm, vx, vy, vt);
        add_terms(s, vx, vy, vt, ka, kb, fa, fb, acc_w);
        return;
    }
    if (__popc(cm) > MAX_SLOTS) set_err(a.err, ERR_CELL_SLOTS);
    const int s0 = cm ? __ffs(cm) - 1 : 0;
    float esum = e0;   // summed in slot order
    for (unsigned m = cm & (cm - 1u); m; m &= m - 1u) esum += cand_slot_eps(cand, eoff, __ffs(m) - 1, xl, yy, a);
    if (esum > 0.0f) {
        const float eps = fminf(esum, 1.0f);
        sm.B = __fdividef(eps * tm, (1.0f - eps) + tm);       // Eq. 14
    }
    const float Bs = sm.B > 0.0f ? __fdividef(sm.B, esum) : 0.0f;
    for (unsigned m = rowc; m; m &= m - 1u) {   // warp-uniform: the row's candidates, ascending
        const int s = __ffs(m) - 1;
        float vx = 0.0f, vy = 0.0f, vt = 0.0f;
        if (((cm >> s) & 1u) && Bs > 0.0f) {
            const PRec &P = cand[s];
            const float Bp = Bs * (s == s0 ? e0 : cand_slot_eps(cand, eoff, s, xl, yy, a));
            node_particle<FORCED>(c, P, xl - P.ci, yy - P.cj, Bp, a, sm, vx, vy, vt);
        }
        add_terms(s, vx, vy, vt, ka, kb, fa, fb, acc_w);
    }
}

// Sum of six per-lane values over the warp with 9 shuffles (each level halves the values a
// lane carries): afterwards lane l holds the warp sum of value 4 b4 + 2 b3 + b2 (bits of l).
__device__ __forceinline__ float warp_sum6(const float (&fa)[3], const float (&fb)[3]) {
    const int lane = threadIdx.x & 31;
    float v[8] = {fa[0], fa[1], fa[2], fb[0], fb[1], fb[2], 0.0f, 0.0f};
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float w4[4], w2[2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float keep = h4 ? v[j + 4] : v[j], send = h4 ? v[j] : v[j + 4];
        w4[j] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float keep = h3 ? w4[j + 2] : w4[j], send = h3 ? w4[j] : w4[j + 2];
        w2[j] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    float r = (h2 ? w2[1] : w2[0]) + __shfl_xor_sync(FULL, h2 ? w2[0] : w2[1], 4);
    r += __shfl_xor_sync(FULL, r, 2);
    r += __shfl_xor_sync(FULL, r, 1);
    return r;
}

// Work unit of the persistent kernel: HROWS rows of a 32 x 32 tile; NST units are staged
// per block, so that while the warps work on one, the others are loading.  TMA boxes: the
// x start must be 16-byte aligned, so the six planes pulled from x - 1 or x + 1 (c_x = +-1)
// take a box HALO cells wider than the tile (starting HALO cells left of the tile for
// c_x = +1), the three with c_x = 0 exactly the tile width.  SMALL: lattices whose units of
// eight rows all fit on the device at once take one such unit per block (no tile counter,
// one stage, the force partials of every unit kept apart).
template <typename S, bool SMALL = false> struct Box {
    static constexpr int HROWS = SMALL ? WARPS : sizeof(S) == 4 ? 16 : 32;   // rows per work unit
    static constexpr int UPT = TILE / HROWS;                 // work units per tile
    static constexpr int RPW = HROWS / WARPS;                // rows per warp per unit
    static constexpr int HALO = 16 / (int)sizeof(S);
    static constexpr int NST = SMALL ? 1 : sizeof(S) == 4 ? 3 : 2;   // stages per block
    static constexpr int BLOCKS_PER_SM = 3;
    static constexpr int WN = TILE, WW = TILE + HALO;
    __host__ __device__ static constexpr int width(int q) { return cx_of(q) == 0 ? WN : WW; }
    __host__ __device__ static constexpr int offset(int q) {   // elements before plane q
        int o = 0;
        for (int k = 0; k < q; ++k) o += width(k) * HROWS;
        return o;
    }
    // shared-memory column of lane xl's source x - c_x in plane q's box
    __host__ __device__ static constexpr int col(int q, int xl) {
        return xl - cx_of(q) + (cx_of(q) == 1 ? HALO : 0);
    }
    static constexpr int POP_BYTES = offset(9) * (int)sizeof(S);
    static constexpr int STAGE_BYTES = (POP_BYTES + (int)sizeof(TileCand) + 127) / 128 * 128;
    // force partials of the block's last NACC tiles: [tile slot][candidate][component][warp]
    // a warp runs at most NST - 1 units ahead of the slowest, so at most two tiles are open at a
    // time; a tile's partials are flushed before the copies of the unit that takes over its
    // stage are issued, so the tile two ahead finds its slot cleared
    static constexpr int NACC = SMALL ? 1 : 2;
    static constexpr int ACC_FLOATS = NACC * TILE_CAND * 3 * WARPS;
    // partials, the tile of each stage (index, column, row, unit), warps done per stage,
    // the producer's state (units issued, tile of the unit group, next tile, end reached)
    // warps with more than two rows per unit keep their rows' coverage masks in shared memory
    // ([warp][row][lane]) rather than in registers
    static constexpr bool MASKS_IN_SMEM = RPW > 2;
    static constexpr int MASK_WORDS = MASKS_IN_SMEM ? WARPS * RPW * 32 : 0;
    static constexpr int EXTRA_BYTES = ACC_FLOATS * 4 + MASK_WORDS * 4 + NST * 16 + (NST + 4 + 3) / 4 * 16;
    static constexpr int SMEM_BYTES = NST * STAGE_BYTES + EXTRA_BYTES + NST * 8;
};
static_assert((Box<float>::WN * Box<float>::HROWS * 4) % 128 == 0 &&
                  (Box<float>::WW * Box<float>::HROWS * 4) % 128 == 0 &&
                  (Box<__half>::WN * Box<__half>::HROWS * 2) % 128 == 0 &&
                  (Box<__half>::WW * Box<__half>::HROWS * 2) % 128 == 0,
              "TMA boxes stay 128-byte aligned in shared memory");
static_assert(Box<float>::EXTRA_BYTES % 8 == 0 && Box<__half>::EXTRA_BYTES % 8 == 0, "mbarrier alignment");
static_assert(Box<float>::BLOCKS_PER_SM * (Box<float>::SMEM_BYTES + 1024) <= 228 * 1024 &&
                  Box<__half>::BLOCKS_PER_SM * (Box<__half>::SMEM_BYTES + 1024) <= 228 * 1024,
              "resident blocks per SM fit in shared memory");
static_assert((Box<float, true>::WW * Box<float, true>::HROWS * 4) % 128 == 0 &&
                  (Box<__half, true>::WW * Box<__half, true>::HROWS * 2) % 128 == 0 &&
                  Box<float, true>::UPT == Box<__half, true>::UPT && Box<float, true>::UPT == SMALL_UPT,
              "small-lattice boxes stay 128-byte aligned; its units per tile");

__device__ __forceinline__ bool tma_tile(int bx, const LatticeArgs &a) {
    // the frame's ghost cells give every pull of the tile, except at the inlet and outlet
    // columns, whose nodes are rebuilt from the pulls of their neighbours
    return a.bc_x != BC_INLET_OUTLET || (bx != 0 && bx != (a.nx - 1) / TILE);
}

// Persistent fused stream-collide.  Tiles are handed out dynamically (a counter in global
// memory), so that blocks finish together whatever their mix of tiles.  NST units are
// staged per block: nine TMA boxes (one per population plane, rows shifted by -c_y, read
// from the frame whose ghost cells carry the boundary rules) plus the tile's candidate
// block; the tiles of the inlet and outlet columns take the candidate block only and pull
// their populations with the boundary rules.  Each
// warp takes its rows of a unit, collides every node and, where a disk reaches into the
// row, the immersed nodes of the row with it.  There is no block-wide barrier: the last
// warp to finish with a stage sums the unit's force partials over the warps (FP64, fixed
// order) into the tile's partial sums, hands the stage back to the copy engine and starts
// the next unit's copies, so warps run up to NST - 1 units apart.
template <typename S, bool FORCED, bool SMALL>
__global__ void __launch_bounds__(BLOCK, Box<S, SMALL>::BLOCKS_PER_SM)
k_stream_collide(const __grid_constant__ CUtensorMap tmap_n, const __grid_constant__ CUtensorMap tmap_w,
                 const S *__restrict__ fin, S *__restrict__ fout, const LatticeArgs a,
                 const TileCand *__restrict__ tiles, const int ntiles, double *__restrict__ tile_force) {
    using G = Box<S, SMALL>;
    constexpr int NST = G::NST, HROWS = G::HROWS, UPT = G::UPT, RPW = G::RPW;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *extra = smem + NST * G::STAGE_BYTES;
    float *acc = reinterpret_cast<float *>(extra);
    unsigned *cm_smem = reinterpret_cast<unsigned *>(extra + G::ACC_FLOATS * 4);
    int4 *stage_tile = reinterpret_cast<int4 *>(extra + G::ACC_FLOATS * 4 + G::MASK_WORDS * 4);
    int *done = reinterpret_cast<int *>(stage_tile + NST);
    int *prod = done + NST;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(extra + G::EXTRA_BYTES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool smag = a.smag_coef > 0.0f;
    fin += a.origin;    // node (0, 0) of plane 0
    fout += a.origin;
    // on small lattices launched as a programmatic dependent of the previous kernel in the
    // stream: nothing that kernel writes or reads is touched before it has completed
    cudaGridDependencySynchronize();

    for (int i = threadIdx.x; i < G::ACC_FLOATS; i += BLOCK) acc[i] = 0.0f;
    if (threadIdx.x < NST) done[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
        prod[0] = 0;
        prod[3] = 0;
        if (!SMALL) prod[2] = (int)atomicAdd(&a.tile_ctr[0], 1u);   // tiles are taken one ahead
    }
    __syncthreads();

    auto stage_pop = [&](int st) { return reinterpret_cast<S *>(smem + st * G::STAGE_BYTES); };
    auto stage_cand = [&](int st) {
        return reinterpret_cast<TileCand *>(smem + st * G::STAGE_BYTES + G::POP_BYTES);
    };
    // Start the copies of the next unit into its stage (one thread; the units are issued in
    // order, by whichever warp released the stage).  Past the last tile a stage gets the end
    // marker, and nothing more is issued.
    auto issue_next = [&]() {
        if (prod[3]) return;
        const int u = prod[0], st = u % NST;
        prod[0] = u + 1;
        int t, h;
        if (SMALL) {   // the block's one unit
            const int unit = u == 0 ? (int)blockIdx.x : ntiles * UPT;
            t = unit / UPT;
            h = unit % UPT;
        } else {
            h = u % UPT;
            if (h == 0) prod[1] = prod[2];
            t = prod[1];
        }
        if (t >= ntiles) {
            prod[3] = 1;
            stage_tile[st] = make_int4(-1, 0, 0, 0);
            mbar_arrive_expect_tx(&mbar[st], 0u);
            return;
        }
        const int bx = t % a.nbx, by = t / a.nbx;
        stage_tile[st] = make_int4(t, bx, by, h);
        const bool in = tma_tile(bx, a);
        mbar_arrive_expect_tx(&mbar[st], (uint32_t)sizeof(TileCand) + (in ? (uint32_t)G::POP_BYTES : 0u));
        bulk_load(stage_cand(st), &tiles[t], (uint32_t)sizeof(TileCand), &mbar[st]);
        if (in) {
            // frame coordinates: column x + ghost_x, row y + 1 (ghost_x * sizeof(S) = 128 and
            // HALO * sizeof(S) = 16, so every box starts 16-byte aligned)
            const int x0 = bx * TILE + a.ghost_x, yb = by * TILE + h * HROWS + 1;
#pragma unroll
            for (int q = 0; q < 9; ++q)
                tma_load_3d(stage_pop(st) + G::offset(q), cx_of(q) == 0 ? (const void *)&tmap_n : (const void *)&tmap_w,
                            cx_of(q) == 1 ? x0 - G::HALO : x0, yb - cy_of(q), q, &mbar[st]);
        }
        if (!SMALL && h == 0) prod[2] = (int)atomicAdd(&a.tile_ctr[0], 1u);   // after the copies are on their way
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < NST; ++k) issue_next();

    bool unstable = false;
    for (int k = 0;; ++k) {
        const int st = k % NST;
        if (!mbar_wait(&mbar[st], (uint32_t)((k / NST) & 1))) {
            if (lane == 0) set_err(a.err, ERR_TMA);
            break;
        }
        const int4 ti = stage_tile[st];
        if (ti.x < 0) break;   // past the last tile (the same value in every warp)
        const int h = ti.w;
        const int x0 = ti.y * TILE, y0 = ti.z * TILE;
        const bool in = tma_tile(ti.y, a);
        const TileCand *tc = stage_cand(st);
        const int nc = min(tc->n, TILE_CAND);
        const S *pop = stage_pop(st);
        float *acc_t = acc + ((k / UPT) % G::NACC) * (TILE_CAND * 3 * WARPS);
        const int x = x0 + lane;
        const bool xin = x < a.nx;
        // the candidates that reach into the nodes of the warp's rows, and the solid ratio of
        // each node's first candidate (its table reads start here, ahead of the rows)
        unsigned cmr[RPW], rowcr[RPW];
        float e0r[RPW];
        unsigned uni = 0u;
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
            const int yy = h * HROWS + warp + WARPS * rr;
            unsigned cm = 0u, fm = 0u;   // candidates that reach into / cover the node whole
            if (nc && y0 + yy < a.ny) {
                for (unsigned m = tc->rowmask[yy]; m; m &= m - 1u) {
                    const int s = __ffs(m) - 1;
                    if (s < IVL_CAND) {   // the row's intervals, decided by k_tile_lists
                        const char4 iv = tc->ivl[s][yy];
                        cm |= (unsigned)(lane >= iv.x && lane <= iv.y) << s;
                        fm |= (unsigned)(lane >= iv.z && lane <= iv.w) << s;
                    } else {
                        const PRec &P = tc->p[s];
                        const float lox = __fsub_rn((float)(lane - P.ci), P.fx), loy = __fsub_rn((float)(yy - P.cj), P.fy);
                        if (covers(lox, loy, P.r)) {
                            cm |= 1u << s;
                            if (fully_covered(lox, loy, P.r)) fm |= 1u << s;
                        }
                    }
                }
                if (!xin) cm = 0u;
            }
            if (G::MASKS_IN_SMEM) cm_smem[(warp * RPW + rr) * 32 + lane] = cm;
            else cmr[rr] = cm;
            const int s0 = cm ? __ffs(cm) - 1 : 0;
            e0r[rr] = !cm ? 0.0f
                          : (a.eps_mode == EPS_EXACT && ((fm >> s0) & 1u)) ? 1.0f
                                                                          : cand_table_eps(tc->eoff, s0, lane, yy, a);
            const unsigned rowc = __reduce_or_sync(FULL, cm);
            if (!G::MASKS_IN_SMEM) rowcr[rr] = rowc;
            uni |= rowc;
        }
        // register sums of the force terms of the first two candidates of these rows
        const int ka = uni ? __ffs(uni) - 1 : -1;
        const int kb = (uni & (uni - 1u)) ? __ffs(uni & (uni - 1u)) - 1 : -1;
        float fa[3] = {0.0f, 0.0f, 0.0f}, fb[3] = {0.0f, 0.0f, 0.0f};
        // the pulls of row rr of the unit
        auto pull_row = [&](int rr, float(&d)[9]) {
            const int yy = h * HROWS + warp + WARPS * rr;
            if (in) {
                const int r = yy - h * HROWS;
#pragma unroll
                for (int q = 0; q < 9; ++q) d[q] = Store<S>::lds(pop + G::offset(q) + r * G::width(q) + G::col(q, lane));
            } else if (xin) {
                pull_cell(fin, a, x, y0 + yy, d);
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) d[q] = 0.0f;
            }
        };
        // no disk reaches into the warp's rows: fluid nodes only, without the immersed-node
        // bookkeeping (16-bit storage, whose time is the instruction stream: 0.338 -> 0.311 ms
        // without disks; the FP32 launch, nearer its memory bound, ran 0.3 % slower with it)
        if (sizeof(S) < 4 && !uni) {
#pragma unroll 1
            for (int rr = 0; rr < RPW; ++rr) {
                const int y = y0 + h * HROWS + warp + WARPS * rr;
                if (y >= a.ny) continue;
                float d[9];
                pull_row(rr, d);
                NodeState c;
                node_state(d, a, FORCED, smag, c);
                if (xin && !(c.usq < 0.09f)) unstable = true;   // Mach guard, also catches NaN
                if (xin) {
                    const SolidMoments none = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                    node_collide_store<S, false, FORCED>(d, c, none, fout + (size_t)y * a.pitch + x, a);
                }
            }
        } else
#pragma unroll 1
        for (int rr = 0; rr < RPW; ++rr) {
            const int yy = h * HROWS + warp + WARPS * rr;
            const int y = y0 + yy;
            if (y >= a.ny) continue;
            unsigned cm, rowc;
            float e0 = e0r[0];
#pragma unroll
            for (int j = 1; j < RPW; ++j)
                if (rr == j) e0 = e0r[j];
            if (G::MASKS_IN_SMEM) {
                cm = cm_smem[(warp * RPW + rr) * 32 + lane];
                rowc = __reduce_or_sync(FULL, cm);
            } else {
                cm = cmr[0];
                rowc = rowcr[0];
#pragma unroll
                for (int j = 1; j < RPW; ++j)
                    if (rr == j) {
                        cm = cmr[j];
                        rowc = rowcr[j];
                    }
            }
            float d[9];
            pull_row(rr, d);
            NodeState c;
            node_state(d, a, FORCED, smag, c);
            if (xin && !(c.usq < 0.09f)) unstable = true;   // Mach guard, also catches NaN
            if (!rowc) {
                if (xin) {
                    const SolidMoments none = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                    node_collide_store<S, false, FORCED>(d, c, none, fout + (size_t)y * a.pitch + x, a);
                }
            } else {
                SolidMoments sm;
                row_imb<FORCED>(c, lane, yy, cm, rowc, e0, tc->p, tc->eoff, ka, kb, fa, fb, acc_t + warp, a, sm);
                if (xin) node_collide_store<S, true, FORCED>(d, c, sm, fout + (size_t)y * a.pitch + x, a);
            }
        }
        if (uni) {   // the unit's sums of ka and kb into the warp's columns of the tile partials
            const float v = warp_sum6(fa, fb);
            const int j = lane >> 2;   // value j: candidate ka (j < 3) or kb, component j % 3
            if ((lane & 3) == 0 && j < 6) {
                const int s = j < 3 ? ka : kb;
                if (s >= 0) acc_t[(3 * s + j % 3) * WARPS + warp] += v;
            }
        }
        // hand the stage back: the last warp to finish with it, after the last unit of a tile,
        // sums the tile's partials over the warps (FP64, fixed order) into the tile's force
        // sums, then starts the copies of the unit NST ahead into the stage
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&done[st], 1) == WARPS - 1;
        }
        if (__shfl_sync(FULL, last, 0)) {
            __threadfence_block();
            if (SMALL || h == UPT - 1) {   // small lattices: the partials of each unit apart
                double *tf = tile_force + ((size_t)ti.x * (SMALL ? UPT : 1) + (SMALL ? h : 0)) * (TILE_CAND * 3);
                for (int i = lane; i < nc * 3; i += 32) {
                    float *pa = acc_t + i * WARPS;
                    double v = 0.0;
#pragma unroll
                    for (int w = 0; w < WARPS; ++w) {
                        v += (double)pa[w];
                        pa[w] = 0.0f;
                    }
                    tf[i] = v;
                }
            }
            __syncwarp();
            if (lane == 0) {   // after the flush: the unit issued here may open the tile that reuses the slot
                done[st] = 0;
                fence_proxy_async_smem();
                issue_next();
            }
            __syncwarp();
        }
    }
    if (__any_sync(FULL, unstable) && lane == 0) set_err(a.err, ERR_UNSTABLE);
    // the kernel that follows may be scheduled now (it waits for this one's completion before
    // it reads; scheduled earlier, its blocks held resources the persistent grid works with)
    cudaTriggerProgrammaticLaunchCompletion();
    __syncthreads();
    if (threadIdx.x == 0) {
        // after a failed wait: let every copy that was started land before the block leaves
        for (int u = max(0, prod[0] - NST); u < prod[0]; ++u) mbar_wait(&mbar[u % NST], (uint32_t)((u / NST) & 1));
        // the last block to finish leaves the tile counter at zero for the next launch
        __threadfence();
        if (atomicAdd(&a.tile_ctr[1], 1u) == gridDim.x - 1) {
            atomicExch(&a.tile_ctr[0], 0u);
            atomicExch(&a.tile_ctr[1], 0u);
        }
    }
}

// Force and torque of particle p: the sum of its partial sums over the tiles whose
// candidate lists hold it, in a fixed order (the 3 x 3 tiles around its bin, row by row), so
// that the result does not depend on the order in which the tiles were worked.
__device__ __forceinline__ void force_gather(const LatticeArgs &a, const double *__restrict__ tile_force, int p) {
    int e[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) e[j] = a.pslot[9 * p + j];
    double fx = 0.0, fy = 0.0, tz = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j)
        if (e[j] >= 0) {   // entry tile * TILE_CAND + slot; tf_units partial sets per tile
            const int t = e[j] / TILE_CAND, sl = e[j] % TILE_CAND;
            for (int v = 0; v < a.tf_units; ++v) {
                const double *tf = tile_force + (((size_t)t * a.tf_units + v) * TILE_CAND + sl) * 3;
                fx += tf[0];
                fy += tf[1];
                tz += tf[2];
            }
        }
    a.F[2 * p] = fx;
    a.F[2 * p + 1] = fy;
    a.T[p] = tz;
}

// Per-tile candidate lists: one warp per tile gathers the particles of the 3 x 3
// surrounding bins whose disk can reach the tile, in ascending id order, then (a lane per
// tile row) the row masks and the row intervals of the first IVL_CAND candidates.
__global__ void __launch_bounds__(256) k_tile_lists(const LatticeArgs a, TileCand *tiles, int ntiles) {
    __shared__ TileShared sh[WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * WARPS + warp;
    if (t >= ntiles) return;
    const int bx = t % a.nbx, by = t / a.nbx;
    const int nc = gather_tile_candidates(a, bx, by, sh[warp]);
    TileCand *out = &tiles[t];
    if (lane == 0) out->n = nc;
    if (lane < nc) {
        // centre cell relative to the tile origin, taking the periodic image nearest to
        // the tile centre: cell offsets inside the tile are then lane - ci and row - cj
        PRec P = sh[warp].p[lane];
        const int xc = bx * TILE + TILE / 2, yc = by * TILE + TILE / 2;
        P.ci = TILE / 2 - wrap_rel(xc - P.ci, a.nx, a.bc_x == BC_PERIODIC);
        P.cj = TILE / 2 - wrap_rel(yc - P.cj, a.ny, a.bc_y == BC_PERIODIC);
        const int pid = sh[warp].id[lane];
        // the solid-ratio table entry of tile node (xl, yy) is eps_tab[eoff + yy tab_w + xl]
        out->eoff[lane] = pid * a.tab_stride + (a.tab_h - P.cj) * a.tab_w + (a.tab_h - P.ci);
        out->p[lane] = P;
        sh[warp].p[lane] = P;
        // the particle's entry for this tile: its place among the 3 x 3 tiles around its bin
        const int b = a.pbin[pid], pbx = b % a.nbx, pby = b / a.nbx;
        const int dx = wrap_rel(bx - pbx, a.nbx, a.bc_x == BC_PERIODIC);
        const int dy = wrap_rel(by - pby, a.nby, a.bc_y == BC_PERIODIC);
        if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) a.pslot[9 * pid + 3 * (dy + 1) + dx + 1] = t * TILE_CAND + lane;
    }
    __syncwarp();
    // tile row `lane`: which candidates can reach into it (dy_near^2 < r^2, the rounding of
    // covers()), and the intervals of the first IVL_CAND from k_particle_rows (the per-row
    // interval search settled with covers() and fully_covered() themselves)
    unsigned rm = 0u;
    for (int s = 0; s < nc; ++s) {
        const PRec P = sh[warp].p[s];
        const float loy = __fsub_rn((float)(lane - P.cj), P.fy);
        const float hiy = __fadd_rn(loy, 1.0f);
        const float dy = loy > 0.0f ? loy : (hiy < 0.0f ? hiy : 0.0f);
        if (__fmul_rn(dy, dy) < __fmul_rn(P.r, P.r)) rm |= 1u << s;
        if (s < IVL_CAND) {
            const int dk = lane - P.cj;   // the particle's row (the same loy as above)
            int L = 1, H = 0, L2 = 1, H2 = 0;
            if (dk >= -a.tab_h && dk <= a.tab_h) {
                const char4 iv = a.pivl[(size_t)sh[warp].id[s] * a.tab_w + (dk + a.tab_h)];
                L = iv.x;
                H = iv.y;
                L2 = iv.z;
                H2 = iv.w;
            }
            int lo = max(L + P.ci, 0), hi = min(H + P.ci, TILE - 1);
            int lo2 = max(L2 + P.ci, 0), hi2 = min(H2 + P.ci, TILE - 1);
            if (L > H || lo > hi) { lo = 64; hi = -64; }
            if (L2 > H2 || lo2 > hi2) { lo2 = 64; hi2 = -64; }
            out->ivl[s][lane] = make_char4((signed char)lo, (signed char)hi, (signed char)lo2, (signed char)hi2);
        }
    }
    out->rowmask[lane] = rm;
}

// The map step of the coupling cycle (Sec. 2.4) for the partially covered cells: one
// warp per particle lists the cells of its bounding box that the disk covers only in
// part (ballot compaction, row by row), then computes their solid ratios with all 32
// lanes busy, into the particle's table (row dk + th, column di + th for the cell at
// offset (di, dk) from the centre cell).  In cell-decomposition mode fully covered
// cells are tabulated too.
constexpr int EPS_WARPS = 4;

// Cells of one row (cell rows [dk, dk + 1) relative to a disk centre at fractional
// offset (fx, fy) in its centre cell) that the disk reaches into, [L, H], and that it
// covers completely, [L2, H2] (empty when L > H).  Along a row the nearest and the
// farthest point of a cell move monotonically away from the centre on either side, so
// both sets are intervals; the ends are estimated from the chord half-widths and then
// settled with covers() and fully_covered() themselves.
__device__ __forceinline__ void row_reach(float fx, float loy, float r, int &L, int &H) {
    const float hiy = __fadd_rn(loy, 1.0f);
    const float dy = loy > 0.0f ? loy : (hiy < 0.0f ? hiy : 0.0f);
    const float r2 = __fmul_rn(r, r), dy2 = __fmul_rn(dy, dy);
    L = 1;
    H = 0;
    if (!(dy2 < r2)) return;
    auto in = [&](int l) { return covers(__fsub_rn((float)l, fx), loy, r); };
    const float w = sqrtf(r2 - dy2);
    L = (int)floorf(fx - w);
    H = (int)floorf(fx + w);
    for (int i = 0; i < 3 && in(L - 1); ++i) --L;
    for (int i = 0; i < 3 && L <= H && !in(L); ++i) ++L;
    for (int i = 0; i < 3 && in(H + 1); ++i) ++H;
    for (int i = 0; i < 3 && H >= L && !in(H); ++i) --H;
}

__device__ __forceinline__ void row_full(float fx, float loy, float r, int &L, int &H) {
    const float fy = fmaxf(fabsf(loy), fabsf(__fadd_rn(loy, 1.0f)));
    const float r2 = __fmul_rn(r, r), fy2 = __fmul_rn(fy, fy);
    L = 1;
    H = 0;
    if (!(fy2 <= r2)) return;
    auto in = [&](int l) { return fully_covered(__fsub_rn((float)l, fx), loy, r); };
    const float w = sqrtf(r2 - fy2);
    L = (int)ceilf(fx - w);
    H = (int)floorf(fx + w - 1.0f);
    for (int i = 0; i < 3 && in(L - 1); ++i) --L;
    for (int i = 0; i < 3 && L <= H && !in(L); ++i) ++L;
    for (int i = 0; i < 3 && in(H + 1); ++i) ++H;
    for (int i = 0; i < 3 && H >= L && !in(H); ++i) --H;
}

// Solid-ratio table of one particle, a warp per particle: the cells the disk reaches into
// but does not cover completely (exact area), or all cells it reaches into (cell
// decomposition).  A lane per cell row finds the row's cells, they are listed in shared
// memory, and the lanes share the list's area evaluations evenly.
constexpr int EPS_LIST = 256;

// Reached and fully covered cell intervals of every row of a particle's bounding box, a warp per
// particle and a lane per row (empty rows as [1, 0]).
__global__ void __launch_bounds__(32 * EPS_WARPS) k_particle_rows(const PRec *__restrict__ prec, int np,
                                                                  char4 *pivl, int tw, int th) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * EPS_WARPS + warp;
    if (p >= np) return;
    const PRec P = prec[p];
    const int span = (int)ceilf(P.r) + 1;
    for (int dk0 = -th; dk0 <= th; dk0 += 32) {
        const int dk = dk0 + lane;
        if (dk > th) break;
        int L = 1, H = 0, L2 = 1, H2 = 0;
        if (dk >= -span && dk <= span) {
            const float loy = __fsub_rn((float)dk, P.fy);
            row_reach(P.fx, loy, P.r, L, H);
            row_full(P.fx, loy, P.r, L2, H2);
        }
        pivl[(size_t)p * tw + (dk + th)] = make_char4((signed char)L, (signed char)H, (signed char)L2, (signed char)H2);
    }
}

__global__ void __launch_bounds__(32 * EPS_WARPS) k_particle_eps(const PRec *__restrict__ prec, int np,
                                                                 int eps_mode, int n_sub, float *tab, int tw,
                                                                 int th, int stride, const char4 *__restrict__ pivl) {
    __shared__ short2 s_lst[EPS_WARPS][EPS_LIST];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * EPS_WARPS + warp;
    if (p >= np) return;
    const PRec P = prec[p];
    const bool exact = eps_mode == EPS_EXACT;
    const int span = (int)ceilf(P.r) + 1;
    float *out = tab + (size_t)p * stride;
    short2 *lst = s_lst[warp];
    for (int dk0 = -span; dk0 <= span; dk0 += 32) {
        const int dk = dk0 + lane;
        const float loy = __fsub_rn((float)dk, P.fy);
        int L = 1, H = 0, L2 = 1, H2 = 0;
        if (dk <= span) {
            const char4 iv = pivl[(size_t)p * tw + (dk + th)];
            L = iv.x;
            H = iv.y;
            if (exact) {
                L2 = iv.z;
                H2 = iv.w;
            }
        }
        // the row's tabulated cells: [L, H] minus the fully covered run [L2, H2]
        const bool split = L2 <= H2 && L2 >= L && H2 <= H;
        const int cnt = H < L ? 0 : (H - L + 1) - (split ? H2 - L2 + 1 : 0);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        for (int base = 0; base < total; base += EPS_LIST) {
            // this lane's cells with list positions in [base, base + EPS_LIST)
            int pos = incl - cnt;
            for (int di = L; di <= H && pos < base + EPS_LIST; ++di) {
                if (split && di >= L2 && di <= H2) {
                    di = H2;
                    continue;
                }
                if (pos >= base) lst[pos - base] = make_short2((short)di, (short)dk);
                ++pos;
            }
            __syncwarp();
            const int n = min(total - base, EPS_LIST);
            for (int k = lane; k < n; k += 32) {
                const short2 c = lst[k];
                const float lox = __fsub_rn((float)c.x, P.fx), ly = __fsub_rn((float)c.y, P.fy);
                out[(c.y + th) * tw + (c.x + th)] = exact ? cell_disk_area(lox, ly, P.r)
                                                          : cell_subcell_ratio(lox, ly, P.r, n_sub);
            }
            __syncwarp();
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
    pull_cell(fin + a.origin, a, x, y, d);
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
// the lattice nodes (the rest of the frame is zero; launch_fill_ghosts follows)
template <typename S>
__global__ void k_init(S *f, const LatticeArgs a, float rho0, float ux0, float uy0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    float d[9];
    equilibrium_shifted(rho0 - 1.0f, rho0, ux0, uy0, d);
    f += a.origin;
#pragma unroll
    for (int q = 0; q < 9; ++q) Store<S>::st(f + (size_t)q * a.plane + (size_t)y * a.pitch + x, d[q]);
}

// the ghost cells of the frame from the stored populations of edge node i: rows 0 and
// ny - 1, then columns 0 and nx - 1 of the rows between
__host__ __device__ constexpr int edge_nodes(int nx, int ny) { return 2 * nx + 2 * (ny - 2); }

template <typename S>
__device__ __forceinline__ void fill_ghosts(S *f, const LatticeArgs &a, int i) {
    int x, y;
    if (i < 2 * a.nx) {
        x = i % a.nx;
        y = i < a.nx ? 0 : a.ny - 1;
    } else {
        const int j = i - 2 * a.nx;
        x = j < a.ny - 2 ? 0 : a.nx - 1;
        y = 1 + j % (a.ny - 2);
    }
    f += a.origin;
    float v[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] = Store<S>::ld(f + (size_t)q * a.plane + (size_t)y * a.pitch + x);
    ghost_store(f, a, x, y, v);
}

// What follows a stream-collide launch, in one launch: the first nbf blocks gather the
// particles' forces, the rest fill the ghost cells of the buffer f the launch wrote.
template <typename S>
__global__ void __launch_bounds__(256) k_step_tail(const LatticeArgs a, const double *__restrict__ tile_force,
                                                   S *f, int nbf) {
    cudaGridDependencySynchronize();   // on small lattices a programmatic dependent of the stream-collide launch
    cudaTriggerProgrammaticLaunchCompletion();
    if ((int)blockIdx.x < nbf) {
        const int p = blockIdx.x * blockDim.x + threadIdx.x;
        if (p < a.np) force_gather(a, tile_force, p);
    } else {
        const int i = (blockIdx.x - nbf) * blockDim.x + threadIdx.x;
        if (i < edge_nodes(a.nx, a.ny)) fill_ghosts(f, a, i);
    }
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
        dim3 grid((a.nx + 255) / 256, a.ny);
        k_init<S><<<grid, 256, 0, s>>>((S *)f, a, rho0, ux0, uy0);
        return cudaGetLastError();
    });
}

static cudaError_t step_tail(void *f, int storage, const LatticeArgs &a, const double *tile_force, int nbf,
                             cudaStream_t s) {
    return by_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nbg = (edge_nodes(a.nx, a.ny) + 255) / 256;
        return launch_dependent(k_step_tail<S>, nbf + nbg, 256, 0, s, a.tf_units == SMALL_UPT, a, tile_force, (S *)f,
                                nbf);
    });
}

cudaError_t launch_fill_ghosts(void *f, int storage, const LatticeArgs &a, cudaStream_t s) {
    return step_tail(f, storage, a, nullptr, 0, s);
}

cudaError_t launch_step_tail(void *f, int storage, const LatticeArgs &a, const double *tile_force, cudaStream_t s) {
    return step_tail(f, storage, a, tile_force, (a.np + 255) / 256, s);
}

template <typename S, bool FORCED, bool SMALL>
static int stream_collide_per_sm() {
    static int per_sm = -1;   // one device per process
    if (per_sm < 0) {
        cudaFuncSetAttribute(k_stream_collide<S, FORCED, SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Box<S, SMALL>::SMEM_BYTES);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide<S, FORCED, SMALL>, BLOCK,
                                                      Box<S, SMALL>::SMEM_BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

static int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

int stream_collide_resident_blocks(int storage) {
    const int per_sm = storage == 0 ? stream_collide_per_sm<float, false, false>()
                                    : stream_collide_per_sm<__half, false, false>();
    return per_sm * device_sms();
}

cudaError_t launch_stream_collide(const void *fin, void *fout, int storage, const LatticeArgs &a,
                                  const CUtensorMap *tmap_narrow, const CUtensorMap *tmap_wide,
                                  const TileCand *tiles, double *tile_force, bool small, cudaStream_t s) {
    const int ntiles = a.nbx * a.nby;
    return by_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        auto go = [&](auto forced, auto sm) {
            constexpr bool F = decltype(forced)::value, SM = decltype(sm)::value;
            // small lattices: one unit per block; else a persistent grid over the tiles
            const int grid = SM ? ntiles * Box<S, true>::UPT
                                : std::min(ntiles, stream_collide_per_sm<S, F, false>() * device_sms());
            if (SM) stream_collide_per_sm<S, F, true>();   // sets the shared-memory attribute
            return launch_dependent(k_stream_collide<S, F, SM>, grid, BLOCK, Box<S, SM>::SMEM_BYTES, s, SM,
                                    *tmap_narrow, *tmap_wide, (const S *)fin, (S *)fout, a, tiles, ntiles, tile_force);
        };
        const bool forced = a.Fx != 0.0f || a.Fy != 0.0f;
        if (forced && small) return go(std::true_type{}, std::true_type{});
        if (forced) return go(std::true_type{}, std::false_type{});
        if (small) return go(std::false_type{}, std::true_type{});
        return go(std::false_type{}, std::false_type{});
    });
}

cudaError_t launch_tile_lists(const LatticeArgs &a, TileCand *tiles, cudaStream_t s) {
    const int ntiles = a.nbx * a.nby;
    k_tile_lists<<<(ntiles + WARPS - 1) / WARPS, BLOCK, 0, s>>>(a, tiles, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_particle_eps(const LatticeArgs &a, cudaStream_t s) {
    if (a.np == 0) return cudaSuccess;
    k_particle_eps<<<(a.np + EPS_WARPS - 1) / EPS_WARPS, 32 * EPS_WARPS, 0, s>>>(
        a.prec, a.np, a.eps_mode, a.n_sub, a.eps_tab, a.tab_w, a.tab_h, a.tab_stride, a.pivl);
    return cudaGetLastError();
}

cudaError_t launch_particle_rows(const LatticeArgs &a, cudaStream_t s) {
    if (a.np == 0) return cudaSuccess;
    k_particle_rows<<<(a.np + EPS_WARPS - 1) / EPS_WARPS, 32 * EPS_WARPS, 0, s>>>(a.prec, a.np, a.pivl, a.tab_w,
                                                                                  a.tab_h);
    return cudaGetLastError();
}

int tma_box_width(int storage, int wide) {
    if (storage == 0) return wide ? Box<float>::WW : Box<float>::WN;
    return wide ? Box<__half>::WW : Box<__half>::WN;
}
int tma_box_rows(int storage, bool small) {
    if (small) return Box<float, true>::HROWS;
    return storage == 0 ? Box<float>::HROWS : Box<__half>::HROWS;
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
