// imb_device.cuh -- device-side definitions shared by the kernels of the
// GB300 IMB-LBM-DEM library: D2Q9 constants, the particle record read by the
// stream-collide kernel, the per-cell solid-ratio geometry, error bits and a
// bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace imb {

// D2Q9 (2D member of the lattice family of Sec. 2.1, weights of Qian et al. 1992)
// order: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
__host__ __device__ constexpr int cx_of(int q) {
    return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int q) {
    return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int q) {
    return q == 0 ? 0 : (q <= 4 ? ((q - 1 + 2) & 3) + 1 : ((q - 5 + 2) & 3) + 5);
}
__host__ __device__ constexpr float w_of(int q) {
    return q == 0 ? 4.0f / 9.0f : (q <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}

// c_q . (a, b) with the zero components of c_q left out (under IEEE rules the compiler may not
// drop a product with 0)
__device__ __forceinline__ float cdot(int q, float a, float b) {
    const int x = cx_of(q), y = cy_of(q);
    const float ta = x > 0 ? a : -a, tb = y > 0 ? b : -b;
    return x == 0 ? (y == 0 ? 0.0f : tb) : (y == 0 ? ta : ta + tb);
}
// c_q c_q : (A xx, A yy, A xy) likewise
__device__ __forceinline__ float ccdot(int q, float axx, float ayy, float axy) {
    const int x = cx_of(q), y = cy_of(q);
    if (x == 0 && y == 0) return 0.0f;
    if (y == 0) return axx;
    if (x == 0) return ayy;
    return (x == y ? axx + 2.0f * axy : axx - 2.0f * axy) + ayy;
}

enum : int { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET_OUTLET = 2 };
enum : int { EPS_EXACT = 0, EPS_SUBCELL = 1 };

// device error bits (translated to IMB_E_* on the host)
enum : unsigned {
    ERR_UNSTABLE = 1u,       // NaN or Mach guard
    ERR_CELL_SLOTS = 2u,     // more than 4 particles cover one cell
    ERR_TILE_LIST = 4u,      // more than TILE_CAND particles touch one tile
    ERR_NEIGHBOURS = 8u,     // DEM neighbour list full
    ERR_SKIN = 16u,          // a particle moved more than skin/2 in one coupling cycle
    ERR_BARRIER = 32u,       // a bounded grid barrier gave up
    ERR_TMA = 64u,           // a bounded wait on a TMA / bulk copy gave up
    ERR_LIST = 128u,         // a per-cycle particle list met its capacity (its count not reset)
};

constexpr int TILE = 32;        // stream-collide tile edge == bin edge (cells)
constexpr int TILE_CAND = 32;   // max particles touching one tile
constexpr int MAX_SLOTS = 4;    // max particles covering one cell
constexpr int MAX_NBR = 16;     // max DEM neighbour candidates per particle

// Particle as seen by the lattice kernels, rebuilt after every DEM update.
// (ci, cj) = floor of the FP64 centre, (fx, fy) = FP64 fractional offset rounded
// to FP32; cell-relative geometry is formed from these in FP32.
struct __align__(16) PRec {
    int ci, cj;
    float fx, fy;
    float r, vx, vy, w;
};

constexpr int IVL_CAND = 4;     // candidates whose per-row cell intervals a tile block carries

// Particles that can reach one 32 x 32 tile, ascending id (built by k_tile_lists,
// bulk-copied into shared memory by the stream-collide kernel), with the offset of each
// one's solid-ratio table such that eps_tab[eoff + yy tab_w + xl] is the entry of tile node
// (xl, yy) (32-bit: n tab_w^2 < 2^31 is checked when the particles are set).  For each tile row, the
// candidates that can reach into it, and for the first IVL_CAND candidates the columns
// (tile-relative) of the row's cells the disk reaches into, [x, y], and covers whole, [z, w]
// (empty when the lower end exceeds the upper): the same decisions as covers() and
// fully_covered() on each cell.
struct __align__(16) TileCand {
    int n;
    int pad[3];
    int eoff[TILE_CAND];
    PRec p[TILE_CAND];
    unsigned rowmask[TILE];
    char4 ivl[IVL_CAND][TILE];
};
static_assert(sizeof(TileCand) % 16 == 0, "bulk copies move multiples of 16 bytes");

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int wrap_rel(int d, int L, bool periodic) {
    // minimum image of an integer cell offset into [-L/2, L/2) (L/2 rounded down)
    if (periodic) {
        int h = L / 2;
        if (d >= h) d -= L;
        else if (d < -h) d += L;
    }
    return d;
}

__device__ __forceinline__ void set_err(unsigned *err, unsigned bit) {
    atomicOr(err, bit);
}

// ------------------------------------------------- solid ratio (Sec. 2.3)
// Coverage decision: does the disk of radius r reach into the open unit cell whose
// lower-left corner is (lox, loy) relative to the centre?  Nearest point of the cell
// strictly inside the circle; every operation rounded separately (no FMA).
__device__ __forceinline__ bool covers(float lox, float loy, float r) {
    float hix = __fadd_rn(lox, 1.0f), hiy = __fadd_rn(loy, 1.0f);
    float dx = lox > 0.0f ? lox : (hix < 0.0f ? hix : 0.0f);
    float dy = loy > 0.0f ? loy : (hiy < 0.0f ? hiy : 0.0f);
    float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return d2 < __fmul_rn(r, r);
}

// Is the whole cell inside the disk?  Farthest corner within the circle, every
// operation rounded separately (the same decision wherever it is taken).
__device__ __forceinline__ bool fully_covered(float lox, float loy, float r) {
    const float fx = fmaxf(fabsf(lox), fabsf(__fadd_rn(lox, 1.0f)));
    const float fy = fmaxf(fabsf(loy), fabsf(__fadd_rn(loy, 1.0f)));
    return __fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)) <= __fmul_rn(r, r);
}

// 0: the disk does not reach into the cell, 1: it covers part of it, 2: all of it.
__device__ __forceinline__ int cover_state(float lox, float loy, float r) {
    if (!covers(lox, loy, r)) return 0;
    return fully_covered(lox, loy, r) ? 2 : 1;
}

// asin(s) - s sqrt(1 - s^2): twice the area of the circular segment of a unit circle
// cut by a chord of half-length s, divided by 2.  Series for small s avoids the
// cancellation: 2/3 s^3 + 1/5 s^5 + 3/28 s^7 + 5/72 s^9 + 35/704 s^11 + ...
__device__ __forceinline__ float segment_unit(float s) {
    if (s < 0.25f) {
        float s2 = s * s;
        float p = fmaf(s2, 35.0f / 704.0f, 5.0f / 72.0f);
        p = fmaf(s2, p, 3.0f / 28.0f);
        p = fmaf(s2, p, 0.2f);
        p = fmaf(s2, p, 2.0f / 3.0f);
        return s * s2 * p;
    }
    return asinf(s) - s * sqrtf(fmaxf(0.0f, 1.0f - s * s));
}

// h(x) - y0 for the upper arc h = sqrt(r^2 - x^2), without cancellation when y0 > 0.
__device__ __forceinline__ float arc_gap(float x, float h, float y0, float r) {
    if (y0 > 0.0f) {
        float num = fmaf(-y0, y0, (r - x) * (r + x));
        return num / (h + y0);
    }
    return h - y0;
}

// Integral over [p, q] of (h(x) - y0) where the arc stays inside the strip:
// trapezoid under the chord plus the circular segment between chord and arc.
__device__ __forceinline__ float arc_piece(float p, float q, float y0, float r) {
    float hp = sqrtf(fmaxf(0.0f, (r - p) * (r + p)));
    float hq = sqrtf(fmaxf(0.0f, (r - q) * (r + q)));
    float gp = arc_gap(p, hp, y0, r), gq = arc_gap(q, hq, y0, r);
    float w = q - p;
    float trap = 0.5f * w * (gp + gq);
    float dh = (hp + hq > 1.0e-3f * r) ? (p - q) * (p + q) / (hp + hq) : (hq - hp);
    float L = sqrtf(w * w + dh * dh);
    float s = fminf(1.0f, 0.5f * L / r);
    return trap + r * r * segment_unit(s);
}

// U = integral over x in [a0, a1] (inside [-r, r]) of (clamp(h(x), y0, y1) - y0):
// the part of the strip y0 <= y <= y1 below the upper arc.
__device__ __forceinline__ float strip_under_arc(float a0, float a1, float y0, float y1, float r) {
    if (!(a1 > a0)) return 0.0f;
    // |x| <= s1: arc above y1 (full strip height); |x| >= s0: arc below y0 (nothing)
    float s1 = (y1 <= 0.0f) ? r : (y1 < r ? sqrtf((r - y1) * (r + y1)) : -1.0f);
    float s0 = (y0 <= 0.0f) ? r : (y0 < r ? sqrtf((r - y0) * (r + y0)) : 0.0f);
    float U = 0.0f;
    if (s1 >= 0.0f) {
        float lo = fmaxf(a0, -s1), hi = fminf(a1, s1);
        if (hi > lo) U += (y1 - y0) * (hi - lo);
    }
    float s1c = fmaxf(s1, 0.0f);
    if (s0 > s1c) {
        float lo = fmaxf(a0, -s0), hi = fminf(a1, -s1c);
        if (hi > lo) U += arc_piece(lo, hi, y0, r);
        lo = fmaxf(a0, s1c); hi = fminf(a1, s0);
        if (hi > lo) U += arc_piece(lo, hi, y0, r);
    }
    return U;
}

// Exact area of the disk (radius r, centred at the origin) inside the unit cell
// [lox, lox+1] x [loy, loy+1], single precision.  The cell is first mapped by the
// symmetries of the disk so that it lies in the sector |x| <= y, where the arc
// crossing it is a graph y = h(x) of slope at most about one.
__device__ __forceinline__ float cell_disk_area(float lox, float loy, float r) {
    float x0 = lox, y0 = loy;
    if (fabsf(x0 + 0.5f) > fabsf(y0 + 0.5f)) { float t = x0; x0 = y0; y0 = t; }
    if (y0 + 0.5f < 0.0f) y0 = -y0 - 1.0f;
    float x1 = x0 + 1.0f, y1 = y0 + 1.0f;
    if (fully_covered(lox, loy, r)) return 1.0f;
    float a0 = fmaxf(x0, -r), a1 = fminf(x1, r);
    if (!(a1 > a0)) return 0.0f;
    float A = strip_under_arc(a0, a1, y0, y1, r);
    if (y0 < 0.0f) A += strip_under_arc(a0, a1, -y1, -y0, r) - (a1 - a0) * (y1 - y0);
    return fminf(1.0f, fmaxf(0.0f, A));
}

// Cell decomposition of Fig. 3b: fraction of n x n sub-cell centres inside the disk
// (a tie counts as inside), every operation rounded separately.
__device__ __forceinline__ float cell_subcell_ratio(float lox, float loy, float r, int n) {
    float r2 = __fmul_rn(r, r);
    float fn = (float)n;
    int inside = 0;
    for (int ky = 0; ky < n; ++ky) {
        float py = __fadd_rn(loy, __fdiv_rn(__fadd_rn((float)ky, 0.5f), fn));
        float py2 = __fmul_rn(py, py);
        for (int kx = 0; kx < n; ++kx) {
            float px = __fadd_rn(lox, __fdiv_rn(__fadd_rn((float)kx, 0.5f), fn));
            inside += __fadd_rn(__fmul_rn(px, px), py2) <= r2;
        }
    }
    return (float)inside / (float)(n * n);
}

// ------------------------------------------------------ population storage
template <typename S> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float lds(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float lds(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ float lds(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// -------------------------------------------------- bounded grid barrier
// Sense-reversing barrier over all blocks of a cooperative launch.  Each wait is
// bounded; on timeout the block records ERR_BARRIER and returns false.
struct GridBarrier {
    unsigned count;
    unsigned gen;
};

__device__ __forceinline__ bool grid_barrier(GridBarrier *b, unsigned nblocks, unsigned *err) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &b->gen;
        unsigned g = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long spins = 0;
            volatile unsigned *verr = err;
            while (*vgen == g) {
                // give up after ~4 s, or at once when another block already gave up
                if (++spins > (1ll << 26) || (*verr & ERR_BARRIER)) {
                    set_err(err, ERR_BARRIER);
                    ok = 0;
                    break;
                }
                if (spins > 64) __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// --------------------------------------------- mbarrier / TMA primitives
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 3D tiled TMA load of one box into shared memory, completing on bar
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)tmap), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
// untiled bulk copy global -> shared (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"((uint64_t)src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace imb
