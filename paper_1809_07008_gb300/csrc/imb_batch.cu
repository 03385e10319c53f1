// imb_batch.cu -- many independent small periodic domains stepped together.
//
// A sweep over resolution, solid fraction, relaxation time and driving force (the paper's
// parameter studies, Sec. 3) is a set of independent lattices.  Each is periodic in x and y,
// driven by a body force (Guo forcing, as in the single-lattice path), and holds fixed disks
// whose summed solid ratio E per cell (exact overlap area, Sec. 2.3) is computed once; its
// relaxation time may carry the Smagorinsky closure of the single-lattice path.  One
// launch advances every domain by one step: each warp takes an equal run of row segments
// (finding the domain of its first segment by binary search in the domains' first items),
// pulls with the periodic wrap of the domain (Eq. 1), collides with the blend of Eq. 13
// (B from Eq. 14, u_s = 0 for disks at rest) and adds the drag B (j - F) (Eq. 15) of the
// nodes it stepped to the domain's accumulator.  Steps run as a replayed CUDA graph of two launches (A -> B,
// B -> A); the block size and the cells per lane are chosen by timing the candidates on the
// batch itself.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/imblbm.h"
#include "imb_device.cuh"
#include "imb_kernels.h"

namespace imb {

struct BatchDomain {
    int nx, ny;
    int item0[2];       // first work item of the domain: row segments of 32 / 64 cells
    size_t off;         // element offset of the domain's plane 0 in the population buffers
    size_t plane;       // nx * ny
    size_t e_off;       // offset of the domain's solid ratios (cells)
    float tau, omega0, Fx, Fy;
    float smag_coef;    // 18 sqrt(2) C^2 of the Smagorinsky closure (0: plain BGK)
    float pad2;
};

// One node of a domain whose disks are at rest.  With u_s = 0 the solid operator of Eq. 12
// summed over the covering disks is B (f_{-q} - f^eq_{-q}(u) + f^eq_q(0) - f_q); in the
// shifted variables d_q = f_q - w_q and n_q = d_q - (f^eq_q(u) - w_q) this is
// B (n_{-q} - d_q + w_q drho), and Eq. 13 becomes
//   d*_q = d_q + (1 - B) [-omega n_q + (1 - omega / 2) w_q S_q] + B (n_{-q} - d_q + w_q drho)
// with S_q / w_q = 3 (c_q - u).F + 9 (c_q.u)(c_q.F) (Guo forcing).  The same algebra as the
// general collision with every solid-velocity moment zero, with fewer operations.
struct RestNode {
    float B, jx, jy;      // drag weight of the node (Eq. 14); jx, jy include the half-force shift
    bool ok;              // |u|^2 below the Mach guard (false for NaN)
};

// The eight moving directions as four pairs (q, -q), q = 1, 2, 5, 6, whose terms differ only in
// the sign of their odd parts: computed with FP32x2 instructions where the operations line up.
__host__ __device__ constexpr int bpair_q(int k) { return k < 2 ? k + 1 : k + 3; }

template <typename S>
__device__ __forceinline__ RestNode rest_node(const float (&d)[9], float e, const BatchDomain &D, S *__restrict__ outp) {
    RestNode r;
    float2 P[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) P[k] = make_float2(d[bpair_q(k)], d[opp_of(bpair_q(k))]);
    const float2 Sm = __fadd2_rn(__fadd2_rn(P[0], P[1]), __fadd2_rn(P[2], P[3]));
    const float drho = d[0] + (Sm.x + Sm.y);
    const float rho = 1.0f + drho;
    float Dq[4];   // d_q - d_-q
#pragma unroll
    for (int k = 0; k < 4; ++k) Dq[k] = P[k].x - P[k].y;
    const float jx = fmaf(0.5f, D.Fx, (Dq[0] + Dq[2]) - Dq[3]);   // Eqs. 3-4
    const float jy = fmaf(0.5f, D.Fy, (Dq[1] + Dq[2]) + Dq[3]);
    const float inv = __fdividef(1.0f, rho);
    const float ux = jx * inv, uy = jy * inv;
    const float usq = ux * ux + uy * uy;
    const float t = fmaf(-1.5f * rho, usq, drho);
    // non-equilibrium parts (Eq. 2): n_{+-q} = d_{+-q} - w_q (t + 4.5 rho (c.u)^2 +- 3 rho c.u)
    const float n0 = d[0] - w_of(0) * t;
    float2 N[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = bpair_q(k);
        const float cu = cdot(q, ux, uy);
        const float rcu = rho * cu;
        const float ev = fmaf(4.5f * rcu, cu, t), od = 3.0f * rcu;
        N[k] = __ffma2_rn(make_float2(-w_of(q), -w_of(q)), make_float2(ev + od, ev - od), P[k]);
    }
    float omega = D.omega0, te = D.tau;
    if (D.smag_coef > 0.0f) {       // Smagorinsky closure, as in the single-lattice path
        const float2 Ep = __fadd2_rn(N[2], N[3]);                            // (n5 + n6, n7 + n8)
        const float2 Fp = __fadd2_rn(N[2], make_float2(-N[3].x, -N[3].y));   // (n5 - n6, n7 - n8)
        const float ee = Ep.x + Ep.y;
        const float pxx = (N[0].x + N[0].y) + ee;
        const float pyy = (N[1].x + N[1].y) + ee;
        const float pxy = Fp.x + Fp.y;
        const float Q = pxx * pxx + pyy * pyy + 2.0f * pxy * pxy;
        const float sq = Q > 0.0f ? Q * rsqrtf(Q) : 0.0f;
        const float disc = fmaf(D.smag_coef * sq, inv, D.tau * D.tau);
        te = 0.5f * (D.tau + disc * rsqrtf(disc));
        omega = __fdividef(1.0f, te);
    }
    const float ec = fminf(e, 1.0f), tm = te - 0.5f;
    const float B = __fdividef(ec * tm, (1.0f - ec) + tm);   // Eq. 14 (0 in uncovered cells)
    const float fl = 1.0f - B, flw = -fl * omega, fls = fl * (1.0f - 0.5f * omega), Bd = B * drho;
    const float g = -3.0f * (ux * D.Fx + uy * D.Fy);
    // d*_q = (1 - B) d_q - (1 - B) omega n_q + B n_{-q} + w_q [(1 - B)(1 - omega/2) S_q + B drho]
    // with S_q / w_q = cF (3 + 9 cu) - 3 u.F (cF = c_q.F); both halves of a pair: cu, cF -> -cu, -cF
    Store<S>::st(outp, fmaf(fl, d[0], fmaf(flw, n0, fmaf(B, n0, fmaf(w_of(0) * fls, g, w_of(0) * Bd)))));
    const float2 fl2 = make_float2(fl, fl), flw2 = make_float2(flw, flw), B2 = make_float2(B, B);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = bpair_q(k), o = opp_of(q);
        const float cu = cdot(q, ux, uy), cF = cdot(q, D.Fx, D.Fy);
        const float kq = w_of(q) * fls, bq = w_of(q) * Bd;
        const float2 Sq = __ffma2_rn(make_float2(cF, -cF), make_float2(fmaf(9.0f, cu, 3.0f), fmaf(-9.0f, cu, 3.0f)),
                                     make_float2(g, g));
        float2 v = __ffma2_rn(make_float2(kq, kq), Sq, make_float2(bq, bq));
        v = __ffma2_rn(B2, make_float2(N[k].y, N[k].x), v);
        v = __ffma2_rn(flw2, N[k], v);
        v = __ffma2_rn(fl2, P[k], v);
        Store<S>::st(outp + (size_t)q * D.plane, v.x);
        Store<S>::st(outp + (size_t)o * D.plane, v.y);
    }
    r.B = B;
    r.jx = jx;
    r.jy = jy;
    r.ok = usq < 0.09f;
    return r;
}

// stored value as loaded (converted to FP32 where it is used)
template <typename S> __device__ __forceinline__ S ld_raw(const S *p) { return __ldg(p); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// A work item is a segment of 32 CPL cells of one row (the last segment of a row may be
// shorter); items are numbered domain by domain, row by row.  Each warp takes an equal run of
// consecutive items, so the warps finish together whatever the domain sizes, the rows a warp
// visits one after another share their neighbour rows in L1, and the drag of a domain is
// summed in registers until the warp leaves the domain.  With one cell per lane the loads of
// the next item of the same domain are issued before the arithmetic of the current one.
template <typename S, int CPL>
__global__ void __launch_bounds__(256, 3) k_batch_step(const S *__restrict__ fin, S *__restrict__ fout, const BatchDomain *__restrict__ dom,
                             int ndom, int nitems, const float *__restrict__ E, double *drag, unsigned *err) {
    constexpr int SEG = 32 * CPL;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int per = nitems / nw, rem = nitems % nw;
    int it = gw * per + min(gw, rem);
    const int end = it + per + (gw < rem ? 1 : 0);
    if (it >= end) return;   // the whole warp: gw is the same on every lane
    int lo = 0, hi = ndom - 1;   // the domain of the first item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dom[mid].item0[CPL - 1] <= it) lo = mid;
        else hi = mid - 1;
    }
    int dd = lo;
    BatchDomain D = dom[dd];
    int nseg = (D.nx + SEG - 1) / SEG;
    int y = (it - D.item0[CPL - 1]) / nseg;
    int sg = it - D.item0[CPL - 1] - y * nseg;
    bool unstable = false;
    float fx_acc = 0.0f, fy_acc = 0.0f;
    if constexpr (CPL == 1) {
        S r[9];
        float e = 0.0f;
        auto fetch = [&](const BatchDomain &Dc, int yc, int sgc) {   // pull (Eq. 1), periodic wrap
            const int x = sgc * 32 + lane, nx = Dc.nx, ny = Dc.ny, plane = (int)Dc.plane;
            if (x >= nx) return;
            const S *src = fin + Dc.off;
            const int rm = (yc == 0 ? ny - 1 : yc - 1) * nx, r0 = yc * nx, rp = (yc == ny - 1 ? 0 : yc + 1) * nx;
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int xs = cx_of(q) == 0 ? x : (cx_of(q) == 1 ? xm : xp);
                const int ys = cy_of(q) == 0 ? r0 : (cy_of(q) == 1 ? rm : rp);
                r[q] = ld_raw(src + (q * plane + ys + xs));
            }
            e = __ldg(E + Dc.e_off + (size_t)yc * nx + x);
        };
        fetch(D, y, sg);
        for (;;) {
            float d[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) d[q] = to_f32(r[q]);
            const float ec = e;
            const int x = sg * 32 + lane;
            const bool act = x < D.nx;
            S *dst = fout + D.off + (size_t)y * D.nx + x;
            ++it;
            if (++sg == nseg) {
                sg = 0;
                ++y;
            }
            const bool last = it == end, leave = last || y == D.ny;
            if (!leave) fetch(D, y, sg);   // in flight during this item's arithmetic
            if (act) {
                const RestNode c = rest_node(d, ec, D, dst);
                if (!c.ok) unstable = true;   // Mach guard, also catches NaN
                fx_acc = fmaf(c.B, c.jx - D.Fx, fx_acc);   // Eq. 15 with u_s = 0
                fy_acc = fmaf(c.B, c.jy - D.Fy, fy_acc);
            }
            if (leave) {   // leaving the domain: add its drag
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    fx_acc += __shfl_xor_sync(0xffffffffu, fx_acc, o);
                    fy_acc += __shfl_xor_sync(0xffffffffu, fy_acc, o);
                }
                if (lane == 0 && (fx_acc != 0.0f || fy_acc != 0.0f)) {
                    atomicAdd(&drag[2 * dd], (double)fx_acc);
                    atomicAdd(&drag[2 * dd + 1], (double)fy_acc);
                }
                fx_acc = fy_acc = 0.0f;
                if (last) break;
                D = dom[++dd];
                nseg = (D.nx + SEG - 1) / SEG;
                y = 0;
                fetch(D, y, sg);
            }
        }
        if (__any_sync(0xffffffffu, unstable) && lane == 0) set_err(err, ERR_UNSTABLE);
        return;
    }
    for (;;) {
        const int nx = D.nx, ny = D.ny, plane = (int)D.plane;
        const S *src = fin + D.off;
        const float *Er = E + D.e_off + (size_t)y * nx;
        S *dst = fout + D.off + (size_t)y * nx;
        const int rm = (y == 0 ? ny - 1 : y - 1) * nx, r0 = y * nx, rp = (y == ny - 1 ? 0 : y + 1) * nx;
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int x = sg * SEG + 32 * k + lane;
            if (x >= nx) continue;
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            float d[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {   // pull from x - c_q with the periodic wrap (Eq. 1)
                const int xs = cx_of(q) == 0 ? x : (cx_of(q) == 1 ? xm : xp);
                const int ys = cy_of(q) == 0 ? r0 : (cy_of(q) == 1 ? rm : rp);
                d[q] = Store<S>::ld(src + (q * plane + ys + xs));
            }
            const RestNode c = rest_node(d, Er[x], D, dst + x);
            if (!c.ok) unstable = true;   // Mach guard, also catches NaN
            fx_acc = fmaf(c.B, c.jx - D.Fx, fx_acc);   // Eq. 15 with u_s = 0
            fy_acc = fmaf(c.B, c.jy - D.Fy, fy_acc);
        }
        ++it;
        if (++sg == nseg) {
            sg = 0;
            ++y;
        }
        const bool last = it == end;
        if (last || y == ny) {   // leaving the domain: add its drag
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                fx_acc += __shfl_xor_sync(0xffffffffu, fx_acc, o);
                fy_acc += __shfl_xor_sync(0xffffffffu, fy_acc, o);
            }
            if (lane == 0 && (fx_acc != 0.0f || fy_acc != 0.0f)) {
                atomicAdd(&drag[2 * dd], (double)fx_acc);
                atomicAdd(&drag[2 * dd + 1], (double)fy_acc);
            }
            fx_acc = fy_acc = 0.0f;
            if (last) break;
            D = dom[++dd];
            nseg = (D.nx + SEG - 1) / SEG;
            y = 0;
        }
    }
    if (__any_sync(0xffffffffu, unstable) && lane == 0) set_err(err, ERR_UNSTABLE);
}

// summed solid ratio: one thread per (disk, cell of its bounding box)
__global__ void k_batch_solid(const BatchDomain *__restrict__ dom, const int *__restrict__ disk_dom,
                              const double *__restrict__ xy, const double *__restrict__ r, int ndisk, int span,
                              float *E) {
    const int w = 2 * span + 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ndisk * w * w) return;
    const int j = (int)(t / (w * w)), cell = (int)(t % (w * w));
    const BatchDomain D = dom[disk_dom[j]];
    const double cx = xy[2 * j], cy = xy[2 * j + 1];
    const int ci = (int)floor(cx), cj = (int)floor(cy);
    const float fx = (float)(cx - ci), fy = (float)(cy - cj), rf = (float)r[j];
    const int di = cell % w - span, dk = cell / w - span;
    const float lox = __fsub_rn((float)di, fx), loy = __fsub_rn((float)dk, fy);
    if (!covers(lox, loy, rf)) return;
    const int i = ((ci + di) % D.nx + D.nx) % D.nx, k = ((cj + dk) % D.ny + D.ny) % D.ny;
    atomicAdd(&E[D.e_off + (size_t)k * D.nx + i], cell_disk_area(lox, loy, rf));
}

// f(x, t) of one domain (the pull of its post-collision field), as FP64 f = w + (f - w)
template <typename S>
__global__ void k_batch_gather(const S *__restrict__ fin, const BatchDomain *__restrict__ dom, int d,
                               double *out) {
    const BatchDomain D = dom[d];
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.plane) return;
    const int x = (int)(c % D.nx), y = (int)(c / D.nx);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int xs = (x - cx_of(q) + D.nx) % D.nx, ys = (y - cy_of(q) + D.ny) % D.ny;
        out[(size_t)q * D.plane + c] =
            (double)w_of(q) + (double)Store<S>::ld(fin + D.off + (size_t)q * D.plane + (size_t)ys * D.nx + xs);
    }
}

}  // namespace imb

using namespace imb;

struct imb_batch {
    int device = 0, storage = 0, elem = 4, ndom = 0, nitems[2] = {0, 0}, ndisk = 0;
    size_t total = 0;          // elements per population buffer
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;               // buffer holding the current post-collision field
    BatchDomain *dom = nullptr;
    std::vector<BatchDomain> hdom;
    float *E = nullptr;
    double *drag = nullptr;
    unsigned *err = nullptr;
    long long steps_run = 0;
    cudaStream_t stream = nullptr;
    int block = 256, cpl = 1, grid = 0;
    bool grid_only = false;    // launch_step only sizes the grid
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // two steps starting from buffer 0 / 1
    std::string last_error;
};

namespace {

int bfail(imb_batch *b, int code, const std::string &msg) {
    if (b) b->last_error = msg;
    return code;
}

#define BCK(call, what)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? IMB_E_NOMEM : IMB_E_CUDA,       \
                         std::string(what) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

template <typename F>
cudaError_t by_storage_b(int storage, F &&fn) {
    switch (storage) {
    case IMB_STORE_FP32: return fn((float *)nullptr);
    case IMB_STORE_FP16: return fn((__half *)nullptr);
    case IMB_STORE_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

template <typename S, int CPL>
cudaError_t launch_step_t(imb_batch *b, int from) {
    auto k = k_batch_step<S, CPL>;
    if (b->grid == 0) {   // resident blocks of this configuration (set before any capture)
        int per = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, b->block, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        const long long need = ((long long)b->nitems[CPL - 1] * 32 + b->block - 1) / b->block;
        b->grid = (int)std::max(1LL, std::min(need, (long long)std::max(per, 1) * sms));
        if (b->grid_only) return cudaSuccess;
    }
    if (b->grid_only) return cudaSuccess;
    k<<<b->grid, b->block, 0, b->stream>>>((const S *)b->buf[from], (S *)b->buf[from ^ 1], b->dom, b->ndom,
                                           b->nitems[CPL - 1], b->E, b->drag, b->err);
    return cudaGetLastError();
}

// largest block the kernel of this storage and cells-per-lane can launch (its registers)
int max_block(imb_batch *b) {
    int m = 0;
    by_storage_b(b->storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        cudaFuncAttributes fa{};
        cudaError_t e = b->cpl == 2 ? cudaFuncGetAttributes(&fa, k_batch_step<S, 2>)
                                    : cudaFuncGetAttributes(&fa, k_batch_step<S, 1>);
        m = e == cudaSuccess ? fa.maxThreadsPerBlock : 0;
        return e;
    });
    return m;
}

cudaError_t launch_step(imb_batch *b, int from) {
    return by_storage_b(b->storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return b->cpl == 2 ? launch_step_t<S, 2>(b, from) : launch_step_t<S, 1>(b, from);
    });
}

void drop_graphs(imb_batch *b) {
    for (auto &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

int batch_wait(imb_batch *b) {
    BCK(cudaStreamSynchronize(b->stream), "batch stream");
    unsigned bits = 0;
    BCK(cudaMemcpy(&bits, b->err, sizeof(bits), cudaMemcpyDeviceToHost), "error flags");
    if (bits & ERR_UNSTABLE) {
        cudaMemset(b->err, 0, sizeof(unsigned));
        return bfail(b, IMB_E_UNSTABLE, "NaN or |u| >= 0.3 in a batch domain (Mach guard)");
    }
    return IMB_OK;
}

}  // namespace

extern "C" int imb_batch_create(imb_batch **out, int n_domains, const int *nx, const int *ny, const double *tau,
                                const double *C_smag, const double *Fx, const double *Fy, const int *n_disks,
                                const double *disk_xy, const double *disk_r, int storage) {
    if (!out) return IMB_E_INVALID_ARG;
    *out = nullptr;
    if (n_domains < 1 || !nx || !ny || !tau || !C_smag || !Fx || !Fy || !n_disks || storage < 0 || storage > 2)
        return IMB_E_INVALID_ARG;
    auto *b = new imb_batch();
    b->storage = storage;
    b->elem = storage == IMB_STORE_FP32 ? 4 : 2;
    b->ndom = n_domains;
    double rmax = 0.0;
    size_t cells = 0;
    long long items = 0, items2 = 0;   // row segments of 32 and of 64 cells
    int ndisk = 0;
    for (int d = 0; d < n_domains; ++d) {
        if (nx[d] < 3 || ny[d] < 3 || 9.0 * nx[d] * ny[d] > 2147483647.0 || !(tau[d] > 0.5) ||
            !(C_smag[d] >= 0.0) || n_disks[d] < 0) {
            delete b;
            return IMB_E_INVALID_ARG;
        }
        BatchDomain D{};
        D.nx = nx[d];
        D.ny = ny[d];
        D.item0[0] = (int)items;
        D.item0[1] = (int)items2;
        D.plane = (size_t)nx[d] * ny[d];
        D.off = 9 * cells;
        D.e_off = cells;
        D.tau = (float)tau[d];
        D.omega0 = (float)(1.0 / tau[d]);
        D.Fx = (float)Fx[d];
        D.Fy = (float)Fy[d];
        D.smag_coef = (float)(18.0 * std::sqrt(2.0) * C_smag[d] * C_smag[d]);
        b->hdom.push_back(D);
        cells += D.plane;
        items += (long long)ny[d] * ((nx[d] + 31) / 32);
        items2 += (long long)ny[d] * ((nx[d] + 63) / 64);
        ndisk += n_disks[d];
    }
    if (ndisk > 0 && (!disk_xy || !disk_r)) {
        delete b;
        return IMB_E_INVALID_ARG;
    }
    std::vector<int> ddom(std::max(ndisk, 1));
    for (int d = 0, j = 0; d < n_domains; ++d)
        for (int k = 0; k < n_disks[d]; ++k, ++j) {
            ddom[j] = d;
            const double x = disk_xy[2 * j], y = disk_xy[2 * j + 1], r = disk_r[j];
            if (!(r > 0.0) || !(x >= 0.0 && x < nx[d] && y >= 0.0 && y < ny[d]) || 2.0 * r + 4.0 > std::min(nx[d], ny[d])) {
                delete b;
                return IMB_E_INVALID_ARG;
            }
            rmax = std::max(rmax, r);
        }
    const long long wd = 2LL * ((long long)std::ceil(rmax) + 1) + 1;   // the solid-ratio launch's box
    if (items > 2147483647LL || ((long long)ndisk * wd * wd + 127) / 128 > 2147483647LL) {
        delete b;
        return IMB_E_INVALID_ARG;
    }
    b->nitems[0] = (int)items;
    b->nitems[1] = (int)items2;
    b->ndisk = ndisk;
    b->total = 9 * cells;
    cudaGetDevice(&b->device);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&b->buf[0], b->total * b->elem)) != cudaSuccess ||
        (e = cudaMalloc(&b->buf[1], b->total * b->elem)) != cudaSuccess ||
        (e = cudaMalloc(&b->dom, sizeof(BatchDomain) * n_domains)) != cudaSuccess ||
        (e = cudaMalloc(&b->E, sizeof(float) * std::max(cells, (size_t)1))) != cudaSuccess ||
        (e = cudaMalloc(&b->drag, sizeof(double) * 2 * n_domains)) != cudaSuccess ||
        (e = cudaMalloc(&b->err, sizeof(unsigned))) != cudaSuccess) {
        *out = b;
        return bfail(b, e == cudaErrorMemoryAllocation ? IMB_E_NOMEM : IMB_E_CUDA, "batch buffers");
    }
    *out = b;
    // fluid at rest with rho = 1: f = w, i.e. zero shifted populations
    BCK(cudaMemsetAsync(b->buf[0], 0, b->total * b->elem, b->stream), "clear");
    BCK(cudaMemsetAsync(b->buf[1], 0, b->total * b->elem, b->stream), "clear");
    BCK(cudaMemsetAsync(b->E, 0, sizeof(float) * cells, b->stream), "clear");
    BCK(cudaMemsetAsync(b->drag, 0, sizeof(double) * 2 * n_domains, b->stream), "clear");
    BCK(cudaMemsetAsync(b->err, 0, sizeof(unsigned), b->stream), "clear");
    BCK(cudaMemcpyAsync(b->dom, b->hdom.data(), sizeof(BatchDomain) * n_domains, cudaMemcpyHostToDevice, b->stream),
        "domains");
    if (ndisk > 0) {
        struct DiskArrays {   // freed on every return (cudaFree waits for the launch)
            int *dd = nullptr;
            double *xy = nullptr, *r = nullptr;
            ~DiskArrays() {
                if (dd) cudaFree(dd);
                if (xy) cudaFree(xy);
                if (r) cudaFree(r);
            }
        } t;
        BCK(cudaMalloc(&t.dd, sizeof(int) * ndisk), "disks");
        BCK(cudaMalloc(&t.xy, sizeof(double) * 2 * ndisk), "disks");
        BCK(cudaMalloc(&t.r, sizeof(double) * ndisk), "disks");
        BCK(cudaMemcpyAsync(t.dd, ddom.data(), sizeof(int) * ndisk, cudaMemcpyHostToDevice, b->stream), "disks");
        BCK(cudaMemcpyAsync(t.xy, disk_xy, sizeof(double) * 2 * ndisk, cudaMemcpyHostToDevice, b->stream), "disks");
        BCK(cudaMemcpyAsync(t.r, disk_r, sizeof(double) * ndisk, cudaMemcpyHostToDevice, b->stream), "disks");
        const int span = (int)std::ceil(rmax) + 1, w = 2 * span + 1;
        const long long nthreads = (long long)ndisk * w * w;   // grid size checked at validation
        k_batch_solid<<<(unsigned)((nthreads + 127) / 128), 128, 0, b->stream>>>(b->dom, t.dd, t.xy, t.r, ndisk,
                                                                               span, b->E);
        BCK(cudaGetLastError(), "solid ratio");
        BCK(cudaStreamSynchronize(b->stream), "solid ratio");
    }
    return batch_wait(b);
}

extern "C" int imb_batch_run(imb_batch *b, int steps) {
    if (!b) return IMB_E_INVALID_ARG;
    if (steps < 0) return bfail(b, IMB_E_INVALID_ARG, "steps must be >= 0");
    BCK(cudaSetDevice(b->device), "cudaSetDevice");
    for (int s = 0; s + 1 < steps; s += 2) {
        cudaGraphExec_t &g = b->graph[b->cur];
        if (!g) {   // two steps from the current buffer, captured once
            if (b->grid == 0) {
                b->grid_only = true;
                launch_step(b, b->cur);
                b->grid_only = false;
            }
            cudaGraph_t gr;
            BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "capture");
            cudaError_t e1 = launch_step(b, b->cur);
            cudaError_t e2 = launch_step(b, b->cur ^ 1);
            BCK(cudaStreamEndCapture(b->stream, &gr), "capture");
            BCK(e1, "capture launch");
            BCK(e2, "capture launch");
            BCK(cudaGraphInstantiate(&g, gr, 0), "graph");
            cudaGraphDestroy(gr);
        }
        BCK(cudaGraphLaunch(g, b->stream), "graph launch");
    }
    if (steps % 2) {
        BCK(launch_step(b, b->cur), "batch step");
        b->cur ^= 1;
    }
    b->steps_run += steps;
    return batch_wait(b);
}

extern "C" int imb_batch_autotune(imb_batch *b, int steps_per_trial, int *block, int *cells_per_lane,
                                  double *best_ms_per_step) {
    if (!b || steps_per_trial < 1) return IMB_E_INVALID_ARG;
    BCK(cudaSetDevice(b->device), "cudaSetDevice");
    // work on a copy of the state, put it back afterwards
    void *save = nullptr;
    BCK(cudaMalloc(&save, b->total * b->elem), "autotune copy");
    BCK(cudaMemcpyAsync(save, b->buf[b->cur], b->total * b->elem, cudaMemcpyDeviceToDevice, b->stream), "copy");
    double *dsave = nullptr;
    BCK(cudaMalloc(&dsave, sizeof(double) * 2 * b->ndom), "autotune copy");
    BCK(cudaMemcpyAsync(dsave, b->drag, sizeof(double) * 2 * b->ndom, cudaMemcpyDeviceToDevice, b->stream), "copy");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks[3] = {128, 256, 512}, cpls[2] = {1, 2};
    float best = 1e30f;
    int bb = b->block, bc = b->cpl;
    for (int bl : blocks)
        for (int cp : cpls) {
            b->block = bl;
            b->cpl = cp;
            b->grid = 0;
            if (max_block(b) < bl) continue;   // too many registers for this block size
            int from = b->cur;
            BCK(launch_step(b, from), "trial");   // warm-up
            from ^= 1;
            cudaEventRecord(e0, b->stream);
            for (int s = 0; s < steps_per_trial; ++s, from ^= 1) BCK(launch_step(b, from), "trial");
            cudaEventRecord(e1, b->stream);
            BCK(cudaEventSynchronize(e1), "trial");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bb = bl;
                bc = cp;
            }
            BCK(cudaMemcpyAsync(b->buf[b->cur], save, b->total * b->elem, cudaMemcpyDeviceToDevice, b->stream),
                "restore");
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->block = bb;
    b->cpl = bc;
    b->grid = 0;
    drop_graphs(b);
    BCK(cudaMemcpyAsync(b->drag, dsave, sizeof(double) * 2 * b->ndom, cudaMemcpyDeviceToDevice, b->stream), "copy");
    BCK(cudaStreamSynchronize(b->stream), "autotune");
    cudaFree(save);
    cudaFree(dsave);
    BCK(cudaMemset(b->err, 0, sizeof(unsigned)), "clear");
    if (block) *block = bb;
    if (cells_per_lane) *cells_per_lane = bc;
    if (best_ms_per_step) *best_ms_per_step = best / steps_per_trial;
    return IMB_OK;
}

extern "C" int imb_batch_set_launch(imb_batch *b, int block, int cells_per_lane) {
    if (!b) return IMB_E_INVALID_ARG;
    if ((block != 128 && block != 256 && block != 512) || (cells_per_lane != 1 && cells_per_lane != 2))
        return bfail(b, IMB_E_INVALID_ARG, "block must be 128, 256 or 512 and cells_per_lane 1 or 2");
    BCK(cudaSetDevice(b->device), "cudaSetDevice");
    const int old_block = b->block, old_cpl = b->cpl;
    b->cpl = cells_per_lane;
    if (max_block(b) < block) {
        b->cpl = old_cpl;
        return bfail(b, IMB_E_INVALID_ARG, "the kernel cannot launch blocks of this size");
    }
    if (block != old_block || cells_per_lane != old_cpl) {
        BCK(cudaStreamSynchronize(b->stream), "batch stream");
        b->block = block;
        b->grid = 0;
        drop_graphs(b);
    }
    return IMB_OK;
}

extern "C" int imb_batch_mean_drag(imb_batch *b, double *Fx_mean, double *Fy_mean) {
    if (!b || !Fx_mean || !Fy_mean) return IMB_E_INVALID_ARG;
    int rc = batch_wait(b);
    if (rc) return rc;
    std::vector<double> h(2 * (size_t)b->ndom);
    BCK(cudaMemcpy(h.data(), b->drag, sizeof(double) * h.size(), cudaMemcpyDeviceToHost), "drag");
    const double n = b->steps_run > 0 ? (double)b->steps_run : 1.0;
    for (int d = 0; d < b->ndom; ++d) {
        Fx_mean[d] = h[2 * d] / n;
        Fy_mean[d] = h[2 * d + 1] / n;
    }
    return IMB_OK;
}

extern "C" int imb_batch_get_populations(imb_batch *b, int domain, double *f) {
    if (!b || !f || domain < 0 || domain >= b->ndom) return IMB_E_INVALID_ARG;
    int rc = batch_wait(b);
    if (rc) return rc;
    const size_t n = 9 * b->hdom[domain].plane;
    double *t = nullptr;
    BCK(cudaMalloc(&t, sizeof(double) * n), "readback buffer");
    cudaError_t e = by_storage_b(b->storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        k_batch_gather<S><<<(unsigned)((b->hdom[domain].plane + 255) / 256), 256, 0, b->stream>>>(
            (const S *)b->buf[b->cur], b->dom, domain, t);
        return cudaGetLastError();
    });
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, t, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(t);
    BCK(e, "populations");
    return IMB_OK;
}

extern "C" long long imb_batch_cells(const imb_batch *b) {
    return b ? (long long)(b->total / 9) : 0;
}

extern "C" const char *imb_batch_last_error(const imb_batch *b) {
    return b ? b->last_error.c_str() : "null batch";
}

extern "C" void imb_batch_destroy(imb_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->dom);
    cudaFree(b->E);
    cudaFree(b->drag);
    cudaFree(b->err);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}
