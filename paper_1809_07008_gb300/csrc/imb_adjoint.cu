// imb_adjoint.cu -- reverse-mode gradient of the time-averaged drag on fixed disks.
//
// The forward step is the stream-collide kernel: f(t) = pull(P(t-1)) with the boundary
// rules (Eq. 1 LHS), P(t) = collision of f(t) (Eqs. 1-2, 12-14), drag D(t) = sum_p F_x,p
// (Eq. 15).  For disks at rest, plain BGK and no body force the solid term summed over a
// cell's disks is B (f_{-i} - f^eq_{-i}(rho, u) + w_i rho - f_i) and the cell's drag is
// B j_x, so J = (1/T) sum_t D(t) depends on the disk positions only through the summed
// solid ratio E of each cell.  Going backwards in time, one kernel per step
//   * gathers the adjoint of P(t) from the adjoint of f(t+1) (the transpose of the pull:
//     a gather at x + c_i, bounce-back entries from the cell itself),
//   * recomputes f(t) from P(t-1) and applies the transposed Jacobian of the collision
//     (plus the drag's own dependence on f),
//   * adds d J / d tau and d J / d E of the cell.
// The inlet rows of the transposed pull (f(0) = f^eq(rho of column 1, u_in), f(nx-1) =
// f^eq(1, u of column nx-2)) run as a separate small kernel, which also adds d J / d u_in.  d E / d (disk
// centre) is the difference of the chord lengths on opposite cell edges.
#include "imb_device.cuh"
#include "imb_kernels.h"
#include "imb_pull.cuh"

namespace imb {

// one block reduces F_x over the disks and adds it to *acc
__global__ void __launch_bounds__(256) k_drag_sum(const double *__restrict__ F, int np, double *acc) {
    __shared__ double s[8];
    double v = 0.0;
    for (int p = threadIdx.x; p < np; p += 256) v += F[2 * p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s[w];
        *acc += t;
    }
}

// summed solid ratio of every cell, in slot order (the order the collision sums them)
__global__ void k_cell_E(const int *__restrict__ count, const float *__restrict__ eps, size_t ncell, float *E) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    float e = 0.0f;
    for (int k = 0; k < count[c]; ++k) e += eps[c * MAX_SLOTS + k];
    E[c] = e;
}

// adjoint of the inlet and outlet columns of the pull, applied in place to the adjoint of
// f(t+1) before the step-t kernel gathers from it; S1 is P(t), from which f(t+1) is pulled.
// One warp per row, lane q < 9 for population q.
__global__ void k_adjoint_inlet(float *__restrict__ lam, const float *__restrict__ S1, const LatticeArgs a,
                                double *g_uin) {
    const int y = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), q = threadIdx.x & 31;
    if (y >= a.ny) return;   // whole warp
    lam += a.origin;         // node (0, 0) of plane 0 in the frame
    S1 += a.origin;
    const bool on = q < 9;
    const size_t row = (size_t)y * a.pitch;
    float *l = lam + (size_t)(on ? q : 0) * a.plane + row;
    // population q of f(t+1) at column col (an interior column), pulled from S1
    auto pulled = [&](int col) -> float {
        if (!on) return 0.0f;
        int ys = y - cy_of(q);
        size_t src;
        if (ys < 0 || ys >= a.ny) {
            if (a.bc_y == BC_PERIODIC) {
                ys = ys < 0 ? ys + a.ny : ys - a.ny;
                src = (size_t)q * a.plane + (size_t)ys * a.pitch + (col - cx_of(q));
            } else {
                src = (size_t)opp_of(q) * a.plane + row + col;   // halfway bounce-back
            }
        } else {
            src = (size_t)q * a.plane + (size_t)ys * a.pitch + (col - cx_of(q));
        }
        return S1[src];
    };
    auto wsum = [](float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    const float cxq = on ? (float)cx_of(q) : 0.0f, cyq = on ? (float)cy_of(q) : 0.0f;
    const float wq = on ? w_of(q) : 0.0f;
    // outlet: f(nx-1) = f^eq(1, u), u = j / rho of f(nx-2); d f^eq_q / d u = w_q (3 c_q +
    // 9 (c_q . u) c_q - 3 u), d u / d f_p(nx-2) = (c_p - u) / rho
    {
        const float dq = pulled(a.nx - 2);
        const float rho = 1.0f + wsum(dq), ux = wsum(cxq * dq) / rho, uy = wsum(cyq * dq) / rho;
        const float lo = on ? l[a.nx - 1] : 0.0f, cu = cxq * ux + cyq * uy;
        const float gx = wsum(lo * wq * (3.0f * cxq + 9.0f * cu * cxq - 3.0f * ux));
        const float gy = wsum(lo * wq * (3.0f * cyq + 9.0f * cu * cyq - 3.0f * uy));
        if (on) {
            l[a.nx - 1] = 0.0f;
            l[a.nx - 2] += (gx * (cxq - ux) + gy * (cyq - uy)) / rho;
        }
    }
    // inlet: f(0) = f^eq(rho1, u_in), rho1 = 1 + the pulled shifted populations of column 1
    const float dq = wsum(pulled(1));
    const float ux = a.u_in_x, uy = a.u_in_y, usq = ux * ux + uy * uy;
    const float cu = cxq * ux + cyq * uy;
    const float l0 = on ? l[0] : 0.0f;
    const float lr = wsum(l0 * wq * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
    const float gq = wsum(l0 * wq * (3.0f * cxq + 9.0f * cu * cxq - 3.0f * ux));
    if (on) {
        l[0] = 0.0f;
        l[1] += lr;
    }
    if (q == 0 && gq != 0.0f) atomicAdd(g_uin, (double)(gq * (1.0f + dq)));
}

// One step backwards: lam1 = d J / d f(t+1) (columns already transposed), S0 = P(t-1)
// (f(t) is pulled from it); writes lam0 = d J / d f(t).
__global__ void __launch_bounds__(256) k_adjoint_step(const float *__restrict__ lam1, const float *__restrict__ S0,
                                                      float *__restrict__ lam0, const LatticeArgs a,
                                                      const float *__restrict__ E, double *__restrict__ gE,
                                                      float inv_T, double *g_tau) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    double gt = 0.0;
    lam1 += a.origin;   // node (0, 0) of plane 0 in the frame
    S0 += a.origin;
    lam0 += a.origin;
    if (x < a.nx) {
        // adjoint of P(t) at (x, y): who pulled P_q(x, y); and f(t) at (x, y), pulled from
        // P(t-1) (shifted populations d = f - w).  Away from the edges no boundary rule applies.
        float L[9], d[9];
        const bool inner = x >= 1 && x <= a.nx - 2 && y >= 1 && y <= a.ny - 2;
        if (inner) {
            const size_t c0 = (size_t)y * a.pitch + x;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const ptrdiff_t off = (ptrdiff_t)cy_of(q) * a.pitch + cx_of(q);
                L[q] = lam1[(size_t)q * a.plane + c0 + off];
                d[q] = S0[(size_t)q * a.plane + c0 - off];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                int xd = x + cx_of(q), yd = y + cy_of(q);
                bool bounce = false, gone = false;
                if (yd < 0 || yd >= a.ny) {
                    if (a.bc_y == BC_PERIODIC) yd = yd < 0 ? yd + a.ny : yd - a.ny;
                    else bounce = true;
                }
                if (!bounce && (xd < 0 || xd >= a.nx)) {
                    if (a.bc_x == BC_PERIODIC) xd = xd < 0 ? xd + a.nx : xd - a.nx;
                    else if (a.bc_x == BC_WALL) bounce = true;
                    else gone = true;
                }
                L[q] = gone ? 0.0f
                       : bounce ? lam1[(size_t)opp_of(q) * a.plane + (size_t)y * a.pitch + x]
                                : lam1[(size_t)q * a.plane + (size_t)yd * a.pitch + xd];
            }
            pull_cell(S0, a, x, y, d);
        }
        float drho = 0.0f, jx = 0.0f, jy = 0.0f;
#pragma unroll
        for (int q = 0; q < 9; ++q) {   // products with a zero velocity component left out
            drho += d[q];
            if (cx_of(q) != 0) jx += cx_of(q) > 0 ? d[q] : -d[q];
            if (cy_of(q) != 0) jy += cy_of(q) > 0 ? d[q] : -d[q];
        }
        const float rho = 1.0f + drho, ux = jx / rho, uy = jy / rho, usq = ux * ux + uy * uy;
        float n[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float cu = cdot(q, ux, uy);
            n[q] = d[q] - w_of(q) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
        }
        const size_t c = (size_t)y * a.nx + x;
        const float Ec = E[c], e = fminf(Ec, 1.0f), tau = a.tau, tm = tau - 0.5f;
        const float B = Ec > 0.0f ? e * tm / ((1.0f - e) + tm) : 0.0f;
        const float af = (1.0f - B) / tau;
        float mu[9], nu = 0.0f;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            mu[q] = af * L[q] - B * L[opp_of(q)];
            nu += B * w_of(q) * L[q];
        }
        float lr = nu, ljx = 0.0f, ljy = 0.0f;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float cxq = (float)cx_of(q), cyq = (float)cy_of(q), cu = cdot(q, ux, uy);
            lr += mu[q] * w_of(q) * (1.0f - 4.5f * cu * cu + 1.5f * usq);
            ljx += mu[q] * w_of(q) * (cx_of(q) != 0 ? 3.0f * cxq + 9.0f * cu * cxq - 3.0f * ux : -3.0f * ux);
            ljy += mu[q] * w_of(q) * (cy_of(q) != 0 ? 3.0f * cyq + 9.0f * cu * cyq - 3.0f * uy : -3.0f * uy);
        }
        float gtf = 0.0f;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float cxq = (float)cx_of(q), cyq = (float)cy_of(q);
            float v = L[q] * (1.0f - af - B) + B * L[opp_of(q)];
            if (cx_of(q) != 0) v += inv_T * B * cxq;
            v += lr;
            if (cx_of(q) != 0) v += cxq * ljx;
            if (cy_of(q) != 0) v += cyq * ljy;
            lam0[(size_t)q * a.plane + (size_t)y * a.pitch + x] = v;
            gtf += L[q] * (1.0f - B) * n[q] / (tau * tau);
        }
        gt = gtf;
        if (B > 0.0f) {
            float lB = inv_T * jx;
#pragma unroll
            for (int q = 0; q < 9; ++q)
                lB += L[q] * (n[q] / tau + n[opp_of(q)] + w_of(q) * drho - d[q]);
            const float den = (1.0f - e) + tm;
            gt += (double)(lB * e * (1.0f - e) / (den * den));
            if (Ec < 1.0f) gE[c] += (double)(lB * tm * (1.0f + tm) / (den * den));
        }
    }
    __shared__ double s[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gt += __shfl_xor_sync(0xffffffffu, gt, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = gt;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        if (t != 0.0) atomicAdd(g_tau, t);
    }
}

// vertical chord of a disk centred at the origin on the line x = a, within [b0, b1]
__device__ __forceinline__ double chord_len(double a, double b0, double b1, double r) {
    if (!(fabs(a) < r)) return 0.0;
    const double h = sqrt(r * r - a * a);
    const double lo = fmax(b0, -h), hi = fmin(b1, h);
    return hi > lo ? hi - lo : 0.0;
}

// d J / d (disk centre) = sum over the cells a disk covers of d J / d E times d E / d centre
__global__ void k_position_grad(const int *__restrict__ count, const int *__restrict__ ids,
                                const double *__restrict__ gE, const double *__restrict__ xp,
                                const double *__restrict__ rp, int nx, int ny, int bc_x, int bc_y,
                                double *dJ_dx) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (size_t)nx * ny || count[c] == 0 || gE[c] == 0.0) return;
    const int i = (int)(c % nx), k = (int)(c / nx);
    for (int sl = 0; sl < count[c]; ++sl) {
        const int p = ids[c * MAX_SLOTS + sl];
        const double cx = xp[2 * p], cy = xp[2 * p + 1], r = rp[p];
        double ax = (double)i - cx, ay = (double)k - cy;   // cell corner relative to the centre
        if (bc_x == BC_PERIODIC) ax -= nx * rint(ax / nx);
        if (bc_y == BC_PERIODIC) ay -= ny * rint(ay / ny);
        // moving the centre by +d moves the cell by -d relative to the disk
        const double gx = chord_len(ax, ay, ay + 1.0, r) - chord_len(ax + 1.0, ay, ay + 1.0, r);
        const double gy = chord_len(ay, ax, ax + 1.0, r) - chord_len(ay + 1.0, ax, ax + 1.0, r);
        atomicAdd(&dJ_dx[2 * p], gE[c] * gx);
        atomicAdd(&dJ_dx[2 * p + 1], gE[c] * gy);
    }
}

cudaError_t launch_drag_sum(const double *F, int np, double *acc, cudaStream_t s) {
    k_drag_sum<<<1, 256, 0, s>>>(F, np, acc);
    return cudaGetLastError();
}

cudaError_t launch_cell_E(const int *count, const float *eps, size_t ncell, float *E, cudaStream_t s) {
    k_cell_E<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(count, eps, ncell, E);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_inlet(float *lam, const float *S1, const LatticeArgs &a, double *g_uin,
                                 cudaStream_t s) {
    k_adjoint_inlet<<<(a.ny + 7) / 8, 256, 0, s>>>(lam, S1, a, g_uin);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const float *lam1, const float *S0, float *lam0, const LatticeArgs &a,
                                const float *E, double *gE, float inv_T, double *g_tau, cudaStream_t s) {
    dim3 grid((a.nx + 255) / 256, a.ny);
    k_adjoint_step<<<grid, 256, 0, s>>>(lam1, S0, lam0, a, E, gE, inv_T, g_tau);
    return cudaGetLastError();
}

cudaError_t launch_position_grad(const int *count, const int *ids, const double *gE, const double *x,
                                 const double *r, int nx, int ny, int bc_x, int bc_y, double *dJ_dx,
                                 cudaStream_t s) {
    const size_t n = (size_t)nx * ny;
    k_position_grad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(count, ids, gE, x, r, nx, ny, bc_x, bc_y, dJ_dx);
    return cudaGetLastError();
}

}  // namespace imb
