// imb_pull.cuh -- the pull half of the stream step (Eq. 1 LHS) with the boundary rules:
// periodic wrap, halfway bounce-back walls (those at y = 0 and y = ny may move along x),
// velocity inlet / pressure outlet with zero velocity gradient.  Shared by the stream-collide kernel and its adjoint.
#pragma once
#include "imb_device.cuh"
#include "imb_kernels.h"

namespace imb {

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
            } else {  // halfway bounce-back: what left (x,y) towards the wall comes back, with
                      // the moving wall's momentum term 2 w_q rho_w (c_q . u_w) / c_s^2, rho_w = 1
                d[q] = Store<S>::ld(fin + self_opp);
                if (cx_of(q) != 0) d[q] += 6.0f * w_of(q) * (float)cx_of(q) * (ys < 0 ? a.uw_bot : a.uw_top);
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

// ---------------------------------------------------------------- ghost cells
// The population buffers hold a frame around the lattice: ghost rows y = -1 and ny and ghost
// columns x = -1 and nx.  A ghost cell of plane q holds what pull_generic gives the node that
// pulls q from it, so that away from the inlet and outlet columns every node reads its nine
// pulls straight from the frame.  They are written from the stored post-collision values v
// (shifted) of the edge node (x, y), after the launch that wrote them:
//  * walls: the node's own pull of q from (x, y) - c_q, when a wall rule decides it, is the
//    halfway bounce-back v_{-q} (plus the moving wall's term 6 w_q c_qx u_w for the walls
//    y = 0 and y = ny, which take precedence over the x rule at the corners);
//  * periodic boundaries: v_q at every periodic image of (x, y) in the frame from which a
//    node of the lattice pulls q.
// Each ghost cell and plane has at most one writer, and the inlet/outlet columns need none.
template <typename S>
__device__ __forceinline__ void ghost_store(S *__restrict__ f, const LatticeArgs &a, int x, int y,
                                            const float (&v)[9]) {
    auto at = [&](int q, int gx, int gy) {
        return f + (ptrdiff_t)q * (ptrdiff_t)a.plane + (ptrdiff_t)gy * a.pitch + gx;
    };
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        const int cx = cx_of(q), cy = cy_of(q);
        const int gx = x - cx, gy = y - cy;   // where the node pulls q from
        const bool yo = gy < 0 || gy >= a.ny, xo = gx < 0 || gx >= a.nx;
        if (yo && a.bc_y != BC_PERIODIC) {
            float t = v[opp_of(q)];
            if (cx != 0) t += 6.0f * w_of(q) * (float)cx * (gy < 0 ? a.uw_bot : a.uw_top);
            Store<S>::st(at(q, gx, gy), t);
        } else if (xo && a.bc_x == BC_WALL) {
            Store<S>::st(at(q, gx, gy), v[opp_of(q)]);
        }
#pragma unroll
        for (int k = -1; k <= 1; ++k)
#pragma unroll
            for (int l = -1; l <= 1; ++l) {
                if ((k == 0 && l == 0) || (k != 0 && a.bc_x != BC_PERIODIC) || (l != 0 && a.bc_y != BC_PERIODIC))
                    continue;
                const int ix = x + k * a.nx, iy = y + l * a.ny;   // a periodic image of the node
                if (ix < -1 || ix > a.nx || iy < -1 || iy > a.ny) continue;
                const int rx = ix + cx, ry = iy + cy;             // the node that pulls q from it
                if (rx < 0 || rx >= a.nx || ry < 0 || ry >= a.ny) continue;
                Store<S>::st(at(q, ix, iy), v[q]);
            }
    }
}

// shifted equilibrium f^eq_q - w_q = w_q (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2))   (Eq. 2)
__device__ __forceinline__ void equilibrium_shifted(float drho, float rho, float ux, float uy,
                                                    float (&d)[9]) {
    const float usq = ux * ux + uy * uy;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float cu = cdot(q, ux, uy);
        d[q] = w_of(q) * (drho + rho * (cu * (3.0f + 4.5f * cu) - 1.5f * usq));
    }
}

template <typename S>
__device__ __forceinline__ void pull_cell(const S *__restrict__ fin, const LatticeArgs &a, int x,
                                          int y, float (&d)[9]) {
    if (a.bc_x == BC_INLET_OUTLET && (x == 0 || x == a.nx - 1)) {
        // inlet: f^eq(rho of column 1, u_in); outlet: f^eq(1, u of column nx-2), the reference
        // pressure with zero velocity gradient
        pull_generic(fin, a, x == 0 ? 1 : a.nx - 2, y, d);
        float drho = 0.0f;
#pragma unroll
        for (int q = 0; q < 9; ++q) drho += d[q];
        if (x == 0) {
            equilibrium_shifted(drho, 1.0f + drho, a.u_in_x, a.u_in_y, d);
        } else {
            const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
            const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
            const float inv = 1.0f / (1.0f + drho);
            equilibrium_shifted(0.0f, 1.0f, jx * inv, jy * inv, d);
        }
        return;
    }
    pull_generic(fin, a, x, y, d);
}

}  // namespace imb
