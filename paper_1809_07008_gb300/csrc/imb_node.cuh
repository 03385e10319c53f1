// imb_node.cuh -- the collision of one lattice node: moments (Eqs. 2-4), the Smagorinsky
// relaxation time, and the blend of the fluid BGK operator with the solid operator of Eq. 12
// (Eq. 13), followed by the store of the post-collision populations.  Shared by the
// stream-collide kernel and the batched-domain kernel.
#pragma once
#include "imb_device.cuh"
#include "imb_kernels.h"

namespace imb {

// Macroscopic state of one node (Eqs. 2-4) and its relaxation rate.
struct NodeState {
    float drho, rho, jx, jy, ux, uy, usq, te, omega;
    float n[9];   // non-equilibrium parts f_i - f_i^eq
};

__device__ __forceinline__ void node_state(const float (&d)[9], const LatticeArgs &a, const bool forced,
                                           const bool smag, NodeState &c) {
    // ---- moments (Eqs. 3-4, Guo half-force shift)
    c.drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    c.rho = 1.0f + c.drho;
    c.jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    c.jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    if (forced) {
        c.jx = fmaf(0.5f, a.Fx, c.jx);
        c.jy = fmaf(0.5f, a.Fy, c.jy);
    }
    const float inv = __fdividef(1.0f, c.rho);
    c.ux = c.jx * inv;
    c.uy = c.jy * inv;
    c.usq = c.ux * c.ux + c.uy * c.uy;
    // ---- non-equilibrium parts (Eq. 2)
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float cu = cdot(q, c.ux, c.uy);
        c.n[q] = d[q] - w_of(q) * (c.drho + c.rho * (cu * (3.0f + 4.5f * cu) - 1.5f * c.usq));
    }
    // ---- Smagorinsky effective relaxation time (Hou et al. 1996 closure)
    c.omega = a.omega0;
    c.te = a.tau;
    if (smag) {
        const float pxx = (c.n[1] + c.n[3]) + (c.n[5] + c.n[6]) + (c.n[7] + c.n[8]);
        const float pyy = (c.n[2] + c.n[4]) + (c.n[5] + c.n[6]) + (c.n[7] + c.n[8]);
        const float pxy = (c.n[5] - c.n[6]) + (c.n[7] - c.n[8]);
        const float Q = pxx * pxx + pyy * pyy + 2.0f * pxy * pxy;
        const float sq = Q > 0.0f ? Q * rsqrtf(Q) : 0.0f;          // sqrt(Q)
        const float disc = fmaf(a.smag_coef * sq, inv, a.tau * a.tau);
        c.te = 0.5f * (a.tau + disc * rsqrtf(disc));                // (tau + sqrt(disc)) / 2
        c.omega = __fdividef(1.0f, c.te);
    }
}

// Solid-velocity moments of the particles covering a node, weighted by B_p.
struct SolidMoments {
    float B, m1x, m1y, m2xx, m2xy, m2yy;
};

// Collision (Eq. 13) -- fluid part weighted 1 - B, solid part (Eq. 12 summed over the
// covering particles) by B -- and store of the post-collision populations.  IMB = false
// compiles the fluid node alone (B = 0); FORCED adds the Guo forcing term.  The solid part
// is written without branches (B = 0 leaves the fluid update unchanged) and takes each
// direction together with its opposite, whose terms differ only in sign.
template <typename S, bool IMB, bool FORCED>
__device__ __forceinline__ void node_collide_store(const float (&d)[9], const NodeState &c,
                                                   const SolidMoments &sm, S *__restrict__ outp,
                                                   const LatticeArgs &a) {
    float upd[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) upd[q] = -c.omega * c.n[q];
    if (FORCED) {  // Guo forcing term
        const float sf = 1.0f - 0.5f * c.omega;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float cxq = (float)cx_of(q), cyq = (float)cy_of(q);
            const float cu = cdot(q, c.ux, c.uy);
            const float S_q = w_of(q) * (3.0f * ((cxq - c.ux) * a.Fx + (cyq - c.uy) * a.Fy) +
                                         9.0f * cu * cdot(q, a.Fx, a.Fy));
            upd[q] = fmaf(sf, S_q, upd[q]);
        }
    }
    if (IMB) {
        const float B = sm.B;
        const float fl = 1.0f - B;
        // sum_p B_p Omega^s_p = B (n_{-q} - n_q) + sum_p B_p (f^eq_q(u_s,p) - f^eq_q(u)), with
        // sum_p B_p f^eq_q(u_s,p) - B f^eq_q(u) = rho w_q (3 c.A1 + 4.5 c.A2.c - 1.5 tr A2)
        const float a1x = sm.m1x - B * c.ux, a1y = sm.m1y - B * c.uy;
        const float a2xx = sm.m2xx - B * c.ux * c.ux, a2yy = sm.m2yy - B * c.uy * c.uy;
        const float a2xy = sm.m2xy - B * c.ux * c.uy;
        const float tra2 = a2xx + a2yy;
        upd[0] = fmaf(fl, upd[0], c.rho * w_of(0) * (-1.5f * tra2));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = k < 2 ? k + 1 : k + 3, o = opp_of(q);   // q = 1, 2, 5, 6
            const float rw = c.rho * w_of(q);
            const float t1 = 3.0f * cdot(q, a1x, a1y);
            const float t2 = 4.5f * ccdot(q, a2xx, a2yy, a2xy) - 1.5f * tra2;
            const float bd = B * (c.n[o] - c.n[q]);
            upd[q] = fmaf(fl, upd[q], bd) + rw * (t2 + t1);
            upd[o] = fmaf(fl, upd[o], -bd) + rw * (t2 - t1);
        }
    }
    S *p = outp;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        Store<S>::st(p, d[q] + upd[q]);
        p += a.plane;
    }
}

}  // namespace imb
