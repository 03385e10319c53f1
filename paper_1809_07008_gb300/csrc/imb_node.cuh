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

// The eight moving directions as four pairs (q, -q), q = 1, 2, 5, 6: their equilibria share
// the even part w (drho + rho (4.5 (c.u)^2 - 1.5 u^2)) and differ in the sign of the odd part
// 3 w rho c.u, so a pair is computed with FP32x2 instructions (two lanes of arithmetic per
// instruction) where the operations line up.
__host__ __device__ constexpr int pair_q(int k) { return k < 2 ? k + 1 : k + 3; }

__device__ __forceinline__ void node_state(const float (&d)[9], const LatticeArgs &a, const bool forced,
                                           const bool smag, NodeState &c) {
    float2 P[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) P[k] = make_float2(d[pair_q(k)], d[opp_of(pair_q(k))]);
    // ---- moments (Eqs. 3-4, Guo half-force shift)
    const float2 S = __fadd2_rn(__fadd2_rn(P[0], P[1]), __fadd2_rn(P[2], P[3]));
    c.drho = d[0] + (S.x + S.y);
    c.rho = 1.0f + c.drho;
    float D[4];   // d_q - d_-q
#pragma unroll
    for (int k = 0; k < 4; ++k) D[k] = P[k].x - P[k].y;
    c.jx = (D[0] + D[2]) - D[3];   // c_x: +1 for q = 1, 5, -1 for q = 6
    c.jy = (D[1] + D[2]) + D[3];   // c_y: +1 for q = 2, 5, 6
    if (forced) {
        c.jx = fmaf(0.5f, a.Fx, c.jx);
        c.jy = fmaf(0.5f, a.Fy, c.jy);
    }
    const float inv = __fdividef(1.0f, c.rho);
    c.ux = c.jx * inv;
    c.uy = c.jy * inv;
    c.usq = c.ux * c.ux + c.uy * c.uy;
    // ---- non-equilibrium parts (Eq. 2)
    const float m15 = -1.5f * c.usq;
    c.n[0] = d[0] - w_of(0) * fmaf(c.rho, m15, c.drho);
    float2 N[4];
    const float2 rho2 = make_float2(c.rho, c.rho), drho2 = make_float2(c.drho, c.drho);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // n_{+-q} = d_{+-q} - w_q (drho + rho (4.5 (c.u)^2 - 1.5 u^2 +- 3 c.u)), each rounded once
        const int q = pair_q(k);
        const float cu = cdot(q, c.ux, c.uy);
        const float e = fmaf(4.5f * cu, cu, m15), o3 = 3.0f * cu;
        const float2 X = __ffma2_rn(rho2, make_float2(e + o3, e - o3), drho2);
        N[k] = __ffma2_rn(make_float2(-w_of(q), -w_of(q)), X, P[k]);
        c.n[q] = N[k].x;
        c.n[opp_of(q)] = N[k].y;
    }
    // ---- Smagorinsky effective relaxation time (Hou et al. 1996 closure)
    c.omega = a.omega0;
    c.te = a.tau;
    if (smag) {
        const float2 E = __fadd2_rn(N[2], N[3]);                                // (n5 + n6, n7 + n8)
        const float2 F = __fadd2_rn(N[2], make_float2(-N[3].x, -N[3].y));       // (n5 - n6, n7 - n8)
        const float e = E.x + E.y;
        const float pxx = (N[0].x + N[0].y) + e;
        const float pyy = (N[1].x + N[1].y) + e;
        const float pxy = F.x + F.y;
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
    float upd0 = -c.omega * c.n[0];
    float2 U[4];   // updates of the pairs (q, -q)
    const float2 mo = make_float2(-c.omega, -c.omega);
    if (IMB || FORCED) {
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = __fmul2_rn(mo, make_float2(c.n[pair_q(k)], c.n[opp_of(pair_q(k))]));
    }
    if (FORCED) {  // Guo forcing term
        const float sf = 1.0f - 0.5f * c.omega;
        upd0 = fmaf(sf, w_of(0) * 3.0f * (-c.ux * a.Fx - c.uy * a.Fy), upd0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = pair_q(k), o = opp_of(q);
            float S2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int qq = h ? o : q;
                const float cxq = (float)cx_of(qq), cyq = (float)cy_of(qq);
                const float cu = cdot(qq, c.ux, c.uy);
                S2[h] = w_of(qq) * (3.0f * ((cxq - c.ux) * a.Fx + (cyq - c.uy) * a.Fy) + 9.0f * cu * cdot(qq, a.Fx, a.Fy));
            }
            U[k] = __ffma2_rn(make_float2(sf, sf), make_float2(S2[0], S2[1]), U[k]);
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
        upd0 = fmaf(fl, upd0, c.rho * w_of(0) * (-1.5f * tra2));
        const float2 fl2 = make_float2(fl, fl);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = pair_q(k), o = opp_of(q);
            const float rw = c.rho * w_of(q);
            const float t1 = 3.0f * cdot(q, a1x, a1y);
            const float t2 = 4.5f * ccdot(q, a2xx, a2yy, a2xy) - 1.5f * tra2;
            const float bd = B * (c.n[o] - c.n[q]);
            U[k] = __ffma2_rn(fl2, U[k], make_float2(bd, -bd));
            U[k] = __ffma2_rn(make_float2(rw, rw), make_float2(t2 + t1, t2 - t1), U[k]);
        }
    }
    Store<S>::st(outp, d[0] + upd0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = pair_q(k), o = opp_of(q);
        const float2 P = make_float2(d[q], d[o]);
        // a fluid node in one rounding: d - omega n (+ the forcing term)
        const float2 out = (IMB || FORCED) ? __fadd2_rn(P, U[k])
                                           : __ffma2_rn(mo, make_float2(c.n[q], c.n[o]), P);
        Store<S>::st(outp + (size_t)q * a.plane, out.x);
        Store<S>::st(outp + (size_t)o * a.plane, out.y);
    }
}

}  // namespace imb
