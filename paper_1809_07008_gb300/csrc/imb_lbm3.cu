// imb_lbm3.cu -- the paper's own lattice: D3Q19 stream-collide with held spheres.
//
// Sec. 2.1 (Tab. 1) lattice, BGK with Guo forcing (Eqs. 1-5), the partially saturated
// collision of Eqs. 12-14 with the solid ratio of each cell counted on its n_sub^3 sub-cells
// (Sec. 2.3), and per-sphere force and torque (Eqs. 15-16).  Spheres are held in place; their
// velocity and spin enter u_s.  One thread per cell, warps along x rows: a pull of the 19
// planes (x and z periodic, y periodic or halfway bounce-back walls), the collision in
// registers, the store, and the sphere's force summed over the warp before one FP64
// atomicAdd per component; each thread walks a short column of cells along z, the loads of
// the next cell in flight during the arithmetic of the current one.  A cell may be covered by
// two spheres (packed beds whose spheres touch): two per-cell map words hold the spheres and
// their sub-cell counts, and B is shared between them by their solid ratios; a third sphere on
// one cell raises IMB_E_OVERFLOW.  With C_smag > 0 every cell relaxes with its Smagorinsky
// relaxation time, in the BGK term, the forcing and B.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/imblbm.h"
#include "imb_device.cuh"

namespace imb3 {

using imb::Store;

// D3Q19 (Tab. 1): 0 rest; 1-6 faces (+x, -x, +y, -y, +z, -z); 7-18 edges in opposite pairs
__host__ __device__ constexpr int cx3(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
           : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy3(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
           : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz3(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
           : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp3(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

// c_q . (a, b, c) with the zero components of c_q left out (under IEEE rules the compiler may
// not drop a product with 0, and these dot products run for every direction of every node)
__device__ __forceinline__ float cdot3(int q, float a, float b, float c) {
    const int x = cx3(q), y = cy3(q), z = cz3(q);
    const float ta = x > 0 ? a : -a, tb = y > 0 ? b : -b, tc = z > 0 ? c : -c;
    if (x == 0 && y == 0 && z == 0) return 0.0f;
    if (y == 0 && z == 0) return ta;
    if (x == 0 && z == 0) return tb;
    if (x == 0 && y == 0) return tc;
    if (z == 0) return ta + tb;
    if (y == 0) return ta + tc;
    return tb + tc;
}
__host__ __device__ constexpr float w3(int q) { return q == 0 ? 1.0f / 3.0f : (q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f); }

constexpr unsigned ID_BITS = 22, ID_MASK = (1u << ID_BITS) - 1u;   // map word: sphere + 1 | count << 22
constexpr unsigned ERR_UNSTABLE = imb::ERR_UNSTABLE, ERR_OVERLAP = imb::ERR_CELL_SLOTS;

struct Args3 {
    int nx, ny, nz, wall_y;
    size_t plane;            // cells
    float tau, omega, Fx, Fy, Fz;
    float inv_nsub3;         // 1 / n_sub^3
    int n_sub;
    float uw_bot, uw_top;    // x velocity of the walls y = 0 and y = ny
    float smag_coef;         // 18 sqrt(2) C^2 (0: plain BGK)
    int two_slots;           // 1 once some cell holds a second sphere
    long long off[19];       // element offset of the source of direction q: q plane - c_q (interior)
};

// sphere as the stream-collide kernel reads it: centre cell and FP32 offset in it, v, spin
struct __align__(16) Sph3 {
    int ci, cj, ck, pad;
    float fx, fy, fz, pad2;
    float vx, vy, vz, pad3;
    float wx, wy, wz, pad4;
};

__device__ __forceinline__ int wrap(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }
__device__ __forceinline__ int min_image(int d, int L) {
    const int h = L / 2;
    return d >= h ? d - L : (d < -h ? d + L : d);
}

// Sec. 2.3: sub-cell centres of cell offset (di, dj, dk) inside the sphere; every FP64
// operation rounded on its own, in the order of the plain definition
__device__ int subcell_count(int di, int dj, int dk, double fx, double fy, double fz, double R, int n) {
    const double R2 = __dmul_rn(R, R);
    const double dn = (double)n;
    int cnt = 0;
    for (int c = 0; c < n; ++c) {
        const double dz = __dsub_rn(__dadd_rn((double)dk, __ddiv_rn(__dadd_rn((double)c, 0.5), dn)), fz);
        for (int b = 0; b < n; ++b) {
            const double dy = __dsub_rn(__dadd_rn((double)dj, __ddiv_rn(__dadd_rn((double)b, 0.5), dn)), fy);
            for (int a = 0; a < n; ++a) {
                const double dx = __dsub_rn(__dadd_rn((double)di, __ddiv_rn(__dadd_rn((double)a, 0.5), dn)), fx);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 <= R2) ++cnt;
            }
        }
    }
    return cnt;
}

// one thread per (sphere, cell of its bounding box of half-width `span`); the first sphere on a
// cell takes map, the second map2 (and sets shared), a third raises the overlap bit.  Slots
// are filled in whatever order the threads arrive: readers order them by sphere
__global__ void k3_map(const double *__restrict__ xyz, const double *__restrict__ R, int n, int span, Args3 a,
                       unsigned *map, unsigned *map2, unsigned *shared, unsigned *err) {
    const int w = 2 * span + 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * w * w * w) return;
    const int s = (int)(t / ((long long)w * w * w));
    int c = (int)(t % ((long long)w * w * w));
    const int di = c % w - span;
    c /= w;
    const int dj = c % w - span, dk = c / w - span;
    const double cx = xyz[3 * s], cy = xyz[3 * s + 1], cz = xyz[3 * s + 2];
    const double fi = floor(cx), fj = floor(cy), fk = floor(cz);
    const int ci = (int)fi, cj = (int)fj, ck = (int)fk;
    int i = ci + di, j = cj + dj, k = ck + dk;
    i = ((i % a.nx) + a.nx) % a.nx;
    k = ((k % a.nz) + a.nz) % a.nz;
    if (a.wall_y) {
        if (j < 0 || j >= a.ny) return;
    } else {
        j = ((j % a.ny) + a.ny) % a.ny;
    }
    const int cnt = subcell_count(di, dj, dk, cx - fi, cy - fj, cz - fk, R[s], a.n_sub);
    if (cnt == 0) return;
    const unsigned word = (unsigned)(s + 1) | ((unsigned)cnt << ID_BITS);
    const size_t cell = ((size_t)k * a.ny + j) * a.nx + i;
    if (atomicCAS(&map[cell], 0u, word) == 0u) return;
    if (atomicCAS(&map2[cell], 0u, word) == 0u) atomicOr(shared, 1u);
    else atomicOr(err, ERR_OVERLAP);
}

template <typename S>
__global__ void k3_init(S *f, size_t plane, float rho0, float ux, float uy, float uz) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= plane) return;
    const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float cu = cx3(q) * ux + cy3(q) * uy + cz3(q) * uz;
        Store<S>::st(f + (size_t)q * plane + c, w3(q) * (rho0 * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu) - 1.0f));
    }
}

// f(x, t) at one cell: the pull of the post-collision field with the boundary rules
template <typename S>
__device__ __forceinline__ void pull3(const S *__restrict__ fin, const Args3 &a, int x, int y, int z, float (&d)[19]) {
    const size_t cell = ((size_t)z * a.ny + y) * a.nx + x;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        int ys = y - cy3(q);
        if (a.wall_y && (ys < 0 || ys >= a.ny)) {   // halfway bounce-back: the cell's own opposite
            d[q] = Store<S>::ld(fin + (size_t)opp3(q) * a.plane + cell);
            if (cx3(q) != 0) d[q] += 6.0f * w3(q) * (float)cx3(q) * (ys < 0 ? a.uw_bot : a.uw_top);
            continue;
        }
        ys = wrap(ys, a.ny);
        const int xs = wrap(x - cx3(q), a.nx), zs = wrap(z - cz3(q), a.nz);
        d[q] = Store<S>::ld(fin + (size_t)q * a.plane + ((size_t)zs * a.ny + ys) * a.nx + xs);
    }
}

template <typename S> __device__ __forceinline__ S ld_raw3(const S *p) { return __ldg(p); }
__device__ __forceinline__ float f32_of(float v) { return v; }
__device__ __forceinline__ float f32_of(__half v) { return __half2float(v); }
__device__ __forceinline__ float f32_of(__nv_bfloat16 v) { return __bfloat162float(v); }

// the 19 stored values a cell pulls (Eq. 1), as stored: interior cells by the per-direction
// offsets, edge cells with the wrap and wall rules
template <typename S>
__device__ __forceinline__ void fetch3(const S *__restrict__ fin, const Args3 &a, int x, int y, int z, S (&r)[19]) {
    const size_t cell = ((size_t)z * a.ny + y) * a.nx + x;
    if (x > 0 && x < a.nx - 1 && y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1) {
#pragma unroll
        for (int q = 0; q < 19; ++q) r[q] = ld_raw3(fin + (cell + a.off[q]));
        return;
    }
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        int ys = y - cy3(q);
        if (a.wall_y && (ys < 0 || ys >= a.ny)) {   // halfway bounce-back: the cell's own opposite
            r[q] = ld_raw3(fin + (size_t)opp3(q) * a.plane + cell);
            continue;
        }
        ys = wrap(ys, a.ny);
        const int xs = wrap(x - cx3(q), a.nx), zs = wrap(z - cz3(q), a.nz);
        r[q] = ld_raw3(fin + (size_t)q * a.plane + ((size_t)zs * a.ny + ys) * a.nx + xs);
    }
}

// u_s = v + w x r at the node of cell (x, y, z), r from the sphere's centre (minimum image)
__device__ __forceinline__ void surface_velocity(const Sph3 &P, const Args3 &a, int x, int y, int z, float (&r)[3],
                                                 float (&us)[3]) {
    r[0] = (float)min_image(x - P.ci, a.nx) + 0.5f - P.fx;
    r[1] = (float)(a.wall_y ? y - P.cj : min_image(y - P.cj, a.ny)) + 0.5f - P.fy;
    r[2] = (float)min_image(z - P.ck, a.nz) + 0.5f - P.fz;
    us[0] = P.vx + (P.wy * r[2] - P.wz * r[1]);
    us[1] = P.vy + (P.wz * r[0] - P.wx * r[2]);
    us[2] = P.vz + (P.wx * r[1] - P.wy * r[0]);
}

// Eqs. 15-16 for one sphere: force B_p (rho u - rho u_s - F), torque r x force
__device__ __forceinline__ void sphere_force(float Bp, float rho, float jx, float jy, float jz, const float (&us)[3],
                                             const float (&r)[3], const Args3 &a, float (&fo)[6]) {
    fo[0] = Bp * (jx - rho * us[0] - a.Fx);
    fo[1] = Bp * (jy - rho * us[1] - a.Fy);
    fo[2] = Bp * (jz - rho * us[2] - a.Fz);
    fo[3] = r[1] * fo[2] - r[2] * fo[1];
    fo[4] = r[2] * fo[0] - r[0] * fo[2];
    fo[5] = r[0] * fo[1] - r[1] * fo[0];
}

// the plain variant of collide3_gen below (one sphere per cell, tau fixed), written out on its
// own: folding the general function down to this case compiled to a 3 % slower FP32 kernel
template <typename S>
__device__ __forceinline__ int collide3_plain(const float (&d)[19], const Args3 &a, int x, int y, int z, size_t cell,
                                        const unsigned *__restrict__ map, const Sph3 *__restrict__ sph,
                                        S *__restrict__ fout, float (&fo)[6], bool &unstable) {
    // the 18 moving directions as nine pairs (q, q + 1) = (q, -q), q odd, computed with FP32x2
    // instructions: their terms differ only in the sign of the odd parts
    float2 P[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) P[k] = make_float2(d[2 * k + 1], d[2 * k + 2]);
    float2 Sp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Sp[k] = P[k];
#pragma unroll
    for (int h = 1; h < 9; h <<= 1)
#pragma unroll
        for (int k = 0; k + h < 9; k += 2 * h) Sp[k] = __fadd2_rn(Sp[k], Sp[k + h]);
    const float drho = d[0] + (Sp[0].x + Sp[0].y);
    float mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {   // c_{-q} = -c_q: first moments from d_q - d_-q
        const int q = 2 * k + 1;
        const float Dk = P[k].x - P[k].y;
        if (cx3(q)) mx += cx3(q) * Dk;
        if (cy3(q)) my += cy3(q) * Dk;
        if (cz3(q)) mz += cz3(q) * Dk;
    }
    const float rho = 1.0f + drho;
    const float jx = fmaf(0.5f, a.Fx, mx), jy = fmaf(0.5f, a.Fy, my), jz = fmaf(0.5f, a.Fz, mz);
    const float inv = __fdividef(1.0f, rho);
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(uu < 0.09f)) unstable = true;   // Mach guard, also catches NaN
    const float t = fmaf(-1.5f * rho, uu, drho);
    const float2 t2 = make_float2(t, t);
    // non-equilibrium parts (Eq. 2), shifted by w: n_{+-q} = d_{+-q} - w_q (t +- rho c.u (3 +- 4.5 c.u))
    const float n0 = d[0] - w3(0) * t;
    float2 N[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        const float cu = cdot3(q, ux, uy, uz), rcu = rho * cu;
        const float2 X = __ffma2_rn(make_float2(rcu, -rcu), make_float2(fmaf(4.5f, cu, 3.0f), fmaf(-4.5f, cu, 3.0f)), t2);
        N[k] = __ffma2_rn(make_float2(-w3(q), -w3(q)), X, P[k]);
    }
    const unsigned word = map[cell];
    int sid = -1;
    float B = 0.0f, usx = 0.0f, usy = 0.0f, usz = 0.0f, rx = 0.0f, ry = 0.0f, rz = 0.0f;
    if (word) {   // Eq. 14 with the sub-cell solid ratio; u_s = v + w x r at the node
        sid = (int)(word & ID_MASK) - 1;
        const float eps = (float)(word >> ID_BITS) * a.inv_nsub3;
        const float tm = a.tau - 0.5f;
        B = __fdividef(eps * tm, (1.0f - eps) + tm);
        const Sph3 Ps = sph[sid];
        rx = (float)min_image(x - Ps.ci, a.nx) + 0.5f - Ps.fx;
        ry = (float)(a.wall_y ? y - Ps.cj : min_image(y - Ps.cj, a.ny)) + 0.5f - Ps.fy;
        rz = (float)min_image(z - Ps.ck, a.nz) + 0.5f - Ps.fz;
        usx = Ps.vx + (Ps.wy * rz - Ps.wz * ry);
        usy = Ps.vy + (Ps.wz * rx - Ps.wx * rz);
        usz = Ps.vz + (Ps.wx * ry - Ps.wy * rx);
    }
    const float fl = 1.0f - B, sf = 1.0f - 0.5f * a.omega;
    const float uF = ux * a.Fx + uy * a.Fy + uz * a.Fz;
    // BGK with Guo forcing (its source divided by 1 - 1/(2 tau)), weighted by 1 - B:
    // -omega n_q + sf w_q (3 (c_q.F - u.F) + 9 (c_q.u)(c_q.F)), for the pair (q, -q)
    const float f0 = fmaf(-a.omega, n0, sf * (w3(0) * (-3.0f * uF)));
    const float2 mo2 = make_float2(-a.omega, -a.omega), muF2 = make_float2(-uF, -uF);
    auto fluid2 = [&](int k) {
        const int q = 2 * k + 1;
        const float cu = cdot3(q, ux, uy, uz), cF = cdot3(q, a.Fx, a.Fy, a.Fz);
        const float e9 = 9.0f * cu * cF;
        const float2 A = __fadd2_rn(make_float2(cF, -cF), muF2);
        const float2 G = __ffma2_rn(make_float2(3.0f, 3.0f), A, make_float2(e9, e9));
        const float sw = sf * w3(q);
        return __ffma2_rn(mo2, N[k], __fmul2_rn(make_float2(sw, sw), G));
    };
    if (word) {   // Eq. 12 in shifted form: n_{-q} + (f^eq_q(u_s) - w_q) - d_q, weighted by B
        const float uss = usx * usx + usy * usy + usz * usz;
        const float ts = fmaf(-1.5f * rho, uss, drho);
        const float2 ts2 = make_float2(ts, ts), B2 = make_float2(B, B), fl2 = make_float2(fl, fl);
        Store<S>::st(fout + cell, d[0] + fmaf(B, n0 + w3(0) * ts - d[0], fl * f0));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int q = 2 * k + 1;
            const float cs = cdot3(q, usx, usy, usz), rcs = rho * cs;
            const float2 Xs = __ffma2_rn(make_float2(rcs, -rcs), make_float2(fmaf(4.5f, cs, 3.0f), fmaf(-4.5f, cs, 3.0f)), ts2);
            // n_{-q} + w_q Xs - d_q for q and -q
            const float2 T = __fadd2_rn(__ffma2_rn(make_float2(w3(q), w3(q)), Xs, make_float2(N[k].y, N[k].x)),
                                        make_float2(-P[k].x, -P[k].y));
            const float2 v = __ffma2_rn(B2, T, __fmul2_rn(fl2, fluid2(k)));
            const float2 o = __fadd2_rn(P[k], v);
            Store<S>::st(fout + (size_t)q * a.plane + cell, o.x);
            Store<S>::st(fout + (size_t)(q + 1) * a.plane + cell, o.y);
        }
    } else {      // no sphere: the fluid operator alone
        Store<S>::st(fout + cell, d[0] + f0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int q = 2 * k + 1;
            const float2 o = __fadd2_rn(P[k], fluid2(k));
            Store<S>::st(fout + (size_t)q * a.plane + cell, o.x);
            Store<S>::st(fout + (size_t)(q + 1) * a.plane + cell, o.y);
        }
    }
    if (word) {   // Eqs. 15-16: force on the sphere B (rho u - rho u_s - F), torque r x force
        fo[0] = B * (jx - rho * usx - a.Fx);
        fo[1] = B * (jy - rho * usy - a.Fy);
        fo[2] = B * (jz - rho * usz - a.Fz);
        fo[3] = ry * fo[2] - rz * fo[1];
        fo[4] = rz * fo[0] - rx * fo[2];
        fo[5] = rx * fo[1] - ry * fo[0];
    }
    return sid;
}

// collision of one cell from its pulled values d, general variant: moments (Eqs. 3-4, Guo
// half-force shift), the Smagorinsky relaxation time (when smag_coef > 0), BGK with Guo
// forcing, Eqs. 12-14 where one or two spheres cover the cell, the 19 stores; returns the
// covering sphere of lower index (-1: none) with its force and torque contribution in fo
// (Eqs. 15-16); a second covering sphere's share goes to FT directly.  The kernel runs it
// only when some cell holds two spheres or C_smag > 0: its code in every cell's schedule
// slowed the plain case by 9-13 %
template <typename S>
__device__ __forceinline__ int collide3_gen(const float (&d)[19], const Args3 &a, int x, int y, int z, size_t cell,
                                        const unsigned *__restrict__ map, const unsigned *__restrict__ map2,
                                        const Sph3 *__restrict__ sph, S *__restrict__ fout, double *FT,
                                        float (&fo)[6], bool &unstable) {
    float drho = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += d[q];
        if (cx3(q)) mx += cx3(q) * d[q];
        if (cy3(q)) my += cy3(q) * d[q];
        if (cz3(q)) mz += cz3(q) * d[q];
    }
    const float rho = 1.0f + drho;
    const float jx = fmaf(0.5f, a.Fx, mx), jy = fmaf(0.5f, a.Fy, my), jz = fmaf(0.5f, a.Fz, mz);
    const float inv = __fdividef(1.0f, rho);
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(uu < 0.09f)) unstable = true;   // Mach guard, also catches NaN
    const float t = fmaf(-1.5f * rho, uu, drho);
    float n[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {   // non-equilibrium parts (Eq. 2), shifted by w
        const float cu = cdot3(q, ux, uy, uz);
        n[q] = d[q] - w3(q) * fmaf(rho * cu, fmaf(4.5f, cu, 3.0f), t);
    }
    float te = a.tau, omega = a.omega;
    if (a.smag_coef > 0.0f) {   // tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 sqrt(Pi : Pi) / rho)) / 2
        float pxx = 0.0f, pyy = 0.0f, pzz = 0.0f, pxy = 0.0f, pxz = 0.0f, pyz = 0.0f;
#pragma unroll
        for (int q = 1; q < 19; ++q) {   // Pi = sum_q c_q c_q n_q
            if (cx3(q)) pxx += n[q];
            if (cy3(q)) pyy += n[q];
            if (cz3(q)) pzz += n[q];
            if (cx3(q) && cy3(q)) pxy += cx3(q) * cy3(q) > 0 ? n[q] : -n[q];
            if (cx3(q) && cz3(q)) pxz += cx3(q) * cz3(q) > 0 ? n[q] : -n[q];
            if (cy3(q) && cz3(q)) pyz += cy3(q) * cz3(q) > 0 ? n[q] : -n[q];
        }
        const float Q = fmaf(pxx, pxx, fmaf(pyy, pyy, pzz * pzz)) + 2.0f * fmaf(pxy, pxy, fmaf(pxz, pxz, pyz * pyz));
        const float sq = Q > 0.0f ? Q * rsqrtf(Q) : 0.0f;   // sqrt(Q)
        const float disc = fmaf(a.smag_coef * sq, inv, a.tau * a.tau);
        te = 0.5f * (a.tau + disc * rsqrtf(disc));
        omega = __fdividef(1.0f, te);
    }
    unsigned w1 = map[cell], w2 = 0u;
    if (w1 && a.two_slots) {
        w2 = map2[cell];
        if (w2 && (w2 & ID_MASK) < (w1 & ID_MASK)) {   // the sphere of lower index first
            const unsigned tw = w1;
            w1 = w2;
            w2 = tw;
        }
    }
    int sid = -1;
    float B = 0.0f, B1 = 0.0f, B2 = 0.0f;
    float r1[3] = {0.0f, 0.0f, 0.0f}, u1[3] = {0.0f, 0.0f, 0.0f}, r2[3] = {0.0f, 0.0f, 0.0f}, u2[3] = {0.0f, 0.0f, 0.0f};
    if (w1) {   // Eq. 14 with the summed sub-cell solid ratio, shared by the spheres' own ratios
        sid = (int)(w1 & ID_MASK) - 1;
        const unsigned c1 = w1 >> ID_BITS, c2 = w2 >> ID_BITS;
        const float eps = fminf(1.0f, (float)(c1 + c2) * a.inv_nsub3);   // two spheres may overlap
        const float tm = te - 0.5f;
        B = __fdividef(eps * tm, (1.0f - eps) + tm);
        B1 = B;
        surface_velocity(sph[sid], a, x, y, z, r1, u1);
        if (w2) {
            const float inv_c = __fdividef(1.0f, (float)(c1 + c2));
            B1 = B * ((float)c1 * inv_c);
            B2 = B * ((float)c2 * inv_c);
            surface_velocity(sph[(w2 & ID_MASK) - 1], a, x, y, z, r2, u2);
        }
    }
    const float fl = 1.0f - B, sf = 1.0f - 0.5f * omega;
    const float uF = ux * a.Fx + uy * a.Fy + uz * a.Fz;
    // BGK with Guo forcing (its source divided by 1 - 1/(2 tau)), weighted by 1 - B
    auto fluid = [&](int q) {
        const float cu = cdot3(q, ux, uy, uz);
        const float cF = cdot3(q, a.Fx, a.Fy, a.Fz);
        const float Sg = w3(q) * (3.0f * (cF - uF) + 9.0f * cu * cF);
        return fmaf(-omega, n[q], sf * Sg);
    };
    // f^eq_q(rho, u_s) - w_q
    auto eq_solid = [&](int q, const float (&us)[3], float ts) {
        const float cs = cdot3(q, us[0], us[1], us[2]);
        return w3(q) * fmaf(rho * cs, fmaf(4.5f, cs, 3.0f), ts);
    };
    if (w2) {     // Eq. 12 summed over both spheres: B (n_{-q} - d_q) + sum_p B_p (f^eq_q(u_s,p) - w_q)
        const float ts1 = fmaf(-1.5f * rho, u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2], drho);
        const float ts2 = fmaf(-1.5f * rho, u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2], drho);
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const float v = fmaf(B, n[opp3(q)] - d[q], fl * fluid(q)) + fmaf(B1, eq_solid(q, u1, ts1), B2 * eq_solid(q, u2, ts2));
            Store<S>::st(fout + (size_t)q * a.plane + cell, d[q] + v);
        }
    } else if (w1) {   // Eq. 12 in shifted form: n_{-q} + (f^eq_q(u_s) - w_q) - d_q, weighted by B
        const float ts = fmaf(-1.5f * rho, u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2], drho);
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const float v = fmaf(B, n[opp3(q)] + eq_solid(q, u1, ts) - d[q], fl * fluid(q));
            Store<S>::st(fout + (size_t)q * a.plane + cell, d[q] + v);
        }
    } else {      // no sphere: the fluid operator alone
#pragma unroll
        for (int q = 0; q < 19; ++q) Store<S>::st(fout + (size_t)q * a.plane + cell, d[q] + fluid(q));
    }
    if (w1) sphere_force(B1, rho, jx, jy, jz, u1, r1, a, fo);
    if (w2) {     // the second sphere's share, summed straight into its totals
        float f2[6];
        sphere_force(B2, rho, jx, jy, jz, u2, r2, a, f2);
        const int s2 = (int)(w2 & ID_MASK) - 1;
#pragma unroll
        for (int c = 0; c < 6; ++c) atomicAdd(&FT[6 * s2 + c], (double)f2[c]);
    }
    return sid;
}

// stream-collide; blocks of 32 x 8 cells, each thread a column of ZC cells along z whose next
// cell's loads are issued before the current cell's arithmetic
constexpr int ZC = 8;

template <bool GEN, typename S>
__global__ void __launch_bounds__(256, 2) k3_stream_collide(const S *__restrict__ fin, S *__restrict__ fout, const Args3 a,
                                                         const unsigned *__restrict__ map,
                                                         const unsigned *__restrict__ map2,
                                                         const Sph3 *__restrict__ sph, double *FT, unsigned *err) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, a.nz);
    const int lane = threadIdx.x;
    const bool in = x < a.nx && y < a.ny;
    bool unstable = false;
    S r[19];
    if (in) fetch3(fin, a, x, y, z0, r);
    for (int z = z0; z < z1; ++z) {
        int sid = -1;
        float fo[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (in) {
            float d[19];
#pragma unroll
            for (int q = 0; q < 19; ++q) d[q] = f32_of(r[q]);
            if (a.wall_y && (y == 0 || y == a.ny - 1)) {   // moving-wall term of the bounced values
#pragma unroll
                for (int q = 0; q < 19; ++q)
                    if (cx3(q) != 0 && ((y == 0 && cy3(q) == 1) || (y == a.ny - 1 && cy3(q) == -1)))
                        d[q] += 6.0f * w3(q) * (float)cx3(q) * (y == 0 ? a.uw_bot : a.uw_top);
            }
            if (z + 1 < z1) fetch3(fin, a, x, y, z + 1, r);   // in flight during this cell's arithmetic
            const size_t cell = ((size_t)z * a.ny + y) * a.nx + x;
            if constexpr (GEN)
                sid = collide3_gen(d, a, x, y, z, cell, map, map2, sph, fout, FT, fo, unstable);
            else
                sid = collide3_plain(d, a, x, y, z, cell, map, sph, fout, fo, unstable);
        }
        // the warp's force: lanes of its first sphere summed by shuffles, any other sphere direct
        const unsigned has = __ballot_sync(0xffffffffu, sid >= 0);
        if (has) {
            const int lead = __shfl_sync(0xffffffffu, sid, __ffs(has) - 1);
            const bool mine = sid == lead;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                float v = mine ? fo[c] : 0.0f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) atomicAdd(&FT[6 * lead + c], (double)v);
                if (sid >= 0 && !mine) atomicAdd(&FT[6 * sid + c], (double)fo[c]);
            }
        }
    }
    if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(err, ERR_UNSTABLE);
}

// f(x, t) = w + pulled deviation, FP64, [19][cells]
template <typename S>
__global__ void k3_gather(const S *__restrict__ fin, const Args3 a, double *out) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.plane) return;
    const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny), z = (int)(c / ((size_t)a.nx * a.ny));
    float d[19];
    pull3(fin, a, x, y, z, d);
#pragma unroll
    for (int q = 0; q < 19; ++q) out[(size_t)q * a.plane + c] = (double)w3(q) + (double)d[q];
}

// rho and u (with the half-force shift) of f(x, t)
template <typename S>
__global__ void k3_macro(const S *__restrict__ fin, const Args3 a, double *rho, double *ux, double *uy, double *uz) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.plane) return;
    const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny), z = (int)(c / ((size_t)a.nx * a.ny));
    float d[19];
    pull3(fin, a, x, y, z, d);
    double r = 1.0, m[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        r += d[q];
        m[0] += cx3(q) * (double)d[q];
        m[1] += cy3(q) * (double)d[q];
        m[2] += cz3(q) * (double)d[q];
    }
    rho[c] = r;
    ux[c] = (m[0] + 0.5 * a.Fx) / r;
    uy[c] = (m[1] + 0.5 * a.Fy) / r;
    uz[c] = (m[2] + 0.5 * a.Fz) / r;
}

}  // namespace imb3

using namespace imb3;

struct imb3_ctx {
    int device = 0, nx = 0, ny = 0, nz = 0, np = 0, elem = 4, cur = 0;
    double tau = 0.0;
    imb3_params p{};
    Args3 a{};
    void *buf[2] = {nullptr, nullptr};
    unsigned *map = nullptr, *map2 = nullptr, *h_err = nullptr;
    unsigned *err = nullptr;   // [0] error bits, [1] set by the cell map when a cell holds two spheres
    Sph3 *sph = nullptr;
    double *FT = nullptr;
    cudaStream_t stream = nullptr;
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    long long launches = 0;
    std::string msg;
};

namespace {

std::string g3_err;

int fail3(imb3_ctx *c, int code, const std::string &m) {
    if (c) c->msg = m;
    else g3_err = m;
    return code;
}

#define CK3(call, what)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail3(c, e_ == cudaErrorMemoryAllocation ? IMB_E_NOMEM : IMB_E_CUDA,            \
                         std::string(what) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

template <typename F>
cudaError_t by_storage3(int storage, F &&fn) {
    switch (storage) {
    case IMB_STORE_FP32: return fn((float *)nullptr);
    case IMB_STORE_FP16: return fn((__half *)nullptr);
    case IMB_STORE_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

// wait for the stream with a deadline, then read and clear the device error bits
int wait3(imb3_ctx *c) {
    cudaEvent_t ev;
    CK3(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    CK3(cudaMemcpyAsync(c->h_err, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "error word");
    CK3(cudaEventRecord(ev, c->stream), "event record");
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t q;
    while ((q = cudaEventQuery(ev)) == cudaErrorNotReady) {
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > c->p.timeout_ms) {
            cudaEventDestroy(ev);
            return fail3(c, IMB_E_TIMEOUT, "stream did not finish within timeout_ms");
        }
        if (ms > 2.0) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    cudaEventDestroy(ev);
    CK3(q, "stream");
    const unsigned bits = *c->h_err;
    if (bits) {
        CK3(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream), "clear");
        CK3(cudaStreamSynchronize(c->stream), "clear");
        if (bits & ERR_OVERLAP) return fail3(c, IMB_E_OVERFLOW, "three spheres cover one cell");
        if (bits & ERR_UNSTABLE) return fail3(c, IMB_E_UNSTABLE, "NaN or |u| >= 0.3 (Mach guard)");
    }
    return IMB_OK;
}

}  // namespace

extern "C" void imb3_default_params(imb3_params *p) {
    if (!p) return;
    p->wall_y = 1;
    p->Fx = p->Fy = p->Fz = 0.0;
    p->n_sub = 5;
    p->storage = IMB_STORE_FP32;
    p->rho0 = 1.0;
    p->ux0 = p->uy0 = p->uz0 = 0.0;
    p->timeout_ms = 60000;
    p->wall_ux_bot = p->wall_ux_top = 0.0;
    p->C_smag = 0.0;
}

extern "C" int imb3_init(imb3_ctx **out, int nx, int ny, int nz, double tau, const imb3_params *params) {
    imb3_ctx *c = nullptr;
    if (!out) return fail3(c, IMB_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    imb3_params p;
    imb3_default_params(&p);
    if (params) p = *params;
    if (nx < 3 || ny < 3 || nz < 3 || !(tau > 0.5) || p.n_sub < 1 || p.n_sub > 10 || p.storage < 0 ||
        p.storage > 2 || (double)nx * ny * nz > 2.0e9 || p.timeout_ms < 1 || !(p.C_smag >= 0.0))
        return fail3(c, IMB_E_INVALID_ARG,
                     "bad lattice size, tau <= 1/2, n_sub outside 1..10, bad storage or C_smag < 0");
    c = new imb3_ctx();
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->tau = tau;
    c->p = p;
    c->elem = p.storage == IMB_STORE_FP32 ? 4 : 2;
    Args3 &a = c->a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.wall_y = p.wall_y ? 1 : 0;
    a.plane = (size_t)nx * ny * nz;
    a.tau = (float)tau;
    a.omega = (float)(1.0 / tau);
    a.Fx = (float)p.Fx;
    a.Fy = (float)p.Fy;
    a.Fz = (float)p.Fz;
    a.n_sub = p.n_sub;
    a.inv_nsub3 = (float)(1.0 / ((double)p.n_sub * p.n_sub * p.n_sub));
    a.uw_bot = (float)p.wall_ux_bot;
    a.uw_top = (float)p.wall_ux_top;
    a.smag_coef = (float)(18.0 * std::sqrt(2.0) * p.C_smag * p.C_smag);
    a.two_slots = 0;
    for (int q = 0; q < 19; ++q)
        a.off[q] = (long long)q * (long long)a.plane -
                   ((long long)cz3(q) * ny * nx + (long long)cy3(q) * nx + (long long)cx3(q));
    *out = c;
    CK3(cudaGetDevice(&c->device), "cudaGetDevice");
    CK3(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
    CK3(cudaMalloc(&c->buf[0], 19 * a.plane * c->elem), "populations");
    CK3(cudaMalloc(&c->buf[1], 19 * a.plane * c->elem), "populations");
    CK3(cudaMalloc(&c->map, a.plane * sizeof(unsigned)), "cell map");
    CK3(cudaMalloc(&c->map2, a.plane * sizeof(unsigned)), "cell map");
    CK3(cudaMalloc(&c->err, 2 * sizeof(unsigned)), "error word");
    CK3(cudaMallocHost(&c->h_err, sizeof(unsigned)), "error word");
    CK3(cudaMemsetAsync(c->map, 0, a.plane * sizeof(unsigned), c->stream), "clear");
    CK3(cudaMemsetAsync(c->map2, 0, a.plane * sizeof(unsigned), c->stream), "clear");
    CK3(cudaMemsetAsync(c->err, 0, 2 * sizeof(unsigned), c->stream), "clear");
    CK3(by_storage3(p.storage, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            k3_init<S><<<(unsigned)((a.plane + 255) / 256), 256, 0, c->stream>>>(
                (S *)c->buf[0], a.plane, (float)p.rho0, (float)p.ux0, (float)p.uy0, (float)p.uz0);
            return cudaGetLastError();
        }),
        "init");
    c->launches++;
    return wait3(c);
}

extern "C" int imb3_set_spheres(imb3_ctx *c, int n, const double *x, const double *v, const double *omega,
                                const double *R) {
    if (!c || n < 0 || (n > 0 && (!x || !v || !omega || !R)) || n >= (int)ID_MASK)
        return fail3(c, IMB_E_INVALID_ARG, "bad sphere arrays");
    const int L[3] = {c->nx, c->ny, c->nz};
    const bool per[3] = {true, !c->p.wall_y, true};
    double rmax = 0.0;
    for (int s = 0; s < n; ++s) {
        if (!(R[s] > 0.0) || R[s] > 1000.0) return fail3(c, IMB_E_INVALID_ARG, "radius must be in (0, 1000]");
        for (int d = 0; d < 3; ++d) {
            if (!(x[3 * s + d] >= 0.0 && x[3 * s + d] < L[d]))
                return fail3(c, IMB_E_INVALID_ARG, "sphere centre outside the lattice");
            if (per[d] && 2.0 * (R[s] + 2.0) > L[d])
                return fail3(c, IMB_E_INVALID_ARG, "periodic extent below 2 (R + 2)");
        }
        rmax = std::max(rmax, R[s]);
    }
    const int span = (int)std::ceil(rmax) + 1, w = 2 * span + 1;   // the cell map's box per sphere
    const long long nt = (long long)n * w * w * w;
    if ((nt + 127) / 128 > 2147483647LL)
        return fail3(c, IMB_E_INVALID_ARG, "spheres x bounding box exceed one cell-map launch");
    CK3(cudaSetDevice(c->device), "cudaSetDevice");
    CK3(cudaStreamSynchronize(c->stream), "stream");
    if (c->sph) cudaFree(c->sph);
    if (c->FT) cudaFree(c->FT);
    c->sph = nullptr;
    c->FT = nullptr;
    c->np = n;
    c->a.two_slots = 0;
    CK3(cudaMemsetAsync(c->map, 0, c->a.plane * sizeof(unsigned), c->stream), "clear map");
    CK3(cudaMemsetAsync(c->map2, 0, c->a.plane * sizeof(unsigned), c->stream), "clear map");
    CK3(cudaMemsetAsync(c->err + 1, 0, sizeof(unsigned), c->stream), "clear map");
    if (n == 0) return wait3(c);
    std::vector<Sph3> hs(n);
    for (int s = 0; s < n; ++s) {
        Sph3 &P = hs[s];
        const double fi = std::floor(x[3 * s]), fj = std::floor(x[3 * s + 1]), fk = std::floor(x[3 * s + 2]);
        P.ci = (int)fi;
        P.cj = (int)fj;
        P.ck = (int)fk;
        P.fx = (float)(x[3 * s] - fi);
        P.fy = (float)(x[3 * s + 1] - fj);
        P.fz = (float)(x[3 * s + 2] - fk);
        P.vx = (float)v[3 * s];
        P.vy = (float)v[3 * s + 1];
        P.vz = (float)v[3 * s + 2];
        P.wx = (float)omega[3 * s];
        P.wy = (float)omega[3 * s + 1];
        P.wz = (float)omega[3 * s + 2];
    }
    double *dx = nullptr, *dR = nullptr;
    CK3(cudaMalloc(&c->sph, sizeof(Sph3) * n), "spheres");
    CK3(cudaMalloc(&c->FT, sizeof(double) * 6 * n), "forces");
    CK3(cudaMalloc(&dx, sizeof(double) * 3 * n), "spheres");
    CK3(cudaMalloc(&dR, sizeof(double) * n), "spheres");
    CK3(cudaMemcpyAsync(c->sph, hs.data(), sizeof(Sph3) * n, cudaMemcpyHostToDevice, c->stream), "spheres");
    CK3(cudaMemcpyAsync(dx, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream), "spheres");
    CK3(cudaMemcpyAsync(dR, R, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "spheres");
    CK3(cudaMemsetAsync(c->FT, 0, sizeof(double) * 6 * n, c->stream), "clear forces");
    k3_map<<<(unsigned)((nt + 127) / 128), 128, 0, c->stream>>>(dx, dR, n, span, c->a, c->map, c->map2, c->err + 1,
                                                                 c->err);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    int rc = e == cudaSuccess ? wait3(c) : fail3(c, IMB_E_CUDA, std::string("cell map: ") + cudaGetErrorString(e));
    cudaFree(dx);
    cudaFree(dR);
    if (rc == IMB_OK) {   // the kernel reads the second slot only once some cell holds two spheres
        unsigned shared = 0;
        e = cudaMemcpy(&shared, c->err + 1, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = fail3(c, IMB_E_CUDA, std::string("cell map: ") + cudaGetErrorString(e));
        c->a.two_slots = shared ? 1 : 0;
    }
    if (rc != IMB_OK) {   // a refused set leaves the lattice without spheres, not half mapped
        c->a.two_slots = 0;
        cudaMemsetAsync(c->map, 0, c->a.plane * sizeof(unsigned), c->stream);
        cudaMemsetAsync(c->map2, 0, c->a.plane * sizeof(unsigned), c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(c->sph);
        cudaFree(c->FT);
        c->sph = nullptr;
        c->FT = nullptr;
        c->np = 0;
    }
    return rc;
}

extern "C" int imb3_step(imb3_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return fail3(c, IMB_E_INVALID_ARG, "bad arguments");
    CK3(cudaSetDevice(c->device), "cudaSetDevice");
    const dim3 blk(32, 8, 1), grd((c->nx + 31) / 32, (c->ny + 7) / 8, (c->nz + ZC - 1) / ZC);
    for (int t = 0; t < nsteps; ++t) {
        if (c->np) CK3(cudaMemsetAsync(c->FT, 0, sizeof(double) * 6 * c->np, c->stream), "clear forces");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->timing) {
            while (c->events.size() < c->ev_used + 2) {
                cudaEvent_t e;
                CK3(cudaEventCreate(&e), "event");
                c->events.push_back(e);
            }
            e0 = c->events[c->ev_used];
            e1 = c->events[c->ev_used + 1];
            c->ev_used += 2;
            CK3(cudaEventRecord(e0, c->stream), "event record");
        }
        CK3(by_storage3(c->p.storage, [&](auto tag) {
                using S = std::remove_pointer_t<decltype(tag)>;
                const S *fin = (const S *)c->buf[c->cur];
                S *fout = (S *)c->buf[c->cur ^ 1];
                if (c->a.smag_coef > 0.0f || c->a.two_slots)
                    k3_stream_collide<true, S><<<grd, blk, 0, c->stream>>>(fin, fout, c->a, c->map, c->map2, c->sph,
                                                                           c->FT, c->err);
                else
                    k3_stream_collide<false, S><<<grd, blk, 0, c->stream>>>(fin, fout, c->a, c->map, c->map2, c->sph,
                                                                            c->FT, c->err);
                return cudaGetLastError();
            }),
            "stream-collide");
        if (c->timing) CK3(cudaEventRecord(e1, c->stream), "event record");
        c->launches++;
        c->cur ^= 1;
    }
    return wait3(c);
}

extern "C" int imb3_get_populations(imb3_ctx *c, double *f) {
    if (!c || !f) return fail3(c, IMB_E_INVALID_ARG, "bad arguments");
    CK3(cudaSetDevice(c->device), "cudaSetDevice");
    double *d = nullptr;
    CK3(cudaMalloc(&d, sizeof(double) * 19 * c->a.plane), "readback buffer");
    cudaError_t e = by_storage3(c->p.storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        k3_gather<S><<<(unsigned)((c->a.plane + 255) / 256), 256, 0, c->stream>>>((const S *)c->buf[c->cur], c->a, d);
        return cudaGetLastError();
    });
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, d, sizeof(double) * 19 * c->a.plane, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    CK3(e, "populations");
    c->launches++;
    return wait3(c);
}

extern "C" int imb3_get_macro(imb3_ctx *c, double *rho, double *ux, double *uy, double *uz) {
    if (!c || !rho || !ux || !uy || !uz) return fail3(c, IMB_E_INVALID_ARG, "bad arguments");
    CK3(cudaSetDevice(c->device), "cudaSetDevice");
    double *d = nullptr;
    const size_t n = c->a.plane;
    CK3(cudaMalloc(&d, sizeof(double) * 4 * n), "readback buffer");
    cudaError_t e = by_storage3(c->p.storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        k3_macro<S><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const S *)c->buf[c->cur], c->a, d, d + n,
                                                                        d + 2 * n, d + 3 * n);
        return cudaGetLastError();
    });
    double *outs[4] = {rho, ux, uy, uz};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(outs[k], d + k * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    CK3(e, "macroscopic fields");
    c->launches++;
    return wait3(c);
}

extern "C" int imb3_get_forces(imb3_ctx *c, double *F, double *T) {
    if (!c || (c->np && (!F || !T))) return fail3(c, IMB_E_INVALID_ARG, "bad arguments");
    int rc = wait3(c);
    if (rc || c->np == 0) return rc;
    std::vector<double> h(6 * (size_t)c->np);
    CK3(cudaMemcpy(h.data(), c->FT, sizeof(double) * h.size(), cudaMemcpyDeviceToHost), "forces");
    for (int s = 0; s < c->np; ++s)
        for (int d = 0; d < 3; ++d) {
            F[3 * s + d] = h[6 * s + d];
            T[3 * s + d] = h[6 * s + 3 + d];
        }
    return IMB_OK;
}

extern "C" int imb3_get_cell_map(imb3_ctx *c, int *sphere, int *count) {
    if (!c || !sphere || !count) return fail3(c, IMB_E_INVALID_ARG, "bad arguments");
    int rc = wait3(c);
    if (rc) return rc;
    std::vector<unsigned> h(c->a.plane), h2(c->a.plane);
    CK3(cudaMemcpy(h.data(), c->map, sizeof(unsigned) * h.size(), cudaMemcpyDeviceToHost), "cell map");
    CK3(cudaMemcpy(h2.data(), c->map2, sizeof(unsigned) * h2.size(), cudaMemcpyDeviceToHost), "cell map");
    for (size_t k = 0; k < h.size(); ++k) {
        unsigned a = h[k], b = h2[k];
        if (b && (b & ID_MASK) < (a & ID_MASK)) std::swap(a, b);   // the sphere of lower index first
        sphere[2 * k] = (int)(a & ID_MASK) - 1;
        count[2 * k] = (int)(a >> ID_BITS);
        sphere[2 * k + 1] = (int)(b & ID_MASK) - 1;
        count[2 * k + 1] = (int)(b >> ID_BITS);
    }
    return IMB_OK;
}

extern "C" int imb3_enable_kernel_timing(imb3_ctx *c, int on) {
    if (!c) return IMB_E_INVALID_ARG;
    c->timing = on != 0;
    c->ev_used = 0;
    return IMB_OK;
}

extern "C" int imb3_kernel_time(imb3_ctx *c, double *ms, long long *launches) {
    if (!c || !ms || !launches) return IMB_E_INVALID_ARG;
    int rc = wait3(c);
    if (rc) return rc;
    double tot = 0.0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float t = 0.0f;
        CK3(cudaEventElapsedTime(&t, c->events[k], c->events[k + 1]), "event elapsed");
        tot += t;
    }
    *ms = tot;
    *launches = (long long)(c->ev_used / 2);
    c->ev_used = 0;
    return IMB_OK;
}

extern "C" long long imb3_launch_count(imb3_ctx *c) { return c ? c->launches : 0; }

extern "C" double imb3_bytes_per_cell(imb3_ctx *c) { return c ? 38.0 * (double)c->elem : 0.0; }

extern "C" const char *imb3_last_error(imb3_ctx *c) { return c ? c->msg.c_str() : g3_err.c_str(); }

extern "C" void imb3_destroy(imb3_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void *b : c->buf)
        if (b) cudaFree(b);
    if (c->map) cudaFree(c->map);
    if (c->map2) cudaFree(c->map2);
    if (c->err) cudaFree(c->err);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->sph) cudaFree(c->sph);
    if (c->FT) cudaFree(c->FT);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}
