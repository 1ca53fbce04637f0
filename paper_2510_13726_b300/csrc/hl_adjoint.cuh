// Device building blocks of the discrete adjoint of the rotor step.
//
// The adjoint differentiates the step as computed, with the cell sets
// (force cells, wall cells, each cell's closest rotor component) held at
// their forward values:
//   * the collision (Eq. (hlbm)) by a hand-derived vector-Jacobian product
//     of its compact Hermite form (below, FP32);
//   * the wall model (Sec. 2.2.1) by a hand-derived reverse pass in which
//     the two Newton solves are differentiated through the iterations they
//     actually took (forward-mode duals in FP64: a solve stopped by the
//     iteration cap is not a root, so the implicit-function derivative would
//     not be the derivative of the step);
//   * the rotor geometry (Sec. 3.1) by forward-mode duals in the pitch.
#pragma once

#include "hl_device.cuh"

namespace hl {

// ---------------------------------------------------------------------------
// Hermite projections of an adjoint population vector lam (slot order):
//   L0 = sum w lam,  L1_a = sum w c_a lam,
//   G2_k = 9/2 sum w lam dH2:A/dA_k   (k = xx yy zz xy xz yz),
//   G3_k = 9/2 sum w lam dH3:A3/dM_k  (M = xxy yyx xxz zzx yyz zzy),
//   Gxyz = 9/2 sum w lam 6 c_x c_y c_z,
// so that sum_i lam_i g*_i = rho L0 + 3 rho L1.u + G2.A + G3.M + Gxyz Axyz
// for the compact form written by assemble<Q>().
// ---------------------------------------------------------------------------
template <int Q>
struct Proj {
    float L0, L1[3], G2[6], G3[6], Gxyz;
};

template <int Q>
__device__ __forceinline__ void project(const float (&lam)[Q], Proj<Q>& r) {
    constexpr int P = npos(Q);
    const float l0 = w0(Q) * lam[0];
    r.L0 = l0;
    r.L1[0] = r.L1[1] = r.L1[2] = 0.f;
    const float t = -(1.0f / 3.0f) * l0;
    r.G2[0] = t; r.G2[1] = t; r.G2[2] = t;
    r.G2[3] = r.G2[4] = r.G2[5] = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.G3[k] = 0.f;
    r.Gxyz = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        const float w = wpos(Q, p);
        const float e = w * (lam[1 + p] + lam[1 + P + p]);
        const float o = w * (lam[1 + p] - lam[1 + P + p]);
        r.L0 += e;
        if (cx != 0) r.L1[0] += float(cx) * o;
        if (cy != 0) r.L1[1] += float(cy) * o;
        if (cz != 0) r.L1[2] += float(cz) * o;
        r.G2[0] += float(cx * cx) * e - (1.0f / 3.0f) * e;
        r.G2[1] += float(cy * cy) * e - (1.0f / 3.0f) * e;
        r.G2[2] += float(cz * cz) * e - (1.0f / 3.0f) * e;
        if (cx * cy != 0) r.G2[3] += float(2 * cx * cy) * e;
        if (cx * cz != 0) r.G2[4] += float(2 * cx * cz) * e;
        if (cy * cz != 0) r.G2[5] += float(2 * cy * cz) * e;
        if (cy != 0) r.G3[0] += float((3 * cx * cx - 1) * cy) * o;
        if (cx != 0) r.G3[1] += float((3 * cy * cy - 1) * cx) * o;
        if (cz != 0) r.G3[2] += float((3 * cx * cx - 1) * cz) * o;
        if (cx != 0) r.G3[3] += float((3 * cz * cz - 1) * cx) * o;
        if (cz != 0) r.G3[4] += float((3 * cy * cy - 1) * cz) * o;
        if (cy != 0) r.G3[5] += float((3 * cz * cz - 1) * cy) * o;
        if (Q == 27 && cx * cy * cz != 0) r.Gxyz += float(6 * cx * cy * cz) * o;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) { r.G2[k] *= 4.5f; r.G3[k] *= 4.5f; }
    r.Gxyz *= 4.5f;
}

// adjoint of the velocity u^ through the equilibrium-like parts
// rho u u (in A), rho u u u and os a1^(3) (in M, Axyz); N = Pi_neq (6 comps)
template <int Q>
__device__ __forceinline__ void uhat_bar(const Proj<Q>& r, float rho, const float (&uh)[3], float os,
                                         const float (&N)[6], float (&ub)[3]) {
    const float ux = uh[0], uy = uh[1], uz = uh[2];
    const float* G2 = r.G2;
    const float* G3 = r.G3;
    ub[0] = 3.0f * rho * r.L1[0] + rho * (2.0f * G2[0] * ux + G2[3] * uy + G2[4] * uz);
    ub[1] = 3.0f * rho * r.L1[1] + rho * (2.0f * G2[1] * uy + G2[3] * ux + G2[5] * uz);
    ub[2] = 3.0f * rho * r.L1[2] + rho * (2.0f * G2[2] * uz + G2[4] * ux + G2[5] * uy);
    // M0 = rho ux^2 uy + os (2 ux Nxy + uy Nxx), and the five others
    ub[0] += G3[0] * (2.0f * rho * ux * uy + 2.0f * os * N[3]);
    ub[1] += G3[0] * (rho * ux * ux + os * N[0]);
    ub[1] += G3[1] * (2.0f * rho * uy * ux + 2.0f * os * N[3]);
    ub[0] += G3[1] * (rho * uy * uy + os * N[1]);
    ub[0] += G3[2] * (2.0f * rho * ux * uz + 2.0f * os * N[4]);
    ub[2] += G3[2] * (rho * ux * ux + os * N[0]);
    ub[2] += G3[3] * (2.0f * rho * uz * ux + 2.0f * os * N[4]);
    ub[0] += G3[3] * (rho * uz * uz + os * N[2]);
    ub[1] += G3[4] * (2.0f * rho * uy * uz + 2.0f * os * N[5]);
    ub[2] += G3[4] * (rho * uy * uy + os * N[1]);
    ub[2] += G3[5] * (2.0f * rho * uz * uy + 2.0f * os * N[5]);
    ub[1] += G3[5] * (rho * uz * uz + os * N[2]);
    if (Q == 27) {
        ub[0] += r.Gxyz * (rho * uy * uz + os * N[5]);
        ub[1] += r.Gxyz * (rho * ux * uz + os * N[4]);
        ub[2] += r.Gxyz * (rho * ux * uy + os * N[3]);
    }
}

// Adjoint of an equilibrium at unit density, g^eq(0, u) (the inlet and
// outlet planes): given lam (adjoint of the written populations), dL/du.
template <int Q>
__device__ __forceinline__ void equilibrium_vjp(const float (&lam)[Q], const float (&u)[3], float (&ub)[3]) {
    Proj<Q> r;
    project<Q>(lam, r);
    const float N0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uhat_bar<Q>(r, 1.0f, u, 0.0f, N0, ub);
}

// Vector-Jacobian product of collide<Q, BAND>() on shifted populations g:
// on entry lam = adjoint of the post-collision populations, on exit the
// adjoint of the pre-collision populations; gd, guB, gS = adjoint of the
// band parameters d, u^B, S (6 comps); u_out, rho returned as in the forward.
template <int Q, bool BAND>
__device__ __forceinline__ void collide_vjp(const float (&g)[Q], const Band& B, float tau_mo, float Ksmag,
                                            float (&lam)[Q], float& gd, float (&guB)[3], float (&gS)[6],
                                            float (&u_out)[3], float& rho_out) {
    constexpr int P = npos(Q);
    // ---- forward quantities (as in collide<Q, BAND>) ----
    float drho = g[0];
    float j[3] = {0.f, 0.f, 0.f};
    float pg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        const float s = g[1 + p] + g[1 + P + p];
        const float d = g[1 + p] - g[1 + P + p];
        drho += s;
        if (cx != 0) { j[0] += float(cx) * d; pg[0] += s; }
        if (cy != 0) { j[1] += float(cy) * d; pg[1] += s; }
        if (cz != 0) { j[2] += float(cz) * d; pg[2] += s; }
        if (cx * cy != 0) pg[3] += float(cx * cy) * s;
        if (cx * cz != 0) pg[4] += float(cx * cz) * s;
        if (cy * cz != 0) pg[5] += float(cy * cz) * s;
    }
    const float rho = 1.0f + drho;
    const float inv = 1.0f / rho;
    const float u[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
    u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2];
    rho_out = rho;
    const float dr3 = drho * (1.0f / 3.0f);
    const float N[6] = {pg[0] - dr3 - j[0] * u[0], pg[1] - dr3 - j[1] * u[1], pg[2] - dr3 - j[2] * u[2],
                        pg[3] - j[0] * u[1],       pg[4] - j[0] * u[2],       pg[5] - j[1] * u[2]};
    const float Qn = N[0] * N[0] + N[1] * N[1] + N[2] * N[2] + 2.0f * (N[3] * N[3] + N[4] * N[4] + N[5] * N[5]);
    const float sq = sqrtf(Qn);
    const float rt = sqrtf(tau_mo * tau_mo + Ksmag * sq * inv);
    const float tau = 0.5f * (tau_mo + rt);
    const float om = 1.0f - 1.0f / tau;
    float uh[3] = {u[0], u[1], u[2]};
    float os = om, sig = 1.0f, dd = 1.0f;
    if constexpr (BAND) {
        dd = B.d;
        const float e = 1.0f - B.d;
        uh[0] = B.d * u[0] + e * B.uB[0];
        uh[1] = B.d * u[1] + e * B.uB[1];
        uh[2] = B.d * u[2] + e * B.uB[2];
        sig = B.sigma;
        os = om * sig;
    }
    // ---- reverse ----
    Proj<Q> r;
    project<Q>(lam, r);
    const float ux = uh[0], uy = uh[1], uz = uh[2];
    const float uu[6] = {ux * ux, uy * uy, uz * uz, ux * uy, ux * uz, uy * uz};
    const float mr[6] = {uu[0] * uy, uu[1] * ux, uu[0] * uz, uu[2] * ux, uu[1] * uz, uu[2] * uy};
    float rb = r.L0 + 3.0f * (r.L1[0] * ux + r.L1[1] * uy + r.L1[2] * uz);
#pragma unroll
    for (int k = 0; k < 6; ++k) rb += r.G2[k] * uu[k] + r.G3[k] * mr[k];
    if (Q == 27) rb += r.Gxyz * (uu[3] * uz);
    float ub[3];
    uhat_bar<Q>(r, rho, uh, os, N, ub);
    // dL/dN (6 independent components)
    float Nb[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Nb[k] = os * r.G2[k];
    Nb[0] += os * (r.G3[0] * uy + r.G3[2] * uz);
    Nb[1] += os * (r.G3[1] * ux + r.G3[4] * uz);
    Nb[2] += os * (r.G3[3] * ux + r.G3[5] * uy);
    Nb[3] += os * (2.0f * r.G3[0] * ux + 2.0f * r.G3[1] * uy);
    Nb[4] += os * (2.0f * r.G3[2] * ux + 2.0f * r.G3[3] * uz);
    Nb[5] += os * (2.0f * r.G3[4] * uy + 2.0f * r.G3[5] * uz);
    if (Q == 27) {
        Nb[5] += os * r.Gxyz * ux;
        Nb[4] += os * r.Gxyz * uy;
        Nb[3] += os * r.Gxyz * uz;
    }
    // dL/d(os)
    float osb = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) osb += r.G2[k] * N[k];
    osb += r.G3[0] * (2.0f * ux * N[3] + uy * N[0]) + r.G3[1] * (2.0f * uy * N[3] + ux * N[1]) +
           r.G3[2] * (2.0f * ux * N[4] + uz * N[0]) + r.G3[3] * (2.0f * uz * N[4] + ux * N[2]) +
           r.G3[4] * (2.0f * uy * N[5] + uz * N[1]) + r.G3[5] * (2.0f * uz * N[5] + uy * N[2]);
    if (Q == 27) osb += r.Gxyz * (ux * N[5] + uy * N[4] + uz * N[3]);
    float omb = osb * sig;
    float taub = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) gS[k] = 0.f;
    if constexpr (BAND) {
        // - om (1 - sigma) (2/3) rho tau S inside A
        const float c = (1.0f - sig) * (2.0f / 3.0f);
        float phi = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) phi += r.G2[k] * B.S[k];
        omb -= c * rho * tau * phi;
        taub -= om * c * rho * phi;
        rb -= om * c * tau * phi;
        const float fd = om * c * rho * tau;
#pragma unroll
        for (int k = 0; k < 6; ++k) gS[k] = -fd * r.G2[k];
    }
    taub += omb / (tau * tau);
    // tau = (tau_mo + sqrt(tau_mo^2 + K sqrt(Qn) / rho)) / 2
    if (Qn > 0.f && Ksmag > 0.f) {
        const float Xb = 0.25f * taub / rt;       // d/dX of tau, X = K sq / rho
        const float X = Ksmag * sq * inv;
        const float sqb = Xb * Ksmag * inv;
        rb -= Xb * X * inv;
        const float Qb = 0.5f * sqb / sq;
        Nb[0] += 2.0f * Qb * N[0];
        Nb[1] += 2.0f * Qb * N[1];
        Nb[2] += 2.0f * Qb * N[2];
        Nb[3] += 4.0f * Qb * N[3];
        Nb[4] += 4.0f * Qb * N[4];
        Nb[5] += 4.0f * Qb * N[5];
    }
    // u^ = d u + (1 - d) u^B
    float uf[3];
    if constexpr (BAND) {
        gd = ub[0] * (u[0] - B.uB[0]) + ub[1] * (u[1] - B.uB[1]) + ub[2] * (u[2] - B.uB[2]);
        const float e = 1.0f - dd;
        guB[0] = e * ub[0]; guB[1] = e * ub[1]; guB[2] = e * ub[2];
        uf[0] = dd * ub[0]; uf[1] = dd * ub[1]; uf[2] = dd * ub[2];
    } else {
        gd = ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2];
        guB[0] = guB[1] = guB[2] = 0.f;
        uf[0] = ub[0]; uf[1] = ub[1]; uf[2] = ub[2];
    }
    // N_aa = pg_aa - drho/3 - j_a^2/rho, N_ab = pg_ab - j_a j_b/rho; u = j/rho
    float drb = rb - (Nb[0] + Nb[1] + Nb[2]) * (1.0f / 3.0f) +
                (Nb[0] * u[0] * u[0] + Nb[1] * u[1] * u[1] + Nb[2] * u[2] * u[2] + Nb[3] * u[0] * u[1] +
                 Nb[4] * u[0] * u[2] + Nb[5] * u[1] * u[2]) -
                (uf[0] * u[0] + uf[1] * u[1] + uf[2] * u[2]) * inv;
    const float jb[3] = {-(2.0f * Nb[0] * u[0] + Nb[3] * u[1] + Nb[4] * u[2]) + uf[0] * inv,
                         -(2.0f * Nb[1] * u[1] + Nb[3] * u[0] + Nb[5] * u[2]) + uf[1] * inv,
                         -(2.0f * Nb[2] * u[2] + Nb[4] * u[0] + Nb[5] * u[1]) + uf[2] * inv};
    lam[0] = drb;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        float h = drb;
        if (cx != 0) h += Nb[0];
        if (cy != 0) h += Nb[1];
        if (cz != 0) h += Nb[2];
        if (cx * cy != 0) h += float(cx * cy) * Nb[3];
        if (cx * cz != 0) h += float(cx * cz) * Nb[4];
        if (cy * cz != 0) h += float(cy * cz) * Nb[5];
        float cj = 0.f;
        if (cx != 0) cj += float(cx) * jb[0];
        if (cy != 0) cj += float(cy) * jb[1];
        if (cz != 0) cj += float(cz) * jb[2];
        lam[1 + p] = h + cj;
        lam[1 + P + p] = h - cj;
    }
}

// ---------------------------------------------------------------------------
// pitch tangents of the geometry (FP32 forward-mode): the blade-frame point
// q(p) = (pR, cp pT - sp ra, cp ra + sp pT) moves with dq/dp = (0, -qA, qT)
// ---------------------------------------------------------------------------
// phi of component `which` at frames (cp, sp) and its pitch derivative
__device__ inline float component_phi_tan(const RotorDev& R, int which, int x, int y, int z, float& dphi) {
    dphi = 0.f;
    const float rl[3] = {(float)x - R.cf[0], (float)y - R.cf[1], (float)z - R.cf[2]};
    const int a = R.axis, b = (a + 1) % 3, c = (a + 2) % 3;
    const float rb = rl[b], rc = rl[c], ra = rl[a];
    if (which >= R.n_blades) return sqrtf(rb * rb + rc * rc + ra * ra) - R.hub;
    const float ck = R.ck[which], sk = R.sk[which], cp = R.cp, sp = R.sp;
    const float pR = ck * rb + sk * rc, pT = ck * rc - sk * rb;
    const float qT = cp * pT - sp * ra, qA = cp * ra + sp * pT;
    const float g0 = (pR - R.origin[0]) * R.inv_h, g1 = (qT - R.origin[1]) * R.inv_h,
                g2 = (qA - R.origin[2]) * R.inv_h;
    const float dg1 = -qA * R.inv_h, dg2 = qT * R.inv_h;
    const float f0 = floorf(g0), f1 = floorf(g1), f2 = floorf(g2);
    if (!(f0 >= 0.0f && f0 <= (float)(R.g[0] - 2) && f1 >= 0.0f && f1 <= (float)(R.g[1] - 2) && f2 >= 0.0f &&
          f2 <= (float)(R.g[2] - 2)))
        return __int_as_float(0x7f800000);
    const int i0 = (int)f0, j0 = (int)f1, k0 = (int)f2;
    const float tx = g0 - f0, ty = g1 - f1, tz = g2 - f2;
    const long long sy = R.g[0], sz = (long long)R.g[0] * R.g[1];
    const float* s = R.sdf + (long long)k0 * sz + (long long)j0 * sy + i0;
    const float s000 = __ldg(s), s100 = __ldg(s + 1), s010 = __ldg(s + sy), s110 = __ldg(s + sy + 1);
    const float s001 = __ldg(s + sz), s101 = __ldg(s + sz + 1), s011 = __ldg(s + sz + sy),
                s111 = __ldg(s + sz + sy + 1);
    const float v00 = s000 + tx * (s100 - s000), v10 = s010 + tx * (s110 - s010);
    const float v01 = s001 + tx * (s101 - s001), v11 = s011 + tx * (s111 - s011);
    const float w0 = v00 + ty * (v10 - v00), w1 = v01 + ty * (v11 - v01);
    const float dty = (1.f - tz) * (v10 - v00) + tz * (v11 - v01);   // d phi / d ty
    const float dtz = w1 - w0;                                         // d phi / d tz
    dphi = dty * dg1 + dtz * dg2;
    return w0 + tz * (w1 - w0);
}

// outward unit normal of component `which` (as rotor_normal) and its pitch derivative
__device__ inline void rotor_normal_tan(const RotorDev& R, int which, int x, int y, int z, float n[3],
                                        float dn[3]) {
    const int a = R.axis, b = (a + 1) % 3, c = (a + 2) % 3;
    const float rl[3] = {(float)x - R.cf[0], (float)y - R.cf[1], (float)z - R.cf[2]};
    float v[3], dv[3] = {0.f, 0.f, 0.f};
    if (which >= R.n_blades) {
        v[0] = rl[0]; v[1] = rl[1]; v[2] = rl[2];
    } else {
        const float ck = R.ck[which], sk = R.sk[which], cp = R.cp, sp = R.sp;
        const float rb = rl[b], rc = rl[c], ra = rl[a];
        const float pR = ck * rb + sk * rc, pT = ck * rc - sk * rb;
        const float qT = cp * pT - sp * ra, qA = cp * ra + sp * pT;
        const float gg[3] = {(pR - R.origin[0]) * R.inv_h, (qT - R.origin[1]) * R.inv_h,
                             (qA - R.origin[2]) * R.inv_h};
        const float dgg[3] = {0.f, -qA * R.inv_h, qT * R.inv_h};
        int i0[3];
        float t[3];
        for (int k = 0; k < 3; ++k) {
            int f = (int)floorf(gg[k]);
            f = f < 0 ? 0 : (f > R.g[k] - 2 ? R.g[k] - 2 : f);
            i0[k] = f;
            t[k] = gg[k] - (float)f;
        }
        float gb[3] = {0.f, 0.f, 0.f}, dgb[3] = {0.f, 0.f, 0.f};
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    const int node[3] = {i0[0] + cx, i0[1] + cy, i0[2] + cz};
                    const float wx = cx ? t[0] : 1.f - t[0], wy = cy ? t[1] : 1.f - t[1], wz = cz ? t[2] : 1.f - t[2];
                    const float wgt = wx * wy * wz;
                    // d wgt / dp (t_x does not move with the pitch)
                    const float dwgt = wx * ((cy ? 1.f : -1.f) * dgg[1] * wz + wy * (cz ? 1.f : -1.f) * dgg[2]);
                    for (int d = 0; d < 3; ++d) {
                        int lo[3] = {node[0], node[1], node[2]}, hi[3] = {node[0], node[1], node[2]};
                        lo[d] = node[d] > 0 ? node[d] - 1 : node[d];
                        hi[d] = node[d] < R.g[d] - 1 ? node[d] + 1 : node[d];
                        const long long olo = ((long long)lo[2] * R.g[1] + lo[1]) * R.g[0] + lo[0];
                        const long long ohi = ((long long)hi[2] * R.g[1] + hi[1]) * R.g[0] + hi[0];
                        const float der = (__ldg(R.sdf + ohi) - __ldg(R.sdf + olo)) / ((float)(hi[d] - lo[d]) * R.h);
                        gb[d] += wgt * der;
                        dgb[d] += dwgt * der;
                    }
                }
        const float vT = cp * gb[1] + sp * gb[2];
        const float vA = -sp * gb[1] + cp * gb[2];
        const float vR = gb[0];
        const float dvT = vA + cp * dgb[1] + sp * dgb[2];
        const float dvA = -vT - sp * dgb[1] + cp * dgb[2];
        const float dvR = dgb[0];
        float lab[3], dlab[3];
        lab[b] = ck * vR - sk * vT;  dlab[b] = ck * dvR - sk * dvT;
        lab[c] = sk * vR + ck * vT;  dlab[c] = sk * dvR + ck * dvT;
        lab[a] = vA;                 dlab[a] = dvA;
        for (int k = 0; k < 3; ++k) { v[k] = lab[k]; dv[k] = dlab[k]; }
    }
    const float nrm = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
    n[0] = v[0] * inv; n[1] = v[1] * inv; n[2] = v[2] * inv;
    const float nd = n[0] * dv[0] + n[1] * dv[1] + n[2] * dv[2];
    for (int k = 0; k < 3; ++k) dn[k] = (dv[k] - n[k] * nd) * inv;
}

// ---------------------------------------------------------------------------
// FP32 forward-mode duals for the two Newton solves of the wall function
// (wall_newton_t / spalding_uplus_t instantiated on Dual<NS>): the value and
// its derivatives along NS seeds
// ---------------------------------------------------------------------------
template <int NS>
struct Dual {
    float v, d[NS];
};

template <int NS>
__device__ __forceinline__ Dual<NS> dual_const(float v) {
    Dual<NS> r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = 0.0f;
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> dual_seed(float v, int k, float dv = 1.0f) {
    Dual<NS> r = dual_const<NS>(v);
    r.d[k] = dv;
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator+(const Dual<NS>& x, const Dual<NS>& y) {
    Dual<NS> r;
    r.v = x.v + y.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = x.d[k] + y.d[k];
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator-(const Dual<NS>& x, const Dual<NS>& y) {
    Dual<NS> r;
    r.v = x.v - y.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = x.d[k] - y.d[k];
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator*(const Dual<NS>& x, const Dual<NS>& y) {
    Dual<NS> r;
    r.v = x.v * y.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = x.d[k] * y.v + x.v * y.d[k];
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator/(const Dual<NS>& x, const Dual<NS>& y) {
    Dual<NS> r;
    r.v = x.v / y.v;
    if (isinf(y.v) && isfinite(x.v)) {
        // a finite value over an infinite one is 0 in a whole neighbourhood
        // (the Newton step of a wall-function solve whose exponential
        // overflowed for a collapsed start value): zero derivatives, where
        // the quotient rule would give 0 * inf
#pragma unroll
        for (int k = 0; k < NS; ++k) r.d[k] = 0.0f;
        return r;
    }
    const float ry = 1.0f / y.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = (x.d[k] - r.v * y.d[k]) * ry;
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator*(float s, const Dual<NS>& x) {
    Dual<NS> r;
    r.v = s * x.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = s * x.d[k];
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator*(const Dual<NS>& x, float s) {
    return s * x;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator+(float s, const Dual<NS>& x) {
    Dual<NS> r = x;
    r.v = s + x.v;
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator-(const Dual<NS>& x, float s) {
    Dual<NS> r = x;
    r.v = x.v - s;
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> operator-(float s, const Dual<NS>& x) {
    Dual<NS> r;
    r.v = s - x.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = -x.d[k];
    return r;
}
template <int NS>
__device__ __forceinline__ float wf_val(const Dual<NS>& x) {
    return x.v;
}
template <int NS>
__device__ __forceinline__ Dual<NS> wf_exp(const Dual<NS>& x) {
    Dual<NS> r;
    r.v = expf(x.v);
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = r.v * x.d[k];
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> wf_log(const Dual<NS>& x) {
    Dual<NS> r;
    r.v = logf(x.v);
    const float rx = 1.0f / x.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = x.d[k] * rx;
    return r;
}
template <int NS>
__device__ __forceinline__ Dual<NS> wf_rcp(const Dual<NS>& x) {
    Dual<NS> r;
    r.v = 1.0f / x.v;
    const float m = -r.v * r.v;
#pragma unroll
    for (int k = 0; k < NS; ++k) r.d[k] = m * x.d[k];
    return r;
}

}  // namespace hl
