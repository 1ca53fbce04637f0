// Bulk collision of two x-adjacent cells per thread in packed FP32x2
// arithmetic (sm_100+ FADD2 / FMUL2 / FFMA2).  The cell model is the bulk
// branch of `collide` (d = 1, sigma = 1; Eq. (hlbm) with the recursive-
// regularized non-equilibrium, the third-order equilibrium and the
// Smagorinsky relaxation time, Sec. 2.2): every component of a packed
// operation is the IEEE round-to-nearest result of the scalar operation, so
// each lane computes the scalar cell model; only the order of a few sums
// differs from the scalar code.  Reciprocal and square roots stay per lane.
//
// Why: the 16-bit storage forms halve the bytes per cell update but not the
// instructions, and the scalar collision issues ~500 instructions per cell;
// packing halves the arithmetic and lets the even-phase (and c_x = 0
// odd-phase) loads and stores move both cells in one access.
#pragma once

#include "hl_device.cuh"

namespace hl {

struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 mk2(float s) { return {make_float2(s, s)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
// a - b as fma(b, -1, a): one rounding, the IEEE difference
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

// two consecutive stored values <-> one packed pair (8-byte / 4-byte access;
// the caller guarantees the alignment)
template <int S>
struct Store2;
template <>
struct Store2<ST_F32> {
    static __device__ __forceinline__ F2 ld(const float* p) { return {*reinterpret_cast<const float2*>(p)}; }
    static __device__ __forceinline__ void st(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <>
struct Store2<ST_F16S> {
    static __device__ __forceinline__ F2 ld(const __half* p) {
        return {__half22float2(*reinterpret_cast<const __half2*>(p))};
    }
    static __device__ __forceinline__ void st(__half* p, F2 v) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.v.x, v.v.y);
    }
};
template <>
struct Store2<ST_BF16S> {
    static __device__ __forceinline__ F2 ld(const __nv_bfloat16* p) {
        return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p))};
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, F2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.v.x, v.v.y);
    }
};

// Sum of integer multiples of packed values whose first term needs no
// addition: inside the fully unrolled loops every coefficient is a constant
// and `on` is known at each point, so the branches fold away.
struct Acc {
    F2 v;
    bool on;
};
__device__ __forceinline__ Acc acc0() { return {mk2(0.0f), false}; }
__device__ __forceinline__ void accum(Acc& a, int c, F2 x) {
    if (c == 0) return;
    if (!a.on) {
        a.v = c == 1 ? x : mk2((float)c) * x;
        a.on = true;
    } else if (c == 1) {
        a.v = a.v + x;
    } else if (c == -1) {
        a.v = a.v - x;
    } else {
        a.v = fma2(mk2((float)c), x, a.v);
    }
}

// Packed form of `assemble` (same Hermite coefficients; see there).
template <int Q>
__device__ __forceinline__ void assemble_pair(F2 (&g)[Q], F2 drho, F2 rho, const F2 (&u)[3], const F2 (&A)[6],
                                              const F2 (&M)[6], F2 Axyz) {
    constexpr int P = npos(Q);
    const F2 trA = A[0] + A[1] + A[2];
    g[0] = mk2(w0(Q)) * fma2(mk2(-1.5f), trA, drho);
    const F2 r3 = mk2(3.0f) * rho;
    const F2 nt3 = trA * mk2(-1.0f / 3.0f);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        // even part: rho + 9/2 H2:A
        Acc h2 = {nt3, true};
        accum(h2, cx * cx, A[0]);
        accum(h2, cy * cy, A[1]);
        accum(h2, cz * cz, A[2]);
        accum(h2, 2 * cx * cy, A[3]);
        accum(h2, 2 * cx * cz, A[4]);
        accum(h2, 2 * cy * cz, A[5]);
        // odd part: 3 rho c.u + 9/2 H3:A3
        Acc cu = acc0();
        accum(cu, cx, u[0]);
        accum(cu, cy, u[1]);
        accum(cu, cz, u[2]);
        Acc h3 = acc0();
        accum(h3, (3 * cx * cx - 1) * cy, M[0]);
        accum(h3, (3 * cy * cy - 1) * cx, M[1]);
        accum(h3, (3 * cx * cx - 1) * cz, M[2]);
        accum(h3, (3 * cz * cz - 1) * cx, M[3]);
        accum(h3, (3 * cy * cy - 1) * cz, M[4]);
        accum(h3, (3 * cz * cz - 1) * cy, M[5]);
        if (Q == 27) accum(h3, 6 * cx * cy * cz, Axyz);
        const F2 w = mk2(wpos(Q, p));
        const F2 E = w * fma2(mk2(4.5f), h2.v, drho);
        const F2 O = w * fma2(r3, cu.v, mk2(4.5f) * h3.v);
        g[1 + p] = E + O;
        g[1 + P + p] = E - O;
    }
}

// Packed form of collide<Q, false>: two bulk cells, in place on shifted
// populations.  Returns rho; u_out = fluid velocity of the pre-collision state.
template <int Q>
__device__ __forceinline__ F2 collide_pair(F2 (&g)[Q], float tau_mo, float Ksmag, F2 (&u_out)[3]) {
    constexpr int P = npos(Q);
    F2 drho = g[0];
    Acc ja[3] = {acc0(), acc0(), acc0()};
    Acc pa[6] = {acc0(), acc0(), acc0(), acc0(), acc0(), acc0()};
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        const F2 s = g[1 + p] + g[1 + P + p];
        const F2 d = g[1 + p] - g[1 + P + p];
        drho = drho + s;
        accum(ja[0], cx, d);
        accum(ja[1], cy, d);
        accum(ja[2], cz, d);
        accum(pa[0], cx * cx, s);
        accum(pa[1], cy * cy, s);
        accum(pa[2], cz * cz, s);
        accum(pa[3], cx * cy, s);
        accum(pa[4], cx * cz, s);
        accum(pa[5], cy * cz, s);
    }
    const F2 j[3] = {ja[0].v, ja[1].v, ja[2].v};
    const F2 pg[6] = {pa[0].v, pa[1].v, pa[2].v, pa[3].v, pa[4].v, pa[5].v};
    const F2 rho = mk2(1.0f) + drho;
    const F2 inv = {make_float2(rcp_approx(rho.v.x), rcp_approx(rho.v.y))};
    const F2 u[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
    u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2];
    const F2 nu[3] = {mk2(-1.0f) * u[0], mk2(-1.0f) * u[1], mk2(-1.0f) * u[2]};
    // non-equilibrium stress Pi_neq = Pi - rho cs2 I - rho u u (fluid velocity)
    const F2 dr3 = drho * mk2(1.0f / 3.0f);
    const F2 N[6] = {fma2(j[0], nu[0], pg[0] - dr3), fma2(j[1], nu[1], pg[1] - dr3), fma2(j[2], nu[2], pg[2] - dr3),
                     fma2(j[0], nu[1], pg[3]),       fma2(j[0], nu[2], pg[4]),       fma2(j[1], nu[2], pg[5])};
    // Smagorinsky, Eqs. (turbVisc), (tauEff), per lane
    const F2 qd = fma2(N[2], N[2], fma2(N[1], N[1], N[0] * N[0]));
    const F2 qo = fma2(N[5], N[5], fma2(N[4], N[4], N[3] * N[3]));
    const F2 Qn = fma2(mk2(2.0f), qo, qd);
    float omx, omy;
    {
        const float tx = 0.5f * (tau_mo + sqrt_approx(fmaf(Ksmag * sqrt_approx(Qn.v.x), inv.v.x, tau_mo * tau_mo)));
        const float ty = 0.5f * (tau_mo + sqrt_approx(fmaf(Ksmag * sqrt_approx(Qn.v.y), inv.v.y, tau_mo * tau_mo)));
        omx = 1.0f - rcp_approx(tx);
        omy = 1.0f - rcp_approx(ty);
    }
    const F2 om = {make_float2(omx, omy)};
    const F2 ru[3] = {rho * u[0], rho * u[1], rho * u[2]};
    const F2 rxx = ru[0] * u[0], ryy = ru[1] * u[1], rzz = ru[2] * u[2];
    const F2 rxy = ru[0] * u[1];
    F2 A[6];
    A[0] = fma2(om, N[0], rxx);
    A[1] = fma2(om, N[1], ryy);
    A[2] = fma2(om, N[2], rzz);
    A[3] = fma2(om, N[3], rxy);
    A[4] = fma2(om, N[4], ru[0] * u[2]);
    A[5] = fma2(om, N[5], ru[1] * u[2]);
    // third order: A3_aab = rho u_a^2 u_b + om (2 u_a N_ab + u_b N_aa)
    const F2 u2[3] = {u[0] + u[0], u[1] + u[1], u[2] + u[2]};
    F2 M[6];
    M[0] = fma2(om, fma2(u2[0], N[3], u[1] * N[0]), rxx * u[1]);
    M[1] = fma2(om, fma2(u2[1], N[3], u[0] * N[1]), ryy * u[0]);
    M[2] = fma2(om, fma2(u2[0], N[4], u[2] * N[0]), rxx * u[2]);
    M[3] = fma2(om, fma2(u2[2], N[4], u[0] * N[2]), rzz * u[0]);
    M[4] = fma2(om, fma2(u2[1], N[5], u[2] * N[1]), ryy * u[2]);
    M[5] = fma2(om, fma2(u2[2], N[5], u[1] * N[2]), rzz * u[1]);
    F2 Axyz = mk2(0.0f);
    if constexpr (Q == 27)
        Axyz = fma2(om, fma2(u[2], N[3], fma2(u[1], N[4], u[0] * N[5])), rxy * u[2]);
    assemble_pair<Q>(g, drho, rho, u, A, M, Axyz);
    return rho;
}

}  // namespace hl
