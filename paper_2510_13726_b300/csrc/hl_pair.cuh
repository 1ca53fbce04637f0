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

// The same with the two values exchanged where sel is SWAP2 (the pair at a
// periodic x wrap of the AA layout with x halves); KEEP2 leaves them.  For
// 16-bit storage one byte permutation of the stored word, for FP32 a select.
constexpr unsigned KEEP2 = 0x3210u, SWAP2 = 0x1032u;
template <int S>
struct Store2x;
template <>
struct Store2x<ST_F32> {
    static __device__ __forceinline__ F2 ld(const float* p, unsigned sel) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        return {sel == SWAP2 ? make_float2(v.y, v.x) : v};
    }
    static __device__ __forceinline__ void st(float* p, F2 v, unsigned sel) {
        *reinterpret_cast<float2*>(p) = sel == SWAP2 ? make_float2(v.v.y, v.v.x) : v.v;
    }
};
template <int S>
struct Store2x16 {
    using T = typename Store<S>::T;
    static __device__ __forceinline__ F2 ld(const T* p, unsigned sel) {
        const unsigned w = __byte_perm(*reinterpret_cast<const unsigned*>(p), 0u, sel);
        return Store2<S>::ld(reinterpret_cast<const T*>(&w));
    }
    static __device__ __forceinline__ void st(T* p, F2 v, unsigned sel) {
        unsigned w;
        Store2<S>::st(reinterpret_cast<T*>(&w), v);
        *reinterpret_cast<unsigned*>(p) = __byte_perm(w, 0u, sel);
    }
};
template <>
struct Store2x<ST_F16S> : Store2x16<ST_F16S> {};
template <>
struct Store2x<ST_BF16S> : Store2x16<ST_BF16S> {};

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

// Slot of velocity (cx, cy, cz), or -1 where the lattice lacks it (the D3Q19
// corners).  Velocities are stored with their first non-zero component
// positive in slots 1..P, opposites in P+1..2P (the order of cpos).
__host__ __device__ constexpr int slot_of(int Q, int cx, int cy, int cz) {
    if (cx == 0 && cy == 0 && cz == 0) return 0;
    const bool neg = cx < 0 || (cx == 0 && (cy < 0 || (cy == 0 && cz < 0)));
    const int x = neg ? -cx : cx, y = neg ? -cy : cy, z = neg ? -cz : cz;
    int p = -1;
    switch ((x + 1) * 9 + (y + 1) * 3 + (z + 1)) {
        case 22: p = 0; break;                    // ( 1, 0, 0)
        case 16: p = 1; break;                    // ( 0, 1, 0)
        case 14: p = 2; break;                    // ( 0, 0, 1)
        case 25: p = 3; break;                    // ( 1, 1, 0)
        case 19: p = 4; break;                    // ( 1,-1, 0)
        case 23: p = 5; break;                    // ( 1, 0, 1)
        case 21: p = 6; break;                    // ( 1, 0,-1)
        case 17: p = 7; break;                    // ( 0, 1, 1)
        case 15: p = 8; break;                    // ( 0, 1,-1)
        case 26: p = Q == 27 ? 9 : -1; break;     // ( 1, 1, 1)
        case 24: p = Q == 27 ? 10 : -1; break;    // ( 1, 1,-1)
        case 20: p = Q == 27 ? 11 : -1; break;    // ( 1,-1, 1)
        case 18: p = Q == 27 ? 12 : -1; break;    // ( 1,-1,-1)
        default: break;
    }
    if (p < 0) return -1;
    return neg ? 1 + npos(Q) + p : 1 + p;
}
__host__ __device__ constexpr bool slot_of_consistent(int Q) {
    for (int s = 0; s < Q; ++s)
        if (slot_of(Q, cslot(Q, s, 0), cslot(Q, s, 1), cslot(Q, s, 2)) != s) return false;
    int n = 0;
    for (int k = 0; k < 27; ++k) n += slot_of(Q, k / 9 - 1, (k / 3) % 3 - 1, k % 3 - 1) >= 0;
    return n == Q;
}
static_assert(slot_of_consistent(19) && slot_of_consistent(27), "slot_of disagrees with the slot tables");

__device__ __forceinline__ void accum(Acc& a, int c, const Acc& x) {
    if (x.on) accum(a, c, x.v);
}

// drho = sum g, j = sum c g, pg = sum c_a c_b g (xx yy zz xy xz yz) by three
// one-axis passes over the {-1, 0, 1}^3 velocity grid: along x the sums of
// c_x^k g (k = 0, 1, 2) per (c_y, c_z); along y and z only the combinations
// of order <= 2 that the ten moments use.
template <int Q>
__device__ __forceinline__ void moments_pair(const F2 (&g)[Q], F2& drho, F2 (&j)[3], F2 (&pg)[6]) {
    Acc S0[3][3], S1[3][3], S2[3][3];
#pragma unroll
    for (int iy = 0; iy < 3; ++iy)
#pragma unroll
        for (int iz = 0; iz < 3; ++iz) {
            const int sp = slot_of(Q, 1, iy - 1, iz - 1), sm = slot_of(Q, -1, iy - 1, iz - 1),
                      s0 = slot_of(Q, 0, iy - 1, iz - 1);
            Acc e = acc0(), o = acc0();
            if (sp >= 0) { accum(e, 1, g[sp]); accum(o, 1, g[sp]); }
            if (sm >= 0) { accum(e, 1, g[sm]); accum(o, -1, g[sm]); }
            S2[iy][iz] = e;
            S1[iy][iz] = o;
            if (s0 >= 0) accum(e, 1, g[s0]);
            S0[iy][iz] = e;
        }
    // T[m][iz], m: 0 (k_x, k_y) = (0, 0), 1 (0, 1), 2 (0, 2), 3 (1, 0), 4 (1, 1), 5 (2, 0)
    Acc T[6][3];
#pragma unroll
    for (int iz = 0; iz < 3; ++iz) {
        Acc b = acc0();
        accum(b, 1, S0[0][iz]);
        accum(b, 1, S0[2][iz]);
        T[2][iz] = b;
        accum(b, 1, S0[1][iz]);
        T[0][iz] = b;
        Acc d = acc0();
        accum(d, 1, S0[2][iz]);
        accum(d, -1, S0[0][iz]);
        T[1][iz] = d;
        Acc c = acc0();
        accum(c, 1, S1[0][iz]);
        accum(c, 1, S1[2][iz]);
        accum(c, 1, S1[1][iz]);
        T[3][iz] = c;
        Acc e = acc0();
        accum(e, 1, S1[2][iz]);
        accum(e, -1, S1[0][iz]);
        T[4][iz] = e;
        Acc f = acc0();
        accum(f, 1, S2[0][iz]);
        accum(f, 1, S2[2][iz]);
        accum(f, 1, S2[1][iz]);
        T[5][iz] = f;
    }
    // along z: plain sums, and the c_z-weighted ones for j_z, pg_xz, pg_yz
    Acc r = acc0();
    accum(r, 1, T[0][0]);
    accum(r, 1, T[0][2]);
    const F2 zz = r.v;                     // sum c_z^2 g
    accum(r, 1, T[0][1]);
    drho = r.v;
    Acc t;
    t = acc0(); accum(t, 1, T[0][2]); accum(t, -1, T[0][0]); j[2] = t.v;
    t = acc0(); accum(t, 1, T[1][0]); accum(t, 1, T[1][2]); accum(t, 1, T[1][1]); j[1] = t.v;
    t = acc0(); accum(t, 1, T[1][2]); accum(t, -1, T[1][0]); pg[5] = t.v;
    t = acc0(); accum(t, 1, T[2][0]); accum(t, 1, T[2][2]); accum(t, 1, T[2][1]); pg[1] = t.v;
    t = acc0(); accum(t, 1, T[3][0]); accum(t, 1, T[3][2]); accum(t, 1, T[3][1]); j[0] = t.v;
    t = acc0(); accum(t, 1, T[3][2]); accum(t, -1, T[3][0]); pg[4] = t.v;
    t = acc0(); accum(t, 1, T[4][0]); accum(t, 1, T[4][2]); accum(t, 1, T[4][1]); pg[3] = t.v;
    t = acc0(); accum(t, 1, T[5][0]); accum(t, 1, T[5][2]); accum(t, 1, T[5][1]); pg[0] = t.v;
    pg[2] = zz;
}

// a += c x for a compile-time constant c (a product for the first term)
__device__ __forceinline__ void accf(Acc& a, float c, F2 x) {
    if (c == 0.0f) return;
    if (!a.on) {
        a.v = c == 1.0f ? x : mk2(c) * x;
        a.on = true;
    } else if (c == 1.0f) {
        a.v = a.v + x;
    } else if (c == -1.0f) {
        a.v = a.v - x;
    } else {
        a.v = fma2(mk2(c), x, a.v);
    }
}
// a += r x for a packed run-time factor r
__device__ __forceinline__ void accr(Acc& a, F2 r, F2 x) {
    if (!a.on) {
        a.v = r * x;
        a.on = true;
    } else {
        a.v = fma2(r, x, a.v);
    }
}
__device__ __forceinline__ void acca(Acc& a, int c, const Acc& x) { accum(a, c, x); }

// Velocity groups of the assembly: the positive velocities whose non-zero
// components sit on the same axes, e.g. (1,1,0) and (1,-1,0), or the four
// D3Q27 corners (1,+-1,+-1).  Members differ only in the signs of their
// non-zero components after the first (the flipped components), so every
// Hermite term splits into parity classes: the set of flipped components it
// is odd in.  Each class sum is built once per group and each member's value
// is the signed sum of its group's classes.
//   groups: 0-2 the axes (p = 0, 1, 2), 3 xy (p = 3, 4), 4 xz (p = 5, 6),
//   5 yz (p = 7, 8), 6 the corners (p = 9..12, D3Q27)
__host__ __device__ constexpr int grp_count(int Q) { return Q == 19 ? 6 : 7; }
__host__ __device__ constexpr int grp_size(int G) { return G < 3 ? 1 : (G < 6 ? 2 : 4); }
__host__ __device__ constexpr int grp_first(int G) { return G < 3 ? G : (G == 3 ? 3 : (G == 4 ? 5 : (G == 5 ? 7 : 9))); }
// bit a set for each flipped component a
__host__ __device__ constexpr int grp_flip(int Q, int G) {
    return (cpos(Q, grp_first(G), 0) != 0)
               ? ((cpos(Q, grp_first(G), 1) != 0 ? 2 : 0) | (cpos(Q, grp_first(G), 2) != 0 ? 4 : 0))
               : (cpos(Q, grp_first(G), 1) != 0 ? (cpos(Q, grp_first(G), 2) != 0 ? 4 : 0) : 0);
}
// sign of member m of group G in the class q (product of its flipped-component signs in q)
__host__ __device__ constexpr int grp_sign(int Q, int G, int m, int q) {
    return ((q & 2) ? cpos(Q, grp_first(G) + m, 1) * cpos(Q, grp_first(G), 1) : 1) *
           ((q & 4) ? cpos(Q, grp_first(G) + m, 2) * cpos(Q, grp_first(G), 2) : 1);
}
static_assert(grp_flip(19, 3) == 2 && grp_flip(19, 4) == 4 && grp_flip(19, 5) == 4 && grp_flip(27, 6) == 6 &&
                  grp_flip(19, 0) == 0 && grp_flip(19, 2) == 0,
              "velocity groups disagree with the slot tables");
static_assert(grp_sign(19, 3, 1, 2) == -1 && grp_sign(27, 6, 1, 4) == -1 && grp_sign(27, 6, 2, 2) == -1 &&
                  grp_sign(27, 6, 3, 6) == 1,
              "velocity group signs disagree with the slot tables");

// Packed form of `assemble` (the same Hermite coefficients; see there), with
// the weights folded into the coefficients:
//   f_c  = E_c + O_c,  f_-c = E_c - O_c,
//   E_c  = w (D + 4.5 (H2 - tr/3) : A), D = drho - 1.5 tr A,
//   O_c  = 3 w rho c.u + 4.5 w H3 : A3,
// each summed per parity class of its group.  Fewer packed operations than
// summing every velocity separately (D3Q19: 75 against about 120 per pair of
// cells), the same terms in another order.
template <int Q>
__device__ __forceinline__ void assemble_pair(F2 (&g)[Q], F2 drho, F2 rho, const F2 (&u)[3], const F2 (&A)[6],
                                              const F2 (&M)[6], F2 Axyz) {
    constexpr int P = npos(Q);
    const F2 trA = A[0] + A[1] + A[2];
    const F2 D = fma2(mk2(-1.5f), trA, drho);
    g[0] = mk2(w0(Q)) * D;
    // per weight shell (|c|^2 = 1, 2, 3): w D and 3 w rho
    F2 wD[3], r3w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float w = Q == 19 ? (k == 0 ? 1.0f / 18.0f : 1.0f / 36.0f)
                                : (k == 0 ? 2.0f / 27.0f : (k == 1 ? 1.0f / 54.0f : 1.0f / 216.0f));
        if (Q == 19 && k == 2) continue;
        wD[k] = mk2(w) * D;
        r3w[k] = mk2(3.0f * w) * rho;
    }
#pragma unroll
    for (int G = 0; G < grp_count(Q); ++G) {
        const int p0 = grp_first(G);
        const int F = grp_flip(Q, G);
        const int cx = cpos(Q, p0, 0), cy = cpos(Q, p0, 1), cz = cpos(Q, p0, 2);
        const int sh = shell(Q, p0) - 1;
        const float w45 = 4.5f * wpos(Q, p0);
        Acc E[8], O[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            E[q] = acc0();
            O[q] = acc0();
            if ((q & ~F) != 0) continue;
            // even part: w D + 4.5 w H2 : A (term parity: its odd components among the flipped)
            if (q == 0) E[q] = {wD[sh], true};
            if ((0 & F) == q) {
                accf(E[q], w45 * (float)(cx * cx), A[0]);
                accf(E[q], w45 * (float)(cy * cy), A[1]);
                accf(E[q], w45 * (float)(cz * cz), A[2]);
            }
            if ((3 & F) == q) accf(E[q], w45 * (float)(2 * cx * cy), A[3]);
            if ((5 & F) == q) accf(E[q], w45 * (float)(2 * cx * cz), A[4]);
            if ((6 & F) == q) accf(E[q], w45 * (float)(2 * cy * cz), A[5]);
            // odd part: 3 w rho c.u + 4.5 w H3 : A3
            if ((1 & F) == q && cx != 0) accr(O[q], r3w[sh], u[0]);
            if ((2 & F) == q && cy != 0) accr(O[q], r3w[sh], u[1]);
            if ((4 & F) == q && cz != 0) accr(O[q], r3w[sh], u[2]);
            if ((2 & F) == q) accf(O[q], w45 * (float)((3 * cx * cx - 1) * cy), M[0]);
            if ((1 & F) == q) accf(O[q], w45 * (float)((3 * cy * cy - 1) * cx), M[1]);
            if ((4 & F) == q) accf(O[q], w45 * (float)((3 * cx * cx - 1) * cz), M[2]);
            if ((1 & F) == q) accf(O[q], w45 * (float)((3 * cz * cz - 1) * cx), M[3]);
            if ((4 & F) == q) accf(O[q], w45 * (float)((3 * cy * cy - 1) * cz), M[4]);
            if ((2 & F) == q) accf(O[q], w45 * (float)((3 * cz * cz - 1) * cy), M[5]);
            if (Q == 27 && (7 & F) == q) accf(O[q], w45 * (float)(6 * cx * cy * cz), Axyz);
        }
        // members: signed sums of the classes (two flipped components: the
        // second sign first, then the first)
        const int b1 = (F & 2) ? 2 : 4, b2 = (F == 6) ? 4 : 0;
#pragma unroll
        for (int m = 0; m < grp_size(G); ++m) {
            Acc e = E[0], o = O[0];
            if (b2) {
                const int s2 = grp_sign(Q, G, m, b2), s1 = grp_sign(Q, G, m, b1);
                Acc te = E[0], ue = E[b1], to = O[0], uo = O[b1];
                acca(te, s2, E[b2]);
                acca(ue, s2, E[b1 | b2]);
                acca(to, s2, O[b2]);
                acca(uo, s2, O[b1 | b2]);
                e = te;
                o = to;
                acca(e, s1, ue);
                acca(o, s1, uo);
            } else if (F) {
                const int s1 = grp_sign(Q, G, m, b1);
                acca(e, s1, E[b1]);
                acca(o, s1, O[b1]);
            }
            const int p = p0 + m;
            // the last two sums per lane: scalar FP32 can issue to both halves of
            // the FMA pipe, packed operations only to the heavy half
            g[1 + p] = {make_float2(e.v.v.x + o.v.v.x, e.v.v.y + o.v.v.y)};
            g[1 + P + p] = {make_float2(e.v.v.x - o.v.v.x, e.v.v.y - o.v.v.y)};
        }
    }
}

// Packed form of collide<Q, false>: two bulk cells, in place on shifted
// populations.  Returns rho; u_out = fluid velocity of the pre-collision state.
template <int Q>
__device__ __forceinline__ F2 collide_pair(F2 (&g)[Q], float tau_mo, float Ksmag, F2 (&u_out)[3]) {
    F2 drho, j[3], pg[6];
    moments_pair<Q>(g, drho, j, pg);
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
