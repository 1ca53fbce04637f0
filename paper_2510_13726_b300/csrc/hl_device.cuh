// Device-side building blocks of the HHRRLBM-LES rotor step (sm_103a).
//
// Population slots: 0 = rest, 1..P = the P "positive" velocities c_p,
// P+1..2P = their opposites -c_p.  Populations are stored shifted by their
// rest weight, g_i = f_i - w_i, in FP32, FP16 or BF16; all arithmetic is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <utility>

namespace hl {

// ---------------------------------------------------------------------------
// velocity sets (Sec. 2.2, Fig. "D3Q19"; D3Q27 is its product-lattice sibling)
//
// The P = (Q-1)/2 "positive" velocities are encoded as bit masks per axis
// (bit p set: component non-zero; second mask: component negative), so the
// components are constant expressions of (Q, p, axis) without any table:
// inside fully unrolled loops every branch on them folds away.
//   D3Q19 p = 0..8 : (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)
//   D3Q27 p = 9..12: (1,1,1) (1,1,-1) (1,-1,1) (1,-1,-1)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int npos(int Q) { return (Q - 1) / 2; }

__host__ __device__ constexpr int cpos(int Q, int p, int a) {
    return ((((Q == 19) ? (a == 0 ? 121u : a == 1 ? 410u : 484u)
                        : (a == 0 ? 7801u : a == 1 ? 8090u : 8164u)) >> p) & 1u)
               ? (((((Q == 19) ? (a == 0 ? 0u : a == 1 ? 16u : 320u)
                               : (a == 0 ? 0u : a == 1 ? 6160u : 5440u)) >> p) & 1u) ? -1 : 1)
               : 0;
}

// slot s: 0 rest, 1..P positive velocities, P+1..2P their opposites
__host__ __device__ constexpr int cslot(int Q, int s, int a) {
    return s == 0 ? 0 : (s <= npos(Q) ? cpos(Q, s - 1, a) : -cpos(Q, s - 1 - npos(Q), a));
}
__host__ __device__ constexpr int oslot(int Q, int s) {
    return s == 0 ? 0 : (s <= npos(Q) ? s + npos(Q) : s - npos(Q));
}
__host__ __device__ constexpr int shell(int Q, int p) {
    return cpos(Q, p, 0) * cpos(Q, p, 0) + cpos(Q, p, 1) * cpos(Q, p, 1) + cpos(Q, p, 2) * cpos(Q, p, 2);
}
__host__ __device__ constexpr float w0(int Q) { return Q == 19 ? 1.0f / 3.0f : 8.0f / 27.0f; }
__host__ __device__ constexpr float wpos(int Q, int p) {
    return Q == 19 ? (shell(Q, p) == 1 ? 1.0f / 18.0f : 1.0f / 36.0f)
                   : (shell(Q, p) == 1 ? 2.0f / 27.0f : (shell(Q, p) == 2 ? 1.0f / 54.0f : 1.0f / 216.0f));
}

// ---------------------------------------------------------------------------
// population storage: FP32, or FP16/BF16 of the weight-shifted value
// ---------------------------------------------------------------------------
enum StoreKind { ST_F32 = 0, ST_F16S = 1, ST_BF16S = 2 };

template <int S>
struct Store;
template <>
struct Store<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T* p) { return *p; }
    static __device__ __forceinline__ void st(T* p, float v) { *p = v; }
};
template <>
struct Store<ST_F16S> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<ST_BF16S> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// local cell model, Eq. (hlbm) with the hybrid recursive-regularized
// non-equilibrium and the third-order equilibrium (Sec. 2.2)
// ---------------------------------------------------------------------------
struct Band {
    float d;       // lattice porosity, 1 = fluid
    float uB[3];   // solid velocity + wall-model velocity
    float sigma;   // hybridisation factor
    float S[6];    // FD strain rate xx, yy, zz, xy, xz, yz
};

// Writes g*_i - the shifted post-collision populations - given the
// coefficient tensors of the Hermite expansion:
//   f*_i = w_i [ rho + 3 rho c.u + 9/2 H2:A + 9/2 H3:A3 ]
// with A = rho u u + (1-1/tau)(sigma Pi_neq - (1-sigma) 2 cs2 rho tau S) and
// A3 = rho u u u + (1-1/tau) sigma a1^(3).  For c in {-1,0,1}^3,
// H2:A = sum_a c_a^2 A_aa - tr(A)/3 + 2 sum_{a<b} c_a c_b A_ab and
// H3:A3 = sum_{a!=b} (3 c_a^2 - 1) c_b A3_aab + 6 c_x c_y c_z A3_xyz.
// Each pair (i, ibar) shares the even part and flips the odd part.
template <int Q>
__device__ __forceinline__ void assemble(float (&g)[Q], float drho, float rho, const float (&u)[3],
                                         const float (&A)[6], const float (&M)[6], float Axyz) {
    constexpr int P = npos(Q);
    const float trA = A[0] + A[1] + A[2];
    g[0] = w0(Q) * (drho - 1.5f * trA);
    const float r3 = 3.0f * rho;
    const float t3 = trA * (1.0f / 3.0f);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        const float w = wpos(Q, p);
        // even part: rho + 9/2 H2:A
        float h2 = -t3;
        if (cx != 0) h2 += A[0];
        if (cy != 0) h2 += A[1];
        if (cz != 0) h2 += A[2];
        if (cx * cy != 0) h2 += float(2 * cx * cy) * A[3];
        if (cx * cz != 0) h2 += float(2 * cx * cz) * A[4];
        if (cy * cz != 0) h2 += float(2 * cy * cz) * A[5];
        // odd part: 3 rho c.u + 9/2 H3:A3; M = (A3_xxy, A3_yyx, A3_xxz, A3_zzx, A3_yyz, A3_zzy)
        float cu = 0.0f;
        if (cx != 0) cu += float(cx) * u[0];
        if (cy != 0) cu += float(cy) * u[1];
        if (cz != 0) cu += float(cz) * u[2];
        float h3 = 0.0f;
        if (cy != 0) h3 += float((3 * cx * cx - 1) * cy) * M[0];
        if (cx != 0) h3 += float((3 * cy * cy - 1) * cx) * M[1];
        if (cz != 0) h3 += float((3 * cx * cx - 1) * cz) * M[2];
        if (cx != 0) h3 += float((3 * cz * cz - 1) * cx) * M[3];
        if (cz != 0) h3 += float((3 * cy * cy - 1) * cz) * M[4];
        if (cy != 0) h3 += float((3 * cz * cz - 1) * cy) * M[5];
        if (Q == 27 && cx * cy * cz != 0) h3 += float(6 * cx * cy * cz) * Axyz;
        const float E = w * (drho + 4.5f * h2);
        const float O = w * (r3 * cu + 4.5f * h3);
        g[1 + p] = E + O;
        g[1 + P + p] = E - O;
    }
}

// Shifted third-order equilibrium g^eq_i = f^eq_i(rho, u) - w_i.
template <int Q>
__device__ __forceinline__ void equilibrium(float (&g)[Q], float drho, const float (&u)[3]) {
    const float rho = 1.0f + drho;
    const float A[6] = {rho * u[0] * u[0], rho * u[1] * u[1], rho * u[2] * u[2],
                        rho * u[0] * u[1], rho * u[0] * u[2], rho * u[1] * u[2]};
    const float M[6] = {A[0] * u[1], A[1] * u[0], A[0] * u[2], A[2] * u[0], A[1] * u[2], A[2] * u[1]};
    const float Axyz = A[3] * u[2];
    assemble<Q>(g, drho, rho, u, A, M, Axyz);
}

// Moments of shifted populations: drho = sum g, j = sum c g.
template <int Q>
__device__ __forceinline__ void moments01(const float (&g)[Q], float& drho, float (&j)[3]) {
    constexpr int P = npos(Q);
    drho = g[0];
    j[0] = j[1] = j[2] = 0.0f;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int cx = cpos(Q, p, 0), cy = cpos(Q, p, 1), cz = cpos(Q, p, 2);
        const float s = g[1 + p] + g[1 + P + p];
        const float d = g[1 + p] - g[1 + P + p];
        drho += s;
        if (cx != 0) j[0] += float(cx) * d;
        if (cy != 0) j[1] += float(cy) * d;
        if (cz != 0) j[2] += float(cz) * d;
    }
}

__device__ __forceinline__ float rcp_approx(float x) { return __fdividef(1.0f, x); }
// sqrt(x) for x >= 0 from the hardware reciprocal square root
__device__ __forceinline__ float sqrt_approx(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// One collision in place on shifted populations.  BAND selects the
// homogenized (HLBM) branch; the bulk branch is d = 1, sigma = 1.
// Returns rho; u_out = fluid velocity of the pre-collision state.
template <int Q, bool BAND>
__device__ __forceinline__ float collide(float (&g)[Q], const Band& B, float tau_mo, float Ksmag,
                                         float (&u_out)[3]) {
    constexpr int P = npos(Q);
    float drho = g[0];
    float j[3] = {0.f, 0.f, 0.f};
    float pg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sum c_a c_b g: xx yy zz xy xz yz
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
    // hardware reciprocal and reciprocal square root (about one ulp): the
    // collision runs at the instruction-issue limit in its 16-bit D3Q27 form
    const float inv = rcp_approx(rho);
    const float u[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
    u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2];
    // non-equilibrium stress Pi_neq = Pi - rho cs2 I - rho u u (fluid velocity)
    const float dr3 = drho * (1.0f / 3.0f);
    const float N[6] = {pg[0] - dr3 - j[0] * u[0], pg[1] - dr3 - j[1] * u[1], pg[2] - dr3 - j[2] * u[2],
                        pg[3] - j[0] * u[1],       pg[4] - j[0] * u[2],       pg[5] - j[1] * u[2]};
    // Smagorinsky, Eqs. (turbVisc), (tauEff): positive root of
    // tau = tau_mo + 3 C_S^2 |S|, S = -Pi_neq / (2 rho cs2 tau)
    const float Qn = N[0] * N[0] + N[1] * N[1] + N[2] * N[2] +
                     2.0f * (N[3] * N[3] + N[4] * N[4] + N[5] * N[5]);
    const float tau = 0.5f * (tau_mo + sqrt_approx(fmaf(Ksmag * sqrt_approx(Qn), inv, tau_mo * tau_mo)));
    const float om = 1.0f - rcp_approx(tau);
    float uh[3] = {u[0], u[1], u[2]};
    float os = om;
    float A[6];
    if constexpr (BAND) {
        // Eq. (convexVelocity), d = 1 in the fluid
        const float e = 1.0f - B.d;
        uh[0] = B.d * u[0] + e * B.uB[0];
        uh[1] = B.d * u[1] + e * B.uB[1];
        uh[2] = B.d * u[2] + e * B.uB[2];
        os = om * B.sigma;
        const float fd = om * (1.0f - B.sigma) * (2.0f / 3.0f) * rho * tau;
        A[0] = rho * uh[0] * uh[0] + os * N[0] - fd * B.S[0];
        A[1] = rho * uh[1] * uh[1] + os * N[1] - fd * B.S[1];
        A[2] = rho * uh[2] * uh[2] + os * N[2] - fd * B.S[2];
        A[3] = rho * uh[0] * uh[1] + os * N[3] - fd * B.S[3];
        A[4] = rho * uh[0] * uh[2] + os * N[4] - fd * B.S[4];
        A[5] = rho * uh[1] * uh[2] + os * N[5] - fd * B.S[5];
    } else {
        A[0] = rho * uh[0] * uh[0] + os * N[0];
        A[1] = rho * uh[1] * uh[1] + os * N[1];
        A[2] = rho * uh[2] * uh[2] + os * N[2];
        A[3] = rho * uh[0] * uh[1] + os * N[3];
        A[4] = rho * uh[0] * uh[2] + os * N[4];
        A[5] = rho * uh[1] * uh[2] + os * N[5];
    }
    // third order: A3_aab = rho u_a^2 u_b + om sigma (2 u_a N_ab + u_b N_aa) (recursion with u^)
    const float rxx = rho * uh[0] * uh[0], ryy = rho * uh[1] * uh[1], rzz = rho * uh[2] * uh[2];
    const float M[6] = {rxx * uh[1] + os * (2.0f * uh[0] * N[3] + uh[1] * N[0]),
                        ryy * uh[0] + os * (2.0f * uh[1] * N[3] + uh[0] * N[1]),
                        rxx * uh[2] + os * (2.0f * uh[0] * N[4] + uh[2] * N[0]),
                        rzz * uh[0] + os * (2.0f * uh[2] * N[4] + uh[0] * N[2]),
                        ryy * uh[2] + os * (2.0f * uh[1] * N[5] + uh[2] * N[1]),
                        rzz * uh[1] + os * (2.0f * uh[2] * N[5] + uh[1] * N[2])};
    float Axyz = 0.0f;
    if constexpr (Q == 27)
        Axyz = rho * uh[0] * uh[1] * uh[2] + os * (uh[0] * N[5] + uh[1] * N[4] + uh[2] * N[3]);
    assemble<Q>(g, drho, rho, uh, A, M, Axyz);
    return rho;
}

// ---------------------------------------------------------------------------
// rotor geometry: binary32 decision value with a fixed operation order
// (explicit round-to-nearest intrinsics, no contraction), Sec. 3.1
// ---------------------------------------------------------------------------
constexpr int MAXROT = 8;
constexpr int MAXBLADES = 8;

// Torque-driven rotation (evolve structure): angle and angular velocity are
// device state, advanced after each step's force reduction; the kernels of a
// step read that step's frames from here instead of the launch parameters.
struct DriveDev {
    double theta, omega;        // angle and angular velocity of the current step
    double inertia, k_gen, q_gen0;
    float ck[MAXBLADES], sk[MAXBLADES], omegaf;   // frames of the current step
};

struct RotorDev {
    int lo[3], n[3];            // box of lattice cells that may be touched
    int zs_lo, zs_hi;           // planes a wall-model sample may read: the box's, or through a slab
                                // face that cuts the box, the halo planes beyond it (zs_lo <= z < zs_hi)
    long long box_cells;
    float cf[3];                // centre (binary32)
    float omega;
    int axis, n_blades;
    float hub;                  // hub sphere radius
    const float* sdf;           // blade grid [gz][gy][gx], frame (R, T, A)
    int g[3];
    float origin[3];
    float inv_h, h;
    float reach_plane2, reach_axial;   // cells beyond these can be neither force nor wall cells
    float ck[MAXBLADES], sk[MAXBLADES], cp, sp;   // per-step frames
    float cpD, spD;             // pitch frames that decide the cell sets (cp, sp unless frozen)
    int frozen;                 // 1: sets from (cpD, spD), porosity / normal / distance from (cp, sp)
    float* d;                   // [box] porosity
    uint8_t* flags;             // [box] bit0: d<1 (force set), bit1: wall cell
    float* wm;                  // [9][box]: du_x du_y du_z S_xx S_yy S_zz S_xy S_xz S_yz
    double* utau;               // [box] friction velocity (Newton warm start)
    uint8_t* active;            // [box]
    int* list;                  // [box] force cells of this step
    int* count;                 // [1] force cells; [1] wall cells at count + 1
    int* wlist;                 // [box] wall cells of this step (box index)
    float* wphi;                // [box] their signed distance
    signed char* wwhich;        // [box] their closest component (blade, or n_blades = hub)
    double* partial;            // [FORCE_BLOCKS][6]
    unsigned* done;             // [1]
    double* acc;                // F(3) M(3) | F_sum(3) M_sum(3)
    // reverse sweep only (null in forward steps)
    float* ddp;                 // [box] d(porosity)/d(pitch) of force cells
    float* gub;                 // [3][box] adjoint of u^B at wall cells
    float* gS;                  // [6][box] adjoint of S^FD at wall cells
    const double* tape_utau;    // [box] friction velocity at the start of the step (Newton start)
    const uint8_t* tape_active; // [box] wall function active in the previous step
    const double* gut_next;     // [box] adjoint of this step's friction velocity
    double* gut_prev;           // [box] adjoint of the previous step's friction velocity
    double* pacc;               // [PACC_SLOTS] pitch-gradient accumulators
    float wT, wQ;               // objective weights / n_avg for this step (0 outside the window)
    DriveDev* drive;            // torque-driven rotor state, or null (prescribed rotation)
};

// frames and angular velocity of the current step
__device__ __forceinline__ float rot_ck(const RotorDev& R, int k) { return R.drive ? R.drive->ck[k] : R.ck[k]; }
__device__ __forceinline__ float rot_sk(const RotorDev& R, int k) { return R.drive ? R.drive->sk[k] : R.sk[k]; }
__device__ __forceinline__ float rot_omega(const RotorDev& R) { return R.drive ? R.drive->omegaf : R.omega; }

constexpr int PACC_SLOTS = 64;

constexpr uint8_t FL_B = 1, FL_W = 2;

__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
    return __fmaf_rn(t, __fsub_rn(b, a), a);
}

__device__ __forceinline__ float blade_sample(const RotorDev& R, float pR, float qT, float qA) {
    const float g0 = __fmul_rn(__fsub_rn(pR, R.origin[0]), R.inv_h);
    const float g1 = __fmul_rn(__fsub_rn(qT, R.origin[1]), R.inv_h);
    const float g2 = __fmul_rn(__fsub_rn(qA, R.origin[2]), R.inv_h);
    const float f0 = floorf(g0), f1 = floorf(g1), f2 = floorf(g2);
    if (!(f0 >= 0.0f && f0 <= (float)(R.g[0] - 2) && f1 >= 0.0f && f1 <= (float)(R.g[1] - 2) &&
          f2 >= 0.0f && f2 <= (float)(R.g[2] - 2)))
        return __int_as_float(0x7f800000);
    const int i0 = (int)f0, j0 = (int)f1, k0 = (int)f2;
    const float tx = __fsub_rn(g0, f0), ty = __fsub_rn(g1, f1), tz = __fsub_rn(g2, f2);
    const long long sy = R.g[0], sz = (long long)R.g[0] * R.g[1];
    const float* s = R.sdf + (long long)k0 * sz + (long long)j0 * sy + i0;
    const float v00 = lerp_rn(__ldg(s), __ldg(s + 1), tx);
    const float v10 = lerp_rn(__ldg(s + sy), __ldg(s + sy + 1), tx);
    const float v01 = lerp_rn(__ldg(s + sz), __ldg(s + sz + 1), tx);
    const float v11 = lerp_rn(__ldg(s + sz + sy), __ldg(s + sz + sy + 1), tx);
    const float w0 = lerp_rn(v00, v10, ty);
    const float w1 = lerp_rn(v01, v11, ty);
    return lerp_rn(w0, w1, tz);
}

// Signed distance of cell (x,y,z) to the rotor at pitch frames (cp, sp);
// which = blade, or n_blades for the hub.
// Component of (v0, v1, v2) along axis k (selects, no local-memory indexing).
__device__ __forceinline__ float fsel3(int k, float v0, float v1, float v2) {
    return k == 0 ? v0 : (k == 1 ? v1 : v2);
}

__device__ __forceinline__ float rotor_phi(const RotorDev& R, float cp, float sp, int x, int y, int z, int& which) {
    const float r0 = __fsub_rn((float)x, R.cf[0]), r1 = __fsub_rn((float)y, R.cf[1]),
                r2l = __fsub_rn((float)z, R.cf[2]);
    const int a = R.axis, b = a == 2 ? 0 : a + 1, c = a == 0 ? 2 : a - 1;
    const float rb = fsel3(b, r0, r1, r2l), rc = fsel3(c, r0, r1, r2l), ra = fsel3(a, r0, r1, r2l);
    float best = __int_as_float(0x7f800000);
    which = -1;
    for (int k = 0; k < R.n_blades; ++k) {
        const float ck = rot_ck(R, k), sk = rot_sk(R, k);
        const float pR = __fmaf_rn(ck, rb, __fmul_rn(sk, rc));
        const float pT = __fmaf_rn(ck, rc, -__fmul_rn(sk, rb));
        const float qT = __fmaf_rn(cp, pT, -__fmul_rn(sp, ra));
        const float qA = __fmaf_rn(cp, ra, __fmul_rn(sp, pT));
        const float v = blade_sample(R, pR, qT, qA);
        if (v < best) { best = v; which = k; }
    }
    if (R.hub > 0.0f) {
        const float r2 = __fmaf_rn(rb, rb, __fmaf_rn(rc, rc, __fmul_rn(ra, ra)));
        const float v = __fsub_rn(__fsqrt_rn(r2), R.hub);
        if (v < best) { best = v; which = R.n_blades; }
    }
    return best;
}

// Signed distance of one component (blade `which`, or the hub) at the
// current pitch frames, with the operations of rotor_phi: for the component
// that attains the minimum the two agree bit for bit.
__device__ __forceinline__ float component_phi(const RotorDev& R, int which, int x, int y, int z) {
    const float r0 = __fsub_rn((float)x, R.cf[0]), r1 = __fsub_rn((float)y, R.cf[1]),
                r2l = __fsub_rn((float)z, R.cf[2]);
    const int a = R.axis, b = a == 2 ? 0 : a + 1, c = a == 0 ? 2 : a - 1;
    const float rb = fsel3(b, r0, r1, r2l), rc = fsel3(c, r0, r1, r2l), ra = fsel3(a, r0, r1, r2l);
    if (which >= R.n_blades) {
        const float r2 = __fmaf_rn(rb, rb, __fmaf_rn(rc, rc, __fmul_rn(ra, ra)));
        return __fsub_rn(__fsqrt_rn(r2), R.hub);
    }
    const int k = which;
    const float ck = rot_ck(R, k), sk = rot_sk(R, k);
    const float pR = __fmaf_rn(ck, rb, __fmul_rn(sk, rc));
    const float pT = __fmaf_rn(ck, rc, -__fmul_rn(sk, rb));
    const float qT = __fmaf_rn(R.cp, pT, -__fmul_rn(R.sp, ra));
    const float qA = __fmaf_rn(R.cp, ra, __fmul_rn(R.sp, pT));
    return blade_sample(R, pR, qT, qA);
}

// Outward unit normal (lab frame): trilinear interpolation of the grid's
// central-difference gradient, rotated back through pitch and azimuth.
__device__ inline void rotor_normal(const RotorDev& R, int which, int x, int y, int z, float n[3]) {
    const int a = R.axis, b = (a + 1) % 3, c = (a + 2) % 3;
    const float rl[3] = {(float)x - R.cf[0], (float)y - R.cf[1], (float)z - R.cf[2]};
    float v[3];
    if (which >= R.n_blades) {
        v[0] = rl[0]; v[1] = rl[1]; v[2] = rl[2];
    } else {
        const float ck = rot_ck(R, which), sk = rot_sk(R, which), cp = R.cp, sp = R.sp;
        const float rb = rl[b], rc = rl[c], ra = rl[a];
        const float pR = ck * rb + sk * rc, pT = ck * rc - sk * rb;
        const float qT = cp * pT - sp * ra, qA = cp * ra + sp * pT;
        const float gg[3] = {(pR - R.origin[0]) * R.inv_h, (qT - R.origin[1]) * R.inv_h,
                             (qA - R.origin[2]) * R.inv_h};
        int i0[3];
        float t[3];
        for (int k = 0; k < 3; ++k) {
            int f = (int)floorf(gg[k]);
            f = f < 0 ? 0 : (f > R.g[k] - 2 ? R.g[k] - 2 : f);
            i0[k] = f;
            t[k] = gg[k] - (float)f;
        }
        float gb[3] = {0.f, 0.f, 0.f};
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    const int node[3] = {i0[0] + cx, i0[1] + cy, i0[2] + cz};
                    const float wgt = (cx ? t[0] : 1.f - t[0]) * (cy ? t[1] : 1.f - t[1]) *
                                      (cz ? t[2] : 1.f - t[2]);
                    for (int d = 0; d < 3; ++d) {
                        int lo[3] = {node[0], node[1], node[2]}, hi[3] = {node[0], node[1], node[2]};
                        lo[d] = node[d] > 0 ? node[d] - 1 : node[d];
                        hi[d] = node[d] < R.g[d] - 1 ? node[d] + 1 : node[d];
                        const long long olo = ((long long)lo[2] * R.g[1] + lo[1]) * R.g[0] + lo[0];
                        const long long ohi = ((long long)hi[2] * R.g[1] + hi[1]) * R.g[0] + hi[0];
                        gb[d] += wgt * (__ldg(R.sdf + ohi) - __ldg(R.sdf + olo)) /
                                 ((float)(hi[d] - lo[d]) * R.h);
                    }
                }
        const float vT = cp * gb[1] + sp * gb[2];
        const float vA = -sp * gb[1] + cp * gb[2];
        const float vR = gb[0];
        float lab[3];
        lab[b] = ck * vR - sk * vT;
        lab[c] = sk * vR + ck * vT;
        lab[a] = vA;
        v[0] = lab[0]; v[1] = lab[1]; v[2] = lab[2];
    }
    const float nrm = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
    n[0] = v[0] * inv; n[1] = v[1] * inv; n[2] = v[2] * inv;
}

// ---------------------------------------------------------------------------
// wall function, Sec. 2.2.1, in FP32.  The Newton step f/f' of Eq.
// (implicitWF) is taken with numerator and denominator both multiplied by
// exp(-kappa u+): the same quotient, but neither factor overflows when an
// iterate lies far below the root (a cold start reaches u+ ~ 250, where
// exp(kappa u+) is beyond the FP32 range; both f and f' grow like it).  The
// stopping rule compares the unscaled residuals, which are +inf beyond
// kappa u+ = 80 (there the residual exceeds 5e33 and the rule cannot stop).
// ---------------------------------------------------------------------------
// Constants of the wall function; divisions by them become products.
struct WallFn {
    float E, kappa, inv_E, kappa_inv_E, inv_kappa, inv_nu, tol;
    int maxit;
};

__host__ __device__ inline WallFn make_wallfn(double E, double kappa, double nu, double tol, int maxit) {
    WallFn W;
    W.E = (float)E;
    W.kappa = (float)kappa;
    W.inv_E = (float)(1.0 / E);
    W.kappa_inv_E = (float)(kappa / E);
    W.inv_kappa = (float)(1.0 / kappa);
    W.inv_nu = (float)(1.0 / nu);
    W.tol = (float)tol;
    W.maxit = maxit;
    return W;
}

// The two solves are written once for a scalar type T: float in the time
// step, forward-mode duals in the reverse sweep (same operations on the
// value part).
__device__ __forceinline__ float wf_val(float x) { return x; }
__device__ __forceinline__ float wf_exp(float x) { return expf(x); }
__device__ __forceinline__ float wf_log(float x) { return logf(x); }
__device__ __forceinline__ float wf_rcp(float x) { return 1.0f / x; }

// y+(u+) of Eq. (spalding) and its derivative dy+/du+, given e = exp(kappa u+)
template <class T>
__device__ __forceinline__ T spalding_yplus_t(const T& up, const T& e, const WallFn& W) {
    const T k = W.kappa * up;
    return up + (e - 1.0f - k - 0.5f * k * k - (1.0f / 6.0f) * k * k * k) * W.inv_E;
}
template <class T>
__device__ __forceinline__ T spalding_dyplus_t(const T& up, const T& e, const WallFn& W) {
    const T k = W.kappa * up;
    return 1.0f + W.kappa_inv_E * (e - 1.0f - k - 0.5f * k * k);
}

// residual f(u_tau) = y+(u / u_tau) - u_tau y / nu of Eq. (implicitWF), for
// the stopping rule only (no derivative); +inf where kappa u+ > 80
__device__ __forceinline__ float wf_residual(float ut, float u, float y_nu, const WallFn& W) {
    const float up = u / ut;
    const float k = W.kappa * up;
    if (!(k <= 80.0f)) return INFINITY;
    return spalding_yplus_t(up, expf(k), W) - ut * y_nu;
}

// Newton step f / f' at u_tau, both scaled by s = exp(-kappa u+):
//   f s  = (u+ - u_tau y / nu) s + (1 - P3 s) / E
//   f' s = -(s + kappa / E (1 - P2 s)) u+ / u_tau - s y / nu
// with P2, P3 the Taylor polynomials of exp(kappa u+) to second and third order
template <class T>
__device__ __forceinline__ T wf_step(const T& ut, const T& u, const T& y_nu, const WallFn& W) {
    const T r = wf_rcp(ut);
    const T up = u * r;
    const T k = W.kappa * up;
    const T s = wf_exp(0.0f - k);
    const T P2 = 1.0f + k + 0.5f * k * k;
    const T P3 = P2 + (1.0f / 6.0f) * k * k * k;
    const T fs = (up - ut * y_nu) * s + (1.0f - P3 * s) * W.inv_E;
    const T fps = 0.0f - (s + W.kappa_inv_E * (1.0f - P2 * s)) * up * r - y_nu * s;
    return fs / fps;
}

// Newton-Raphson on Eq. (implicitWF): stop when the residual changes by less
// than tol, at most maxit iterations; a non-positive iterate is halved.  One
// exponential and one reciprocal per step, one more exponential per
// residual.
template <class T>
__device__ inline T wall_newton_t(const T& u, const T& y, const T& guess, const WallFn& W) {
    const T y_nu = y * W.inv_nu;
    T ut = guess;
    float fv = wf_residual(wf_val(ut), wf_val(u), wf_val(y_nu), W);
    for (int it = 0; it < W.maxit; ++it) {
        T un = ut - wf_step(ut, u, y_nu, W);
        if (!(wf_val(un) > 0.0f)) un = 0.5f * ut;
        const float fn = wf_residual(wf_val(un), wf_val(u), wf_val(y_nu), W);
        ut = un;
        if (fabsf(fn - fv) < W.tol) break;
        fv = fn;
    }
    return ut;
}

// inverse of Eq. (spalding): u+ for y+, Newton from the right of the root
// (y+ is convex and increasing in u+, so the iterates fall monotonically
// from a start value of at most ln(1 + E y+)/kappa: no overflow)
template <class T>
__device__ inline T spalding_uplus_t(const T& yp, const WallFn& W) {
    const T lg = wf_log(1.0f + W.E * yp) * W.inv_kappa;
    T up = wf_val(yp) < wf_val(lg) ? yp : lg;
    T e = wf_exp(W.kappa * up);
    T g = spalding_yplus_t(up, e, W) - yp;
    for (int it = 0; it < W.maxit; ++it) {
        T un = up - g / spalding_dyplus_t(up, e, W);
        if (!(wf_val(un) > 0.0f)) un = 0.5f * up;
        const T en = wf_exp(W.kappa * un);
        const T gn = spalding_yplus_t(un, en, W) - yp;
        up = un;
        e = en;
        if (fabsf(wf_val(gn) - wf_val(g)) < W.tol) break;
        g = gn;
    }
    return up;
}

}  // namespace hl
