// Discrete adjoint of the rotor time step and the checkpointed reverse
// sweep behind hl_grad().
//
// Objective (Sec. 3.2 forces, time-averaged over a window):
//   J = (1/n_avg) sum over the last n_avg of T steps of
//       sum_k [ wT_k F_k(t).a_k + wQ_k M_k(t).a_k ],
// gradients with respect to each rotor's pitch and the static porosity
// multiplier d0 (d = d0 d_rotor in Eq. (convexVelocity)), with the cell sets
// held at their forward values.
//
// Per reverse step t (the forward quantities of step t recomputed from the
// stored pre-collision state f_t):
//   band_kernel (tangent)   porosity, sets and d(porosity)/d(pitch)
//   wall_kernel             wall-model outputs of step t (linearisation point)
//   adj_bulk_kernel         cells outside every rotor box and the open planes:
//                           lam*_i(x) = lam_{t+1,i}(x + c_i) (transpose of the
//                           streaming), collision VJP, outlet equilibrium and
//                           the outlet's use of the upstream velocity
//   adj_box_kernel          rotor-box cells: the same plus the transpose of the
//                           momentum exchange and the band parameters
//   adj_wall_kernel         reverse pass of the wall model: corner populations,
//                           pitch, the next step's Newton start
//   adj_band_strain_kernel  (sigma < 1) reverse pass of the band strain: the
//                           neighbours' populations
// Memory: checkpoints of the full state every K steps, and the K states of a
// segment recomputed out of place (read buffer j, write buffer j + 1).
#include <cmath>
#include <cstring>

#include "hl_adjoint.cuh"
#include "hl_host.h"
#include "hl_pair.cuh"

namespace hl {

struct AdjArgs {
    const float* lam_next;   // [Q][N] adjoint of the pre-collision populations of step t + 1
    const float* lshift[27]; // lam_next + s N + (c_s . strides): lam_{t+1,s}(x + c_s) at lshift[s] + x
    float* lam;              // [Q][N] adjoint of the pre-collision populations of step t
    float* dJdd0;            // [N] accumulated gradient, or null
    const float* gup_cur;    // [3][plane] adjoint of the upstream velocity this step hands to the outlet
    float* gup_prev;         // [3][plane] adjoint of the velocity the outlet read in this step
};

namespace {

struct Offs {
    int x[3], y[3], z[3];
};

__device__ __forceinline__ void make_offs(const StepArgs& a, int x, int y, int z, Offs& o) {
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2], nxy = a.nxy;
    o.x[0] = x == 0 ? nx - 1 : x - 1;
    o.x[1] = x;
    o.x[2] = x == nx - 1 ? 0 : x + 1;
    o.y[0] = (y == 0 ? ny - 1 : y - 1) * nx;
    o.y[1] = y * nx;
    o.y[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    o.z[0] = (z == 0 ? nz - 1 : z - 1) * nxy;
    o.z[1] = z * nxy;
    o.z[2] = (z == nz - 1 ? 0 : z + 1) * nxy;
}

__device__ __forceinline__ int sel3(int ax, int a0, int a1, int a2) { return ax == 0 ? a0 : (ax == 1 ? a1 : a2); }

// pre-collision populations of a cell in the AA layout of phase PH
template <int Q, int S, int PH>
__device__ __forceinline__ void load_pre(const StepArgs& a, int cell, const Offs& o, float (&g)[Q]) {
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        if (PH == 0) {
            g[s] = Store<S>::ld(static_cast<const typename Store<S>::T*>(a.slot[s]) + cell);
        } else {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            const int src = o.x[1 - cx] + o.y[1 - cy] + o.z[1 - cz];
            g[s] = Store<S>::ld(static_cast<const typename Store<S>::T*>(a.slot[oslot(Q, s)]) + src);
        }
    }
}

// Esoteric-twist state <-> AA state of the same step.  Each layout keeps
// the pre-collision f_s(x) of a step at one place: AA, slot s at x (even
// steps) or slot sbar at x - c_s (odd steps); esoteric twist, slot s (even)
// or sbar (odd) at x + max(-c_s, 0); with periodic neighbour indices these
// places cover the buffer once over all (x, s), so the change of layout is a
// permutation of the stored values (raw storage words, no rounding).
template <int Q, int S, int PH>
__global__ void __launch_bounds__(128) relayout_kernel(const StepArgs a, const void* src, void* dst, int to_eso) {
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= a.n[0]) return;
    Offs o;
    make_offs(a, x, y, z, o);
    const long long N = a.N;
    const T* in = static_cast<const T*>(src);
    T* out = static_cast<T*>(dst);
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
        const long long base = (long long)(PH == 0 ? s : oslot(Q, s)) * N;
        const long long aa = base + (PH == 0 ? o.x[1] + o.y[1] + o.z[1] : o.x[1 - cx] + o.y[1 - cy] + o.z[1 - cz]);
        const long long es = base + (o.x[1 + (cx < 0)] + o.y[1 + (cy < 0)] + o.z[1 + (cz < 0)]);
        if (to_eso) out[es] = in[aa];
        else out[aa] = in[es];
    }
}

// AA layout with x halves <-> AA layout: every stored value moves along its
// x row, cell x's place 2x (x < nx/2) or 2(x - nx/2) + 1 <-> x (raw storage
// words, either step parity)
template <int S>
__global__ void __launch_bounds__(128) xhalves_kernel(const StepArgs a, int q, const void* src, void* dst,
                                                      int to_halves) {
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= a.n[0]) return;
    const int hx = a.n[0] / 2;
    const long long row = ((long long)z * a.n[1] + y) * a.n[0];
    const long long xh = row + (x < hx ? 2 * x : 2 * (x - hx) + 1), xa = row + x;
    const T* in = static_cast<const T*>(src);
    T* out = static_cast<T*>(dst);
    for (int s = 0; s < q; ++s) {
        const long long b = (long long)s * a.N;
        if (to_halves) out[b + xh] = in[b + xa];
        else out[b + xa] = in[b + xh];
    }
}

// lam*_s(x) = lam_{t+1, s}(x + c_s); the adjoint is zero on the open planes,
// so the periodic index of a neighbour across an open face reads a zero
template <int Q>
__device__ __forceinline__ void gather_next(const AdjArgs& j, long long N, const Offs& o, float (&ls)[Q]) {
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
        ls[s] = __ldg(j.lam_next + (long long)s * N + (o.x[1 + cx] + o.y[1 + cy] + o.z[1 + cz]));
    }
}

__device__ __forceinline__ void solid_vel(const RotorDev& R, float x, float y, float z, float us[3]) {
    const float r[3] = {x - R.cf[0], y - R.cf[1], z - R.cf[2]};
    const int ax = R.axis;
    if (ax == 0) { us[0] = 0.f; us[1] = -R.omega * r[2]; us[2] = R.omega * r[1]; }
    else if (ax == 1) { us[1] = 0.f; us[2] = -R.omega * r[0]; us[0] = R.omega * r[2]; }
    else { us[2] = 0.f; us[0] = -R.omega * r[1]; us[1] = R.omega * r[0]; }
}

// objective weight vector of a force cell: J_step = F . v, v = wT a + wQ (a x r)
__device__ __forceinline__ void force_weight(const RotorDev& R, float x, float y, float z, float v[3]) {
    const float r[3] = {x - R.cf[0], y - R.cf[1], z - R.cf[2]};
    const int ax = R.axis, b = (ax + 1) % 3, c = (ax + 2) % 3;
    v[ax] = R.wT;
    v[b] = -R.wQ * r[c];
    v[c] = R.wQ * r[b];
}

// ---------------------------------------------------------------------------
// cells outside every rotor box (and the open planes)
// ---------------------------------------------------------------------------
// D3Q19: at most 48 registers (10 blocks of 128 per SM, 16 bytes of spill), 2 %
// faster over a gradient sweep than the unbounded 56 (8 blocks)
template <int Q, int S, int PH, bool D0>
__global__ void __launch_bounds__(128, Q == 19 ? 10 : 1) adj_bulk_kernel(const StepArgs a, const AdjArgs j) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.n[0] || y >= a.n[1]) return;
    const int cell = (z * a.n[1] + y) * a.n[0] + x;
    for (int k = 0; k < a.nrot; ++k) {
        const unsigned dx = (unsigned)(x - a.rot[k].lo[0]), dy = (unsigned)(y - a.rot[k].lo[1]),
                       dz = (unsigned)(z - a.rot[k].lo[2]);
        if (dx < (unsigned)a.rot[k].n[0] && dy < (unsigned)a.rot[k].n[1] && dz < (unsigned)a.rot[k].n[2]) return;
    }
    const long long N = a.N;
    const int ax = a.flow_axis;
    const int ca = sel3(ax, x, y, z);
    const int na = sel3(ax, a.n[0], a.n[1], a.n[2]);
    const bool inlet = a.open && ca == 0;
    const bool outlet = a.open && ca == na - 1;
    if (inlet) {
        // f* = f^eq(1, u_in(t)): no dependence on the state
#pragma unroll
        for (int s = 0; s < Q; ++s) j.lam[(long long)s * N + cell] = 0.0f;
        return;
    }
    // away from the lattice faces every neighbour is at a fixed offset: one
    // per-thread index into per-slot shifted bases
    const bool shifted = x > 0 && x < a.n[0] - 1 && y > 0 && y < a.n[1] - 1 && z > 0 && z < a.n[2] - 1;
    Offs o;
    make_offs(a, x, y, z, o);
    float ls[Q];
    if (shifted) {
#pragma unroll
        for (int s = 0; s < Q; ++s) ls[s] = __ldg(j.lshift[s] + cell);
    } else {
        gather_next<Q>(j, N, o, ls);
    }
    const int nb = sel3(ax, a.n[1], a.n[2], a.n[0]);
    const int pl = sel3(ax, z, x, y) * nb + sel3(ax, y, z, x);
    if (outlet) {
        // f* = f^eq(1, u_plane), u_plane = upstream velocity of the previous step
        const float up[3] = {a.uplane_prev[pl], a.uplane_prev[a.nplane + pl], a.uplane_prev[2 * a.nplane + pl]};
        float ub[3];
        equilibrium_vjp<Q>(ls, up, ub);
        j.gup_prev[pl] = ub[0];
        j.gup_prev[a.nplane + pl] = ub[1];
        j.gup_prev[2 * a.nplane + pl] = ub[2];
#pragma unroll
        for (int s = 0; s < Q; ++s) j.lam[(long long)s * N + cell] = 0.0f;
        return;
    }
    float g[Q];
    if (shifted && PH == 1) {
        using T = typename Store<S>::T;
#pragma unroll
        for (int s = 0; s < Q; ++s) g[s] = Store<S>::ld(static_cast<const T*>(a.rshift[s]) + cell);
    } else {
        load_pre<Q, S, PH>(a, cell, o, g);
    }
    float gd, guB[3], gS[6], u[3], rho;
    if (D0) {
        Band B;
        B.d = a.d0[cell];
        B.uB[0] = B.uB[1] = B.uB[2] = 0.0f;
        B.sigma = 1.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) B.S[k] = 0.0f;
        collide_vjp<Q, true>(g, B, a.tau_mo, a.Ksmag, ls, gd, guB, gS, u, rho);
    } else {
        Band B0;
        collide_vjp<Q, false>(g, B0, a.tau_mo, a.Ksmag, ls, gd, guB, gS, u, rho);
    }
    if (j.dJdd0) j.dJdd0[cell] += gd;
    if (a.open && ca == na - 2) {
        // this cell's velocity is the outlet's u_plane of the next step
        const float inv = 1.0f / rho;
        const float gu[3] = {j.gup_cur[pl] * inv, j.gup_cur[a.nplane + pl] * inv, j.gup_cur[2 * a.nplane + pl] * inv};
        const float gu_u = gu[0] * u[0] + gu[1] * u[1] + gu[2] * u[2];
#pragma unroll
        for (int s = 0; s < Q; ++s) {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            ls[s] += float(cx) * gu[0] + float(cy) * gu[1] + float(cz) * gu[2] - gu_u;
        }
    }
#pragma unroll
    for (int s = 0; s < Q; ++s) j.lam[(long long)s * N + cell] = ls[s];
}

// ---------------------------------------------------------------------------
// the box of one rotor: band collision, momentum-exchange transpose, pitch
// ---------------------------------------------------------------------------
template <int Q, int S, int PH, bool D0>
__global__ void __launch_bounds__(128) adj_box_kernel(const StepArgs a, const AdjArgs j, int rk, int force_on) {
    const RotorDev& R = a.rot[rk];
    const int bx = blockIdx.x * blockDim.x + threadIdx.x;
    const int by = blockIdx.y * blockDim.y + threadIdx.y;
    const int bz = blockIdx.z;
    const bool valid = bx < R.n[0] && by < R.n[1];
    double pv = 0.0;
    if (valid) {
        const int x = R.lo[0] + bx, y = R.lo[1] + by, z = R.lo[2] + bz;
        const int cell = (z * a.n[1] + y) * a.n[0] + x;
        const long long bi = ((long long)bz * R.n[1] + by) * R.n[0] + bx;
        const long long N = a.N, BC = R.box_cells;
        Offs o;
        make_offs(a, x, y, z, o);
        float ls[Q];
        gather_next<Q>(j, N, o, ls);
        const uint8_t fl = R.flags[bi];
        if (force_on) {
            // transpose of the momentum exchange over the force cells (force_kernel)
            if (fl & FL_B) {
                float us[3], v[3];
                solid_vel(R, (float)x, (float)y, (float)z, us);
                force_weight(R, (float)x, (float)y, (float)z, v);
                const float uv = us[0] * v[0] + us[1] * v[1] + us[2] * v[2];
#pragma unroll
                for (int s = 1; s < Q; ++s) {
                    const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
                    ls[s] -= float(cx) * v[0] + float(cy) * v[1] + float(cz) * v[2] - uv;
                }
            }
#pragma unroll
            for (int s = 1; s < Q; ++s) {
                const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
                const int nx = bx + cx, ny = by + cy, nz = bz + cz;
                if (nx < 0 || ny < 0 || nz < 0 || nx >= R.n[0] || ny >= R.n[1] || nz >= R.n[2]) continue;
                if (!(R.flags[((long long)nz * R.n[1] + ny) * R.n[0] + nx] & FL_B)) continue;
                float us[3], v[3];
                const float X = (float)(x + cx), Y = (float)(y + cy), Z = (float)(z + cz);
                solid_vel(R, X, Y, Z, us);
                force_weight(R, X, Y, Z, v);
                ls[s] += float(cx) * v[0] + float(cy) * v[1] + float(cz) * v[2] -
                         (us[0] * v[0] + us[1] * v[1] + us[2] * v[2]);
            }
        }
        float g[Q];
        load_pre<Q, S, PH>(a, cell, o, g);
        Band B;
        const float d0 = D0 ? a.d0[cell] : 1.0f;
        B.d = d0 * R.d[bi];
        if (fl & FL_B) {
            solid_vel(R, (float)x, (float)y, (float)z, B.uB);
        } else {
            B.uB[0] = B.uB[1] = B.uB[2] = 0.0f;
        }
        // band parameters as the forward box collision takes them
        B.sigma = (fl & FL_B) ? a.sigma_band : 1.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) B.S[k] = 0.0f;
        const bool wall = a.wall_model && (fl & FL_W);
        const bool hybrid = !wall && (fl & FL_B) && a.sigma_band < 1.0f;
        if (wall) {
            const float* wm = R.wm + bi;
            B.uB[0] += wm[0];
            B.uB[1] += wm[BC];
            B.uB[2] += wm[2 * BC];
#pragma unroll
            for (int k = 0; k < 6; ++k) B.S[k] = wm[(3 + k) * BC];
            B.sigma = 0.0f;
        } else if (hybrid) {
            // S^FD of the band-strain kernel (taped with the wall-model rows)
            const float* wm = R.wm + bi;
#pragma unroll
            for (int k = 0; k < 6; ++k) B.S[k] = wm[(3 + k) * BC];
        }
        float gd, guB[3], gS[6], u[3], rho;
        collide_vjp<Q, true>(g, B, a.tau_mo, a.Ksmag, ls, gd, guB, gS, u, rho);
        if (j.dJdd0) j.dJdd0[cell] += gd * R.d[bi];
        if (fl & FL_B) pv = (double)(gd * d0 * R.ddp[bi]);
        if (wall) {
            R.gub[bi] = guB[0];
            R.gub[BC + bi] = guB[1];
            R.gub[2 * BC + bi] = guB[2];
        }
        if (wall || hybrid) {
#pragma unroll
            for (int k = 0; k < 6; ++k) R.gS[k * BC + bi] = gS[k];
        }
#pragma unroll
        for (int s = 0; s < Q; ++s) j.lam[(long long)s * N + cell] = ls[s];
    }
    // pitch contribution of the block: FP64 block sum, one atomic per block
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) pv += __shfl_down_sync(0xffffffffu, pv, off);
    __shared__ double sh[4];
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = pv;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double t = 0.0;
        const int nw = (blockDim.x * blockDim.y) >> 5;
        for (int w = 0; w < nw; ++w) t += sh[w];
        if (t != 0.0) {
            const unsigned b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            atomicAdd(R.pacc + b % PACC_SLOTS, t);
        }
    }
}

// ---------------------------------------------------------------------------
// reverse pass of the band strain (sigma < 1, Sec. 2.2): S^FD of a force cell
// off the wall set is (g + g^T) / 2 with g_mb = (u_b(x + e_m) - u_b(x - e_m)) / 2
// from the neighbours' pre-collision populations; its adjoint (the six stored
// components, from the box adjoint) goes to those velocities and through
// du_b/df_s = (c_sb - u_b) / rho to the neighbours' population adjoints
// (atomics: neighbouring band cells share neighbours)
// ---------------------------------------------------------------------------
template <int Q, int S, int PH>
__global__ void __launch_bounds__(128) adj_band_strain_kernel(const StepArgs a, const AdjArgs j) {
    const RotorDev& R = a.rot[blockIdx.y];
    int count = *((volatile int*)R.count);
    if ((long long)count > R.box_cells) count = (int)R.box_cells;
    const long long N = a.N, BC = R.box_cells;
    for (int idx = list_first(); idx < count; idx += list_stride()) {
        const long long bi = R.list[idx];
        if (a.wall_model && (R.flags[bi] & FL_W)) continue;
        const int bx = (int)(bi % R.n[0]);
        const long long r2 = bi / R.n[0];
        const int by = (int)(r2 % R.n[1]);
        const int bz = (int)(r2 / R.n[1]);
        // the forward left S^FD = 0 where the stencil leaves the box
        if (bx < 1 || by < 1 || bz < 1 || bx > R.n[0] - 2 || by > R.n[1] - 2 || bz > R.n[2] - 2) continue;
        const int x = R.lo[0] + bx, y = R.lo[1] + by, z = R.lo[2] + bz;
        float Sb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Sb[k] = R.gS[k * BC + bi];
        // adjoint of g_mb (xx yy zz xy xz yz storage order of S)
        const float G[3][3] = {{Sb[0], 0.5f * Sb[3], 0.5f * Sb[4]},
                               {0.5f * Sb[3], Sb[1], 0.5f * Sb[5]},
                               {0.5f * Sb[4], 0.5f * Sb[5], Sb[2]}};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int sg = side == 0 ? 1 : -1;
                const int xn = x + (m == 0) * sg, yn = y + (m == 1) * sg, zn = z + (m == 2) * sg;
                const int cn = (zn * a.n[1] + yn) * a.n[0] + xn;
                Offs o;
                make_offs(a, xn, yn, zn, o);
                float g[Q];
                load_pre<Q, S, PH>(a, cn, o, g);
                float rho = 1.0f, jm[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int s = 0; s < Q; ++s) {
                    rho += g[s];
                    jm[0] += float(cslot(Q, s, 0)) * g[s];
                    jm[1] += float(cslot(Q, s, 1)) * g[s];
                    jm[2] += float(cslot(Q, s, 2)) * g[s];
                }
                const float inv = 1.0f / rho;
                const float ub[3] = {0.5f * sg * G[m][0] * inv, 0.5f * sg * G[m][1] * inv, 0.5f * sg * G[m][2] * inv};
                const float ubu = (ub[0] * jm[0] + ub[1] * jm[1] + ub[2] * jm[2]) * inv;
#pragma unroll
                for (int s = 0; s < Q; ++s)
                    atomicAdd(j.lam + (long long)s * N + cn, float(cslot(Q, s, 0)) * ub[0] +
                                                                 float(cslot(Q, s, 1)) * ub[1] +
                                                                 float(cslot(Q, s, 2)) * ub[2] - ubu);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// reverse pass of the wall model (Sec. 2.2.1) on the wall-cell list
// ---------------------------------------------------------------------------
template <int Q, int S, int PH>
__global__ void __launch_bounds__(128) adj_wall_kernel(const StepArgs a, const AdjArgs j) {
    const RotorDev& R = a.rot[blockIdx.y];
    int count = *((volatile int*)(R.count + 1));
    if ((long long)count > R.box_cells) count = (int)R.box_cells;
    const long long N = a.N, BC = R.box_cells;
    // four lanes per wall cell: corners m = sub and sub + 4 are gathered and
    // scattered by lane sub, and lanes 0, 1, 2 (3 repeats 0) carry the
    // derivative of the Newton solve along seed 0, 1, 2; each group of four
    // takes the same list entries, so its branches are uniform
    const int sub = threadIdx.x & 3;
    const unsigned gm = 0xfu << (threadIdx.x & 28);
    const int gbase = threadIdx.x & 28;
    for (int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 2); idx < count;
         idx += (int)((gridDim.x * blockDim.x) >> 2)) {
        const long long bi = R.wlist[idx];
        const float phi = R.wphi[idx];
        const int which = R.wwhich[idx];
        const int bx = (int)(bi % R.n[0]);
        const long long r2 = bi / R.n[0];
        const int by = (int)(r2 % R.n[1]);
        const int bz = (int)(r2 / R.n[1]);
        const int x = R.lo[0] + bx, y = R.lo[1] + by, z = R.lo[2] + bz;
        float n[3], dn[3], dphi;
        rotor_normal_tan(R, which, x, y, z, n, dn);
        component_phi_tan(R, which, x, y, z, dphi);
        const bool far = phi > 0.5f;
        const float y1 = far ? phi : 0.5f;
        const float ys = a.wmYs;
        // the forward wall model's corner and weights (from the offset y_s n)
        const float dv[3] = {ys * n[0], ys * n[1], ys * n[2]};
        const int xc[3] = {x, y, z};
        int i0[3];
        float t[3];
        bool clamped[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float fl = floorf(dv[k]);
            i0[k] = xc[k] + (int)fl;
            t[k] = dv[k] - fl;
            clamped[k] = false;
            if (a.open && k == a.flow_axis) {
                if (i0[k] < 0) { i0[k] = 0; t[k] = 0.f; clamped[k] = true; }
                if (i0[k] > a.n[k] - 2) { i0[k] = a.n[k] - 2; t[k] = 1.f; clamped[k] = true; }
            }
        }
        if (sub == 0) R.gut_prev[bi] = 0.0;
        bool inside = true;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            inside = inside && i0[k] - R.lo[k] >= 0 && i0[k] + 1 - R.lo[k] < R.n[k];
        if (!inside) continue;   // the forward left this cell unmodelled (error word set)
        // this lane's corners h = 0, 1: m = sub + 4 h
        int cidx[2];
        float uc[2][3], irho[2], wc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = sub + 4 * h;
            const int cx = m & 1, cy = (m >> 1) & 1, cz = m >> 2;
            int p[3] = {i0[0] + cx, i0[1] + cy, i0[2] + cz};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (!(a.open && k == a.flow_axis)) p[k] = ((p[k] % a.n[k]) + a.n[k]) % a.n[k];
            const int c = (p[2] * a.n[1] + p[1]) * a.n[0] + p[0];
            cidx[h] = c;
            Offs o;
            make_offs(a, p[0], p[1], p[2], o);
            float g[Q];
            load_pre<Q, S, PH>(a, c, o, g);
            float drho, jj[3];
            moments01<Q>(g, drho, jj);
            irho[h] = 1.0f / (1.0f + drho);
            uc[h][0] = jj[0] * irho[h]; uc[h][1] = jj[1] * irho[h]; uc[h][2] = jj[2] * irho[h];
            const float wgt = (cx ? t[0] : 1.f - t[0]) * (cy ? t[1] : 1.f - t[1]) * (cz ? t[2] : 1.f - t[2]);
            wc[h] = wgt;
        }
        // the trilinear sum in corner order 0..7 with the forward wall model's
        // expression, so that the replayed Newton starts from the same |u_t|
        float us[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int h = m >> 2, src = gbase + (m & 3);
            const float wgt = __shfl_sync(gm, h ? wc[1] : wc[0], src);
            const float u0 = __shfl_sync(gm, h ? uc[1][0] : uc[0][0], src);
            const float u1 = __shfl_sync(gm, h ? uc[1][1] : uc[0][1], src);
            const float u2 = __shfl_sync(gm, h ? uc[1][2] : uc[0][2], src);
            us[0] += wgt * u0; us[1] += wgt * u1; us[2] += wgt * u2;
        }
        float usol[3];
        solid_vel(R, (float)x, (float)y, (float)z, usol);
        const float ur[3] = {us[0] - usol[0], us[1] - usol[1], us[2] - usol[2]};
        const float un = ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2];
        const float ut[3] = {ur[0] - un * n[0], ur[1] - un * n[1], ur[2] - un * n[2]};
        const float utm = sqrtf(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
        if (!(utm >= 1e-12f)) continue;   // the forward left this cell inactive
        const float th[3] = {ut[0] / utm, ut[1] / utm, ut[2] / utm};
        // forward Newton solves with derivatives along (|u_t|, y_sample, start value),
        // with the forward wall model's FP32 expressions
        const float ysamp = y1 + ys;
        const bool warm = R.tape_active[bi] != 0;
        const WallFn W = make_wallfn(a.wmE, a.wmK, a.nu, a.wmTol, a.wmMaxit);
        // seeds: 0 = |u_t|, 1 = y_sample, 2 = Newton start value, one per lane
        const int seed = sub == 3 ? 0 : sub;
        Dual<1> guess;
        if (warm) {
            const float gw = (float)R.tape_utau[bi];
            guess = seed == 2 ? dual_seed<1>(gw, 0) : dual_const<1>(gw);
        } else {
            // Eq. (guess): g0 = sqrt(nu |u_t| / y_s), d g0 / d|u_t| = nu / (2 y_s g0)
            const float g0 = sqrtf(utm / (ys * W.inv_nu));
            guess = seed == 0 ? dual_seed<1>(g0, 0, 1.0f / (2.0f * ys * W.inv_nu * g0)) : dual_const<1>(g0);
        }
        const Dual<1> utau = wall_newton_t(seed == 0 ? dual_seed<1>(utm, 0) : dual_const<1>(utm),
                                           seed == 1 ? dual_seed<1>(ysamp, 0) : dual_const<1>(ysamp), guess, W);
        float utd[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) utd[q] = __shfl_sync(gm, utau.d[0], gbase + q);
        const float y1p = y1 * utau.v * W.inv_nu;
        const Dual<1> up = spalding_uplus_t(dual_seed<1>(y1p, 0), W);
        const float uw = utau.v * up.v;
        const float gs = 0.5f * (utm - uw) / ys;
        // ---- reverse ----
        const float gdu[3] = {R.gub[bi], R.gub[BC + bi], R.gub[2 * BC + bi]};
        float Sb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Sb[k] = R.gS[k * BC + bi];
        // du = uw th
        float uwb = gdu[0] * th[0] + gdu[1] * th[1] + gdu[2] * th[2];
        float thb[3] = {uw * gdu[0], uw * gdu[1], uw * gdu[2]};
        // S = gs (2 th_a n_a | th_a n_b + n_a th_b)
        const float gsb = 2.0f * (Sb[0] * th[0] * n[0] + Sb[1] * th[1] * n[1] + Sb[2] * th[2] * n[2]) +
                          Sb[3] * (th[0] * n[1] + n[0] * th[1]) + Sb[4] * (th[0] * n[2] + n[0] * th[2]) +
                          Sb[5] * (th[1] * n[2] + n[1] * th[2]);
        thb[0] += gs * (2.0f * Sb[0] * n[0] + Sb[3] * n[1] + Sb[4] * n[2]);
        thb[1] += gs * (2.0f * Sb[1] * n[1] + Sb[3] * n[0] + Sb[5] * n[2]);
        thb[2] += gs * (2.0f * Sb[2] * n[2] + Sb[4] * n[0] + Sb[5] * n[1]);
        float nb[3] = {gs * (2.0f * Sb[0] * th[0] + Sb[3] * th[1] + Sb[4] * th[2]),
                       gs * (2.0f * Sb[1] * th[1] + Sb[3] * th[0] + Sb[5] * th[2]),
                       gs * (2.0f * Sb[2] * th[2] + Sb[4] * th[0] + Sb[5] * th[1])};
        // gs = (|u_t| - utau u+) / (2 y_s)
        float utmb = 0.5f * gsb / ys;
        const float uwdb = uwb - 0.5f * gsb / ys;
        float utaub = uwdb * up.v + (float)R.gut_next[bi];
        const float upb = uwdb * utau.v;
        // u+ = U(y1 utau / nu)
        const float y1pb = upb * up.d[0];
        utaub += y1pb * y1 * W.inv_nu;
        float y1b = y1pb * utau.v * W.inv_nu;
        // utau = Newton(|u_t|, y1 + y_s, start)
        utmb += utaub * utd[0];
        y1b += utaub * utd[1];
        if (sub == 0) R.gut_prev[bi] = warm ? (double)(utaub * utd[2]) : 0.0;
        // th = u_t / |u_t|
        const float td = thb[0] * th[0] + thb[1] * th[1] + thb[2] * th[2];
        float utb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) utb[k] = (thb[k] - td * th[k]) / utm + utmb * th[k];
        // u_t = u_r - (u_r . n) n
        const float utn = utb[0] * n[0] + utb[1] * n[1] + utb[2] * n[2];
        float urb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            urb[k] = utb[k] - utn * n[k];
            nb[k] -= un * utb[k] + utn * ur[k];
        }
        // u_s = sum_m w_m u_m (trilinear at x_s = x + y_s n)
        float xsb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = sub + 4 * h;
            const int cx = m & 1, cy = (m >> 1) & 1, cz = m >> 2;
            const float wx = cx ? t[0] : 1.f - t[0], wy = cy ? t[1] : 1.f - t[1], wz = cz ? t[2] : 1.f - t[2];
            const float wgt = wx * wy * wz;
            const float ucb[3] = {wgt * urb[0], wgt * urb[1], wgt * urb[2]};
            const float dot = uc[h][0] * urb[0] + uc[h][1] * urb[1] + uc[h][2] * urb[2];
            if (!clamped[0]) xsb[0] += (cx ? 1.f : -1.f) * wy * wz * dot;
            if (!clamped[1]) xsb[1] += (cy ? 1.f : -1.f) * wx * wz * dot;
            if (!clamped[2]) xsb[2] += (cz ? 1.f : -1.f) * wx * wy * dot;
            // u_m = j_m / rho_m: d u_m / d g_s = (c_s - u_m) / rho_m
            const float ir = irho[h];
            const float cu = (ucb[0] * uc[h][0] + ucb[1] * uc[h][1] + ucb[2] * uc[h][2]) * ir;
            float* lp = j.lam + cidx[h];
#pragma unroll
            for (int s = 0; s < Q; ++s) {
                const int sx = cslot(Q, s, 0), sy = cslot(Q, s, 1), sz = cslot(Q, s, 2);
                const float v = (float(sx) * ucb[0] + float(sy) * ucb[1] + float(sz) * ucb[2]) * ir - cu;
                if (v != 0.0f) atomicAdd(lp + (long long)s * N, v);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xsb[k] += __shfl_xor_sync(gm, xsb[k], 1);
            xsb[k] += __shfl_xor_sync(gm, xsb[k], 2);
            nb[k] += ys * xsb[k];
        }
        // pitch: through the normal and the wall distance y1 = max(phi, 1/2)
        double pg = (double)(nb[0] * dn[0] + nb[1] * dn[1] + nb[2] * dn[2]);
        if (far) pg += (double)(y1b * dphi);
        if (sub == 0) atomicAdd(R.pacc + (unsigned)idx % PACC_SLOTS, pg);
    }
}

// collision VJP of n independent cells (unit checks)
template <int Q>
__global__ void debug_collide_vjp_kernel(int n, const float* gin, const float* d, const float* uB, const float* sigma,
                                         const float* S, float tau_mo, float Ksmag, const float* lin, float* lout,
                                         float* gd_out, float* guB_out, float* gS_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float g[Q], l[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) { g[s] = gin[(long long)c * Q + s]; l[s] = lin[(long long)c * Q + s]; }
    float gd, guB[3], gS[6], u[3], rho;
    if (d) {
        Band B;
        B.d = d[c];
        B.uB[0] = uB[3 * c]; B.uB[1] = uB[3 * c + 1]; B.uB[2] = uB[3 * c + 2];
        B.sigma = sigma[c];
#pragma unroll
        for (int k = 0; k < 6; ++k) B.S[k] = S[6 * c + k];
        collide_vjp<Q, true>(g, B, tau_mo, Ksmag, l, gd, guB, gS, u, rho);
    } else {
        Band B0;
        collide_vjp<Q, false>(g, B0, tau_mo, Ksmag, l, gd, guB, gS, u, rho);
    }
#pragma unroll
    for (int s = 0; s < Q; ++s) lout[(long long)c * Q + s] = l[s];
    if (gd_out) gd_out[c] = gd;
    if (guB_out) for (int k = 0; k < 3; ++k) guB_out[3 * c + k] = guB[k];
    if (gS_out) for (int k = 0; k < 6; ++k) gS_out[6 * c + k] = gS[k];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
dim3 cell_block(int nx) {
    if (nx >= 128) return dim3(128, 1, 1);
    const int bx = ((nx + 31) / 32) * 32;
    return dim3(bx, 128 / bx >= 1 ? 128 / bx : 1, 1);
}

// cells outside every rotor box (and the open planes)
template <int Q, int S>
cudaError_t launch_adj_bulk_t(const StepArgs& a, const AdjArgs& j, cudaStream_t s) {
    const dim3 blk = cell_block(a.n[0]);
    const dim3 grd((a.n[0] + blk.x - 1) / blk.x, (a.n[1] + blk.y - 1) / blk.y, a.n[2]);
    if (a.d0) {
        if (a.phase == 0) adj_bulk_kernel<Q, S, 0, true><<<grd, blk, 0, s>>>(a, j);
        else adj_bulk_kernel<Q, S, 1, true><<<grd, blk, 0, s>>>(a, j);
    } else {
        if (a.phase == 0) adj_bulk_kernel<Q, S, 0, false><<<grd, blk, 0, s>>>(a, j);
        else adj_bulk_kernel<Q, S, 1, false><<<grd, blk, 0, s>>>(a, j);
    }
    return cudaGetLastError();
}

// the rotor boxes, then the wall-model reverse pass
template <int Q, int S>
cudaError_t launch_adj_box_t(const StepArgs& a, const AdjArgs& j, bool force_on, cudaStream_t s) {
    for (int k = 0; k < a.nrot; ++k) {
        const int* n = a.rot[k].n;
        const dim3 blk = cell_block(n[0]);
        const dim3 grd((n[0] + blk.x - 1) / blk.x, (n[1] + blk.y - 1) / blk.y, n[2]);
        const int fo = force_on ? 1 : 0;
        if (a.d0) {
            if (a.phase == 0) adj_box_kernel<Q, S, 0, true><<<grd, blk, 0, s>>>(a, j, k, fo);
            else adj_box_kernel<Q, S, 1, true><<<grd, blk, 0, s>>>(a, j, k, fo);
        } else {
            if (a.phase == 0) adj_box_kernel<Q, S, 0, false><<<grd, blk, 0, s>>>(a, j, k, fo);
            else adj_box_kernel<Q, S, 1, false><<<grd, blk, 0, s>>>(a, j, k, fo);
        }
    }
    if (a.nrot > 0 && a.wall_model) {
        const dim3 grd(WALL_GROUP_BLOCKS, a.nrot);
        if (a.phase == 0) adj_wall_kernel<Q, S, 0><<<grd, WALL_THREADS, 0, s>>>(a, j);
        else adj_wall_kernel<Q, S, 1><<<grd, WALL_THREADS, 0, s>>>(a, j);
    }
    if (a.nrot > 0 && a.sigma_band < 1.0f) {
        const dim3 grd(WALL_BLOCKS, a.nrot);
        if (a.phase == 0) adj_band_strain_kernel<Q, S, 0><<<grd, WALL_THREADS, 0, s>>>(a, j);
        else adj_band_strain_kernel<Q, S, 1><<<grd, WALL_THREADS, 0, s>>>(a, j);
    }
    return cudaGetLastError();
}

#define HL_ADJ_DISPATCH(Q, S, FN, ...)                                        \
    do {                                                                      \
        if (Q == 19 && S == ST_F32) return FN<19, ST_F32>(__VA_ARGS__);       \
        if (Q == 19 && S == ST_F16S) return FN<19, ST_F16S>(__VA_ARGS__);     \
        if (Q == 19 && S == ST_BF16S) return FN<19, ST_BF16S>(__VA_ARGS__);   \
        if (Q == 27 && S == ST_F32) return FN<27, ST_F32>(__VA_ARGS__);       \
        if (Q == 27 && S == ST_F16S) return FN<27, ST_F16S>(__VA_ARGS__);     \
        if (Q == 27 && S == ST_BF16S) return FN<27, ST_BF16S>(__VA_ARGS__);   \
        return cudaErrorInvalidValue;                                         \
    } while (0)

cudaError_t launch_adj_bulk(int Q, int S, const StepArgs& a, const AdjArgs& j, cudaStream_t s) {
    HL_ADJ_DISPATCH(Q, S, launch_adj_bulk_t, a, j, s);
}
cudaError_t launch_adj_box(int Q, int S, const StepArgs& a, const AdjArgs& j, bool force_on, cudaStream_t s) {
    HL_ADJ_DISPATCH(Q, S, launch_adj_box_t, a, j, force_on, s);
}

template <int Q, int S>
cudaError_t launch_relayout_t(const StepArgs& a, const void* src, void* dst, bool to_eso, cudaStream_t s) {
    const dim3 grd((a.n[0] + 127) / 128, a.n[1], a.n[2]);
    if (a.phase == 0) relayout_kernel<Q, S, 0><<<grd, 128, 0, s>>>(a, src, dst, to_eso ? 1 : 0);
    else relayout_kernel<Q, S, 1><<<grd, 128, 0, s>>>(a, src, dst, to_eso ? 1 : 0);
    return cudaGetLastError();
}
cudaError_t launch_relayout(int Q, int S, const StepArgs& a, const void* src, void* dst, bool to_eso,
                            cudaStream_t s) {
    HL_ADJ_DISPATCH(Q, S, launch_relayout_t, a, src, dst, to_eso, s);
}

cudaError_t launch_xhalves(int Q, int S, const StepArgs& a, const void* src, void* dst, bool to_halves,
                           cudaStream_t st) {
    const dim3 grd((a.n[0] + 127) / 128, a.n[1], a.n[2]);
    if (S == ST_F32) xhalves_kernel<ST_F32><<<grd, 128, 0, st>>>(a, Q, src, dst, to_halves ? 1 : 0);
    else xhalves_kernel<ST_F16S><<<grd, 128, 0, st>>>(a, Q, src, dst, to_halves ? 1 : 0);   // 16-bit words
    return cudaGetLastError();
}

// unit check of the packed bulk collision: cells 2k and 2k+1 of [n][q] in one thread
template <int Q>
__global__ void debug_collide_pair_kernel(int n, const float* gin, float tau_mo, float Ksmag, float* gout) {
    const int c = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c + 1 >= n) return;
    F2 g[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) g[s] = {make_float2(gin[(long long)c * Q + s], gin[(long long)(c + 1) * Q + s])};
    F2 u[3];
    collide_pair<Q>(g, tau_mo, Ksmag, u);
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        gout[(long long)c * Q + s] = g[s].v.x;
        gout[(long long)(c + 1) * Q + s] = g[s].v.y;
    }
}

}  // namespace
}  // namespace hl

// ===========================================================================
// host driver
// ===========================================================================
using namespace hl;
using namespace hl::host;

namespace {

long long pop_bytes(const hl_lattice* lat) {
    return (long long)lat->cfg.q * lat->N * store_bytes(lat->cfg.storage);
}

// one checkpoint: populations, both outlet planes (in buffer order), and
// per rotor the wall-model state (u_tau, active)
size_t ckpt_bytes(const hl_lattice* lat) {
    size_t o = align_up((size_t)pop_bytes(lat));
    o += 2 * align_up(sizeof(float) * 3 * plane_cells(lat->cfg));
    for (int k = 0; k < lat->nrot; ++k) {
        o += align_up(sizeof(double) * lat->rot[k].dev.box_cells);
        o += align_up((size_t)lat->rot[k].dev.box_cells);
    }
    return o;
}

// per step of a segment: the outlet velocity read by the step and the
// wall-model state at its start
// layout of one step's tape entry: outlet plane | per rotor: u_tau, active
// (at the start of the step), wall-model output of the step [9][box]
struct SmallOff {
    size_t utau[MAXROT], active[MAXROT], wm[MAXROT];
};

size_t small_layout(const hl_lattice* lat, SmallOff* so) {
    size_t o = align_up(sizeof(float) * 3 * plane_cells(lat->cfg));
    for (int k = 0; k < lat->nrot; ++k) {
        const long long b = lat->rot[k].dev.box_cells;
        if (so) so->utau[k] = o;
        o += align_up(sizeof(double) * b);
        if (so) so->active[k] = o;
        o += align_up((size_t)b);
        if (so) so->wm[k] = o;
        o += align_up(sizeof(float) * 9 * b);
    }
    return o;
}

size_t small_bytes(const hl_lattice* lat) { return small_layout(lat, nullptr); }

size_t rotor_adj_bytes(const hl_lattice* lat, int k) {
    const long long b = lat->rot[k].dev.box_cells;
    return align_up(sizeof(float) * b) + align_up(sizeof(float) * 3 * b) + align_up(sizeof(float) * 6 * b) +
           2 * align_up(sizeof(double) * b) + align_up(sizeof(double) * PACC_SLOTS) + align_up(sizeof(double) * 12);
}

struct GradLayout {
    int n_ck;
    size_t ck, seg, small, lam, gup, radj[MAXROT], total;
};

GradLayout grad_layout(const hl_lattice* lat, int steps, int K) {
    GradLayout G{};
    G.n_ck = (steps + K - 1) / K;
    size_t o = 0;
    G.ck = o; o += (size_t)(G.n_ck + 1) * ckpt_bytes(lat);
    G.seg = o; o += (size_t)(K - 1) * align_up((size_t)pop_bytes(lat));
    G.small = o; o += (size_t)K * small_bytes(lat);
    G.lam = o; o += 2 * align_up(sizeof(float) * lat->cfg.q * lat->N);
    G.gup = o; o += 2 * align_up(sizeof(float) * 3 * plane_cells(lat->cfg));
    for (int k = 0; k < lat->nrot; ++k) {
        G.radj[k] = o;
        o += rotor_adj_bytes(lat, k);
    }
    G.total = o;
    return G;
}

float* uplane_prev_of(hl_lattice* lat, long long t) { return lat->uplane[(t + 1) & 1]; }

// copy the lattice state (populations, outlet planes, wall-model state) to
// or from a checkpoint
hl_status ckpt_copy(hl_lattice* lat, char* ck, bool save, bool with_pops) {
    const cudaMemcpyKind kd = cudaMemcpyDeviceToDevice;
    cudaStream_t st = lat->stream;
    size_t o = 0;
    const size_t pb = (size_t)pop_bytes(lat);
    if (with_pops)
        HL_CUDA(lat, save ? cudaMemcpyAsync(ck, lat->f, pb, kd, st) : cudaMemcpyAsync(lat->f, ck, pb, kd, st));
    o = align_up(pb);
    const size_t plb = sizeof(float) * 3 * plane_cells(lat->cfg);
    for (int b = 0; b < 2; ++b) {
        HL_CUDA(lat, save ? cudaMemcpyAsync(ck + o, lat->uplane[b], plb, kd, st)
                          : cudaMemcpyAsync(lat->uplane[b], ck + o, plb, kd, st));
        o += align_up(plb);
    }
    for (int k = 0; k < lat->nrot; ++k) {
        RotorDev& D = lat->rot[k].dev;
        const size_t ub = sizeof(double) * D.box_cells;
        HL_CUDA(lat, save ? cudaMemcpyAsync(ck + o, D.utau, ub, kd, st) : cudaMemcpyAsync(D.utau, ck + o, ub, kd, st));
        o += align_up(ub);
        const size_t ab = (size_t)D.box_cells;
        HL_CUDA(lat, save ? cudaMemcpyAsync(ck + o, D.active, ab, kd, st)
                          : cudaMemcpyAsync(D.active, ck + o, ab, kd, st));
        o += align_up(ab);
    }
    return HL_OK;
}

// the step's small state: the outlet velocity it reads (saved on the
// lattice stream, which writes it) and the wall-model state at its start
// (saved on the box stream bs, which owns it)
hl_status small_save(hl_lattice* lat, char* sm, long long t, cudaStream_t bs) {
    const cudaMemcpyKind kd = cudaMemcpyDeviceToDevice;
    SmallOff so;
    small_layout(lat, &so);
    HL_CUDA(lat, cudaMemcpyAsync(sm, uplane_prev_of(lat, t), sizeof(float) * 3 * plane_cells(lat->cfg), kd,
                                 lat->stream));
    for (int k = 0; k < lat->nrot; ++k) {
        RotorDev& D = lat->rot[k].dev;
        HL_CUDA(lat, cudaMemcpyAsync(sm + so.utau[k], D.utau, sizeof(double) * D.box_cells, kd, bs));
        HL_CUDA(lat, cudaMemcpyAsync(sm + so.active[k], D.active, (size_t)D.box_cells, kd, bs));
    }
    return HL_OK;
}

// the wall-model rows of a step (u^B and S^WM of wall cells, S^FD of hybrid
// band cells) live in the step's tape entry: the recompute's wall model and
// band strain write them there and its box collision reads them there, and
// the reverse step reads them in place (no copies)
void wm_rows_in_tape(hl_lattice* lat, StepArgs& a, char* sm) {
    SmallOff so;
    small_layout(lat, &so);
    for (int k = 0; k < lat->nrot; ++k) a.rot[k].wm = reinterpret_cast<float*>(sm + so.wm[k]);
}

// arguments of step t with explicit read / write population buffers
StepArgs args_at(hl_lattice* lat, long long t, void* rd, void* wr) {
    const long long keep = lat->t;
    lat->t = t;
    StepArgs a = make_args(lat);
    lat->t = keep;
    const size_t sb = (size_t)lat->N * store_bytes(lat->cfg.storage);
    for (int q = 0; q < lat->cfg.q; ++q) {
        a.f = rd;
        a.slot[q] = static_cast<char*>(rd) + q * sb;
        a.wslot[q] = static_cast<char*>(wr) + q * sb;
    }
    set_shifted_bases(&a, lat->cfg.q, store_bytes(lat->cfg.storage));
    return a;
}

hl_status fork_aux(hl_lattice* lat) {
    if (!(lat->have_aux && lat->nrot > 0)) return HL_OK;
    HL_CUDA(lat, cudaEventRecord(lat->ev_fork, lat->stream));
    HL_CUDA(lat, cudaStreamWaitEvent(lat->aux, lat->ev_fork, 0));
    return HL_OK;
}

hl_status join_aux(hl_lattice* lat) {
    if (!(lat->have_aux && lat->nrot > 0)) return HL_OK;
    HL_CUDA(lat, cudaEventRecord(lat->ev_join, lat->aux));
    HL_CUDA(lat, cudaStreamWaitEvent(lat->stream, lat->ev_join, 0));
    HL_CUDA(lat, cudaEventRecord(lat->ev_join_f, lat->fst));
    HL_CUDA(lat, cudaStreamWaitEvent(lat->stream, lat->ev_join_f, 0));
    return HL_OK;
}

// the lattice state between the esoteric twist and the AA layout of the
// current step, through a scratch buffer of the gradient workspace
hl_status relayout_state(hl_lattice* lat, void* scratch, bool to_eso) {
    const StepArgs a = make_args(lat);
    if (lat->cfg.layout == 2) {
        // the AA layout with x halves <-> the AA layout
        HL_CUDA(lat, launch_xhalves(lat->cfg.q, lat->cfg.storage, a, lat->f, scratch, to_eso, lat->stream));
    } else {
        HL_CUDA(lat, launch_relayout(lat->cfg.q, lat->cfg.storage, a, lat->f, scratch, to_eso, lat->stream));
    }
    HL_CUDA(lat, cudaMemcpyAsync(lat->f, scratch, (size_t)pop_bytes(lat), cudaMemcpyDeviceToDevice, lat->stream));
    return HL_OK;
}

}  // namespace

extern "C" {

hl_status hl_grad_workspace_size(const hl_lattice* lat, int steps, int ckpt_every, size_t* bytes) {
    if (!lat || steps < 1 || ckpt_every < 1 || !bytes) return HL_ERR_ARG;
    *bytes = grad_layout(lat, steps, ckpt_every).total;
    return HL_OK;
}

}  // extern "C"

// arguments and lattice state hl_grad accepts
static hl_status grad_check(hl_lattice* lat, int steps, int avg_last, int ckpt_every, const double* w_thrust,
                            const double* w_torque, const void* d_work, size_t bytes) {
    if (steps < 1 || avg_last < 1 || avg_last > steps || ckpt_every < 1 || !w_thrust || !w_torque || !d_work)
        return fail(lat, HL_ERR_ARG, "hl_grad: invalid arguments");
    if (reinterpret_cast<size_t>(d_work) % ALIGN) return fail(lat, HL_ERR_ARG, "hl_grad: workspace not aligned");
    for (int k = 0; k < lat->nrot; ++k)
        if (lat->rot[k].driven)
            return fail(lat, HL_ERR_STATE, "hl_grad: gradients cover prescribed rotation only (rotor is torque-driven)");
    if (bytes < grad_layout(lat, steps, ckpt_every).total)
        return fail(lat, HL_ERR_WORKSPACE, "hl_grad: workspace too small");
    return HL_OK;
}

// the sweep on a lattice in the AA layout
static hl_status grad_aa(hl_lattice* lat, int steps, int avg_last, int ckpt_every, const double* w_thrust,
                         const double* w_torque, double* J, double* dJ_dpitch, float* d_dJ_dd0, void* d_work,
                         size_t bytes) {
    hl_status rc = grad_check(lat, steps, avg_last, ckpt_every, w_thrust, w_torque, d_work, bytes);
    if (rc != HL_OK) return rc;
    const int T = steps, K = ckpt_every, na = avg_last;
    const GradLayout G = grad_layout(lat, T, K);
    char* ws = static_cast<char*>(d_work);
    const int Q = lat->cfg.q, S = lat->cfg.storage;
    cudaStream_t st = lat->stream;
    const long long t0 = lat->t;
    const size_t ckb = ckpt_bytes(lat), smb = small_bytes(lat), pb = align_up((size_t)pop_bytes(lat));
    const size_t plb = sizeof(float) * 3 * plane_cells(lat->cfg);
    // the wall-model rows (u^B and S^WM of wall cells, S^FD of hybrid band
    // cells) are taped per step when either is in use
    const bool tape_wm = lat->cfg.wall_model || lat->cfg.sigma_band < 1.0;

    // per-rotor adjoint arrays
    struct RAdj { float *ddp, *gub, *gS; double *gut[2], *pacc, *accsnap; } ra[MAXROT];
    for (int k = 0; k < lat->nrot; ++k) {
        const long long b = lat->rot[k].dev.box_cells;
        char* p = ws + G.radj[k];
        ra[k].ddp = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * b);
        ra[k].gub = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * 3 * b);
        ra[k].gS = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * 6 * b);
        ra[k].gut[0] = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * b);
        ra[k].gut[1] = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * b);
        ra[k].pacc = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * PACC_SLOTS);
        ra[k].accsnap = reinterpret_cast<double*>(p);
    }

    // ---- forward pass: checkpoints every K steps, force sums at the window start ----
    for (int s = 0; s < T;) {
        if (s % K == 0) {
            if ((rc = ckpt_copy(lat, ws + G.ck + (size_t)(s / K) * ckb, true, true)) != HL_OK) return rc;
        }
        if (s == T - na)
            for (int k = 0; k < lat->nrot; ++k)
                HL_CUDA(lat, cudaMemcpyAsync(ra[k].accsnap, lat->rot[k].dev.acc, 12 * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
        int n = K - s % K;
        if (s < T - na && s + n > T - na) n = T - na - s;
        if (s + n > T) n = T - s;
        if ((rc = hl_step_async(lat, n)) != HL_OK) return rc;
        s += n;
    }
    if ((rc = ckpt_copy(lat, ws + G.ck + (size_t)G.n_ck * ckb, true, true)) != HL_OK) return rc;
    if ((rc = read_error_word(lat)) != HL_OK) return rc;
    // J from the force sums at the window start and end
    {
        double Jv = 0.0;
        for (int k = 0; k < lat->nrot; ++k) {
            double a0[12], a1[12];
            HL_CUDA(lat, cudaMemcpyAsync(a0, ra[k].accsnap, sizeof a0, cudaMemcpyDeviceToHost, st));
            HL_CUDA(lat, cudaMemcpyAsync(a1, lat->rot[k].dev.acc, sizeof a1, cudaMemcpyDeviceToHost, st));
            HL_CUDA(lat, cudaStreamSynchronize(st));
            const int ax = lat->rot[k].geom.axis;
            Jv += (w_thrust[k] * (a1[6 + ax] - a0[6 + ax]) + w_torque[k] * (a1[9 + ax] - a0[9 + ax])) / na;
        }
        if (J) *J = Jv;
    }

    // ---- reverse sweep ----
    float* lam[2] = {reinterpret_cast<float*>(ws + G.lam),
                     reinterpret_cast<float*>(ws + G.lam + align_up(sizeof(float) * Q * lat->N))};
    float* gup[2] = {reinterpret_cast<float*>(ws + G.gup), reinterpret_cast<float*>(ws + G.gup + align_up(plb))};
    HL_CUDA(lat, cudaMemsetAsync(ws + G.lam, 0, 2 * align_up(sizeof(float) * Q * lat->N), st));
    HL_CUDA(lat, cudaMemsetAsync(ws + G.gup, 0, 2 * align_up(plb), st));
    for (int k = 0; k < lat->nrot; ++k) HL_CUDA(lat, cudaMemsetAsync(ws + G.radj[k], 0, rotor_adj_bytes(lat, k), st));
    if (d_dJ_dd0) HL_CUDA(lat, cudaMemsetAsync(d_dJ_dd0, 0, sizeof(float) * lat->N, st));
    // streams and events of the reverse sweep (the box chain on the aux stream)
    const bool two = lat->have_aux && lat->nrot > 0;
    cudaStream_t bs = two ? lat->aux : st;
    struct Events {
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evs;
    for (int i = 0; two && i < 4; ++i)
        HL_CUDA(lat, cudaEventCreateWithFlags(&evs.e[i], cudaEventDisableTiming));
    cudaEvent_t ev_bulk[2] = {evs.e[0], evs.e[1]}, ev_box[2] = {evs.e[2], evs.e[3]};
    // offsets of the neighbour x + c_s in the adjoint arrays (interior cells)
    long long lshift_off[27];
    {
        std::vector<int> cv(3 * Q);
        std::vector<double> wv(Q);
        hl_velocity_set(Q, cv.data(), wv.data());
        for (int sl = 0; sl < Q; ++sl)
            lshift_off[sl] = cv[3 * sl] + (long long)cv[3 * sl + 1] * lat->cfg.nx +
                             (long long)cv[3 * sl + 2] * lat->cfg.nx * lat->cfg.ny;
    }
    int ln = 0;      // lam[ln] = adjoint of the populations at t + 1
    int gc = 0;      // gup[gc] = adjoint of the outlet velocity written at t
    int uc = 0;      // gut[uc] = adjoint of the friction velocity of step t
    for (int m = G.n_ck - 1; m >= 0; --m) {
        const long long ts = t0 + (long long)m * K;
        const int L = (int)std::min<long long>(K, T - (long long)m * K);
        char* ck = ws + G.ck + (size_t)m * ckb;
        auto buf = [&](int jj) -> void* { return jj == 0 ? (void*)ck : (void*)(ws + G.seg + (size_t)(jj - 1) * pb); };
        // recompute the segment out of place, recording each step's small state;
        // the cell lists start empty (the last reverse step left them filled)
        if ((rc = ckpt_copy(lat, ck, false, false)) != HL_OK) return rc;
        for (int k = 0; k < lat->nrot; ++k) HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.count, 0, COUNT_BYTES, st));
        if ((rc = fork_aux(lat)) != HL_OK) return rc;
        for (int jj = 0; jj < L; ++jj) {
            const long long t = ts + jj;
            char* sm = ws + G.small + (size_t)jj * smb;
            if ((rc = small_save(lat, sm, t, bs)) != HL_OK) return rc;
            if (jj < L - 1) {
                StepArgs a = args_at(lat, t, buf(jj), buf(jj + 1));
                if (tape_wm) wm_rows_in_tape(lat, a, sm);
                if ((rc = issue_step(lat, a, false)) != HL_OK) return rc;
            } else if (lat->nrot > 0) {
                // the segment's last state is not advanced: run its embedding and
                // wall model alone
                StepArgs a = args_at(lat, t, buf(jj), buf(jj));
                if (tape_wm) wm_rows_in_tape(lat, a, sm);
                a.part = 0;
                HL_CUDA(lat, launch_band(Q, S, a, bs));
                HL_CUDA(lat, launch_band_strain(Q, S, a, bs));
                if (lat->cfg.wall_model) HL_CUDA(lat, launch_wall(Q, S, a, bs));
                for (int k = 0; k < lat->nrot; ++k)
                    HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.count, 0, COUNT_BYTES, bs));
            }
        }
        // both halves of the reverse step read states written by both halves
        // of the recomputation
        if ((rc = join_aux(lat)) != HL_OK) return rc;
        if ((rc = fork_aux(lat)) != HL_OK) return rc;
        // adjoint steps of the segment, last to first: the cells outside the
        // rotor boxes on the lattice stream, the box chain (embedding, wall
        // model, box adjoint, wall-model adjoint) on the box stream; step t
        // gathers the adjoint of step t + 1 from both halves and overwrites
        // the buffer step t + 1 read, so each half waits for the other's t + 1
        for (int jj = L - 1; jj >= 0; --jj) {
            const long long t = ts + jj;
            const int p = (int)(t & 1), q = p ^ 1;
            char* sm = ws + G.small + (size_t)jj * smb;
            StepArgs a = args_at(lat, t, buf(jj), buf(jj));
            a.uplane_prev = reinterpret_cast<const float*>(sm);
            a.tangent = 1;
            const bool force_on = t >= t0 + T - na;
            AdjArgs adj;
            adj.lam_next = lam[ln];
            for (int sl = 0; sl < Q; ++sl)
                adj.lshift[sl] = lam[ln] + (long long)sl * lat->N + lshift_off[sl];
            adj.lam = lam[ln ^ 1];
            adj.dJdd0 = d_dJ_dd0;
            adj.gup_cur = gup[gc];
            adj.gup_prev = gup[gc ^ 1];
            // lattice stream: bulk cells
            if (two) HL_CUDA(lat, cudaStreamWaitEvent(st, ev_box[q], 0));
            HL_CUDA(lat, launch_adj_bulk(Q, S, a, adj, st));
            if (two) HL_CUDA(lat, cudaEventRecord(ev_bulk[p], st));
            // box stream: forward quantities of step t, then the box adjoint
            if (lat->nrot > 0) {
                // the step's wall-model output is read from the tape (the linearisation point)
                if (tape_wm) wm_rows_in_tape(lat, a, sm);
                SmallOff so;
                small_layout(lat, &so);
                for (int k = 0; k < lat->nrot; ++k) {
                    RotorDev& D = a.rot[k];
                    D.ddp = ra[k].ddp;
                    D.gub = ra[k].gub;
                    D.gS = ra[k].gS;
                    D.tape_utau = reinterpret_cast<const double*>(sm + so.utau[k]);
                    D.tape_active = reinterpret_cast<const uint8_t*>(sm + so.active[k]);
                    D.gut_next = ra[k].gut[uc];
                    D.gut_prev = ra[k].gut[uc ^ 1];
                    D.pacc = ra[k].pacc;
                    D.wT = force_on ? (float)(w_thrust[k] / na) : 0.0f;
                    D.wQ = force_on ? (float)(w_torque[k] / na) : 0.0f;
                    HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.count, 0, COUNT_BYTES, bs));
                    // only this step's wall cells hand an adjoint to the previous step's u_tau
                    HL_CUDA(lat, cudaMemsetAsync(ra[k].gut[uc ^ 1], 0, sizeof(double) * D.box_cells, bs));
                }
                a.part = 0;
                HL_CUDA(lat, launch_band(Q, S, a, bs));
                if (two) HL_CUDA(lat, cudaStreamWaitEvent(bs, ev_bulk[q], 0));
                HL_CUDA(lat, launch_adj_box(Q, S, a, adj, force_on, bs));
                if (two) HL_CUDA(lat, cudaEventRecord(ev_box[p], bs));
            }
            ln ^= 1;
            gc ^= 1;
            uc ^= 1;
        }
        if ((rc = join_aux(lat)) != HL_OK) return rc;
    }
    // the lattice ends where the forward pass ended
    if ((rc = ckpt_copy(lat, ws + G.ck + (size_t)G.n_ck * ckb, false, true)) != HL_OK) return rc;
    for (int k = 0; k < lat->nrot; ++k) HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.count, 0, COUNT_BYTES, st));
    for (int k = 0; k < lat->nrot; ++k) {
        double pacc[PACC_SLOTS];
        HL_CUDA(lat, cudaMemcpyAsync(pacc, ra[k].pacc, sizeof pacc, cudaMemcpyDeviceToHost, st));
        HL_CUDA(lat, cudaStreamSynchronize(st));
        double s = 0.0;
        for (int i = 0; i < PACC_SLOTS; ++i) s += pacc[i];
        if (dJ_dpitch) dJ_dpitch[k] = s;
    }
    return read_error_word(lat);
}

extern "C" {

hl_status hl_grad(hl_lattice* lat, int steps, int avg_last, int ckpt_every, const double* w_thrust,
                  const double* w_torque, double* J, double* dJ_dpitch, float* d_dJ_dd0, void* d_work,
                  size_t bytes) {
    if (!lat) return HL_ERR_ARG;
    if (lat->cfg.halo_lo || lat->cfg.halo_hi)
        return fail(lat, HL_ERR_STATE, "hl_grad: the gradient covers a whole lattice, not a slab");
    if (lat->cfg.layout == 0)
        return grad_aa(lat, steps, avg_last, ckpt_every, w_thrust, w_torque, J, dJ_dpitch, d_dJ_dd0, d_work, bytes);
    // esoteric twist and the AA layout with x halves: the sweep runs on the
    // AA form of the same state (the esoteric twist gives the same
    // trajectory; with x halves the forward steps of the sweep take the AA
    // layout's cell pairs); the adjoint arrays of the workspace, not yet or
    // no longer in use, hold the permuted copy
    hl_status rc = grad_check(lat, steps, avg_last, ckpt_every, w_thrust, w_torque, d_work, bytes);
    if (rc != HL_OK) return rc;
    void* scratch = static_cast<char*>(d_work) + grad_layout(lat, steps, ckpt_every).lam;
    if ((rc = relayout_state(lat, scratch, false)) != HL_OK) return rc;
    const int layout = lat->cfg.layout;
    lat->cfg.layout = 0;
    rc = grad_aa(lat, steps, avg_last, ckpt_every, w_thrust, w_torque, J, dJ_dpitch, d_dJ_dd0, d_work, bytes);
    lat->cfg.layout = layout;
    // back at the step the lattice ended on, also after a failed sweep
    const hl_status rb = relayout_state(lat, scratch, true);
    if (rc != HL_OK) return rc;
    if (rb != HL_OK) return rb;
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    return HL_OK;
}

hl_status hl_set_d0(hl_lattice* lat, const float* d_d0) {
    if (!lat) return HL_ERR_ARG;
    lat->d0 = d_d0;
    return HL_OK;
}

hl_status hl_set_inflow_plane(hl_lattice* lat, const float* d_plane) {
    if (!lat) return HL_ERR_ARG;
    if (d_plane && (!lat->cfg.open_boundaries || (lat->cfg.flow_axis == 2 && lat->cfg.halo_lo)))
        return fail(lat, HL_ERR_STATE, "hl_set_inflow_plane: the lattice has no inlet");
    lat->inflow = d_plane;
    return HL_OK;
}

hl_status hl_set_pitch(hl_lattice* lat, int rotor, double pitch) {
    if (!lat || rotor < 0 || rotor >= lat->nrot || !std::isfinite(pitch)) return HL_ERR_ARG;
    lat->rot[rotor].pitch = pitch;
    if (!lat->frozen) lat->rot[rotor].pitch_sets = pitch;
    return HL_OK;
}

hl_status hl_freeze_sets(hl_lattice* lat, int on) {
    if (!lat) return HL_ERR_ARG;
    lat->frozen = on != 0;
    for (int k = 0; k < lat->nrot; ++k) lat->rot[k].pitch_sets = lat->rot[k].pitch;
    return HL_OK;
}

hl_status hl_debug_collide_pair(int q, int n, const float* d_g_in, double tau_mo, double c_smag, float* d_g_out,
                                void* stream) {
    if ((q != 19 && q != 27) || n < 0 || (n % 2) != 0 || (n > 0 && (!d_g_in || !d_g_out))) return HL_ERR_ARG;
    if (n == 0) return HL_OK;
    const float Ks = (float)(18.0 * std::sqrt(2.0) * c_smag * c_smag);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (n / 2 + 127) / 128;
    if (q == 19) debug_collide_pair_kernel<19><<<blocks, 128, 0, s>>>(n, d_g_in, (float)tau_mo, Ks, d_g_out);
    else debug_collide_pair_kernel<27><<<blocks, 128, 0, s>>>(n, d_g_in, (float)tau_mo, Ks, d_g_out);
    return cudaGetLastError() == cudaSuccess ? HL_OK : HL_ERR_CUDA;
}

hl_status hl_debug_collide_vjp(int q, int n, const float* d_g_in, const float* d_d, const float* d_uB,
                               const float* d_sigma, const float* d_S, double tau_mo, double c_smag,
                               const float* d_lam_star, float* d_lam, float* d_gd, float* d_guB, float* d_gS,
                               void* stream) {
    if ((q != 19 && q != 27) || n < 0 || !d_g_in || !d_lam_star || !d_lam) return HL_ERR_ARG;
    if (d_d && (!d_uB || !d_sigma || !d_S)) return HL_ERR_ARG;
    if (n == 0) return HL_OK;
    const float Ks = (float)(18.0 * std::sqrt(2.0) * c_smag * c_smag);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (n + 127) / 128;
    if (q == 19)
        debug_collide_vjp_kernel<19><<<blocks, 128, 0, s>>>(n, d_g_in, d_d, d_uB, d_sigma, d_S, (float)tau_mo, Ks,
                                                            d_lam_star, d_lam, d_gd, d_guB, d_gS);
    else
        debug_collide_vjp_kernel<27><<<blocks, 128, 0, s>>>(n, d_g_in, d_d, d_uB, d_sigma, d_S, (float)tau_mo, Ks,
                                                            d_lam_star, d_lam, d_gd, d_guB, d_gS);
    return cudaGetLastError() == cudaSuccess ? HL_OK : HL_ERR_CUDA;
}

}  // extern "C"
