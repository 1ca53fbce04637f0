// Kernels of the HHRRLBM-LES rotor step on B300 (sm_103a).
//
// Per time step (listing "HHRRLBM-FSI", Sec. 3.2).  The bulk launch runs on
// the lattice stream; the rotor-box chain (embedding, wall model, box
// collision, force, evolve) runs beside it on a second stream:
//   band_kernel         porosity embedding of the rotor boxes (Definition
//                       "Lattice Porosity", Sec. 3.1): d, force/wall flags,
//                       compacted lists of force cells and wall cells
//   band_strain_kernel  (sigma < 1) finite-difference strain of the force
//                       cells off the wall set (Sec. 2.2)
//   wall_kernel         wall model on the wall-cell list (Sec. 2.2.1, 3.2)
//   collide_pair_kernel fused collide-and-stream of the bulk cells, two
//                       x-adjacent cells per thread in packed FP32x2
//                       arithmetic (RRLBM-LES, Eq. (hlbm) with d = 1)
//   collide_kernel      fused collide-and-stream, one cell per thread: the
//                       rotor boxes (HHRRLBM-LES band branch), the pairs the
//                       packed path does not take, equilibrium inlet/outlet
//   force_kernel        momentum exchange over the force cells, FP64 block
//                       reduction, deterministic last-block combine (Sec. 2.2.2)
//   evolve_kernel       (torque-driven rotors) rotor angle and speed
//   mass_kernel         (every K steps) FP64 mass total + non-finite check
//
// AA pattern: with phase p = t & 1 of the step,
//   p = 0: f_i(x) is read from slot i of x, f*_i(x) written to slot ibar of x;
//   p = 1: f_i(x) is read from slot ibar of x - c_i, f*_i(x) written to slot i
//          of x + c_i.
// Every memory location is read and written by the same thread, so one
// buffer suffices and no synchronisation is needed inside the kernel.
#include "hl_adjoint.cuh"
#include "hl_internal.h"
#include "hl_pair.cuh"

namespace hl {


// periodic neighbour index contributions along x, y, z (-1, 0, +1)
struct Offs {
    int x[3], y[3], z[3];
};

// Position of cell x within its row of a population slot.  The AA layout
// with x halves stores cells x and x + nx/2 side by side (x < nx/2 at 2x,
// x >= nx/2 at 2(x - nx/2) + 1), so that a shift by one cell along x moves a
// whole pair of stored values (see collide_halves_kernel).
__device__ __forceinline__ int xmap(const StepArgs& a, int x) {
    return a.xpair ? (x < a.hx ? 2 * x : 2 * (x - a.hx) + 1) : x;
}

__device__ __forceinline__ void make_offs(const StepArgs& a, int x, int y, int z, Offs& o) {
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2], nxy = a.nxy;
    o.x[0] = xmap(a, x == 0 ? nx - 1 : x - 1);
    o.x[1] = xmap(a, x);
    o.x[2] = xmap(a, x == nx - 1 ? 0 : x + 1);
    o.y[0] = (y == 0 ? ny - 1 : y - 1) * nx;
    o.y[1] = y * nx;
    o.y[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    o.z[0] = (z == 0 ? nz - 1 : z - 1) * nxy;
    o.z[1] = z * nxy;
    o.z[2] = (z == nz - 1 ? 0 : z + 1) * nxy;
}

template <int Q, int S>
__device__ __forceinline__ typename Store<S>::T* slot_ptr(const StepArgs& a, int s) {
    return static_cast<typename Store<S>::T*>(a.slot[s]);
}
template <int Q, int S>
__device__ __forceinline__ typename Store<S>::T* wslot_ptr(const StepArgs& a, int s) {
    return static_cast<typename Store<S>::T*>(a.wslot[s]);
}

// Esoteric twist: the link between x and x + c lives at cell x + max(c, 0).
// Cell index of the link a cell reads f_s over (towards x - c_s) or writes
// f*_s onto (towards x + c_s), periodic wrap from the neighbour offsets.
__device__ __forceinline__ int eso_read_node(const Offs& o, int cx, int cy, int cz) {
    return o.x[1 + (cx < 0)] + o.y[1 + (cy < 0)] + o.z[1 + (cz < 0)];
}
__device__ __forceinline__ int eso_write_node(const Offs& o, int cx, int cy, int cz) {
    return o.x[1 + (cx > 0)] + o.y[1 + (cy > 0)] + o.z[1 + (cz > 0)];
}

// pre-collision populations of a cell in the layout of phase PH (the
// neighbour across an open face wraps: that value is undefined by the scheme
// and only read for cells on an open boundary plane)
template <int Q, int S, int PH, int L>
__device__ __forceinline__ void load_pre(const StepArgs& a, const Offs& o, float (&g)[Q]) {
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        if (L == 1) {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            g[s] = Store<S>::ld(slot_ptr<Q, S>(a, PH == 0 ? s : oslot(Q, s)) + eso_read_node(o, cx, cy, cz));
        } else if (PH == 0) {
            g[s] = Store<S>::ld(slot_ptr<Q, S>(a, s) + (o.x[1] + o.y[1] + o.z[1]));
        } else {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            const int src = o.x[1 - cx] + o.y[1 - cy] + o.z[1 - cz];
            g[s] = Store<S>::ld(slot_ptr<Q, S>(a, oslot(Q, s)) + src);
        }
    }
}

__device__ __forceinline__ void solid_velocity(const RotorDev& R, int x, int y, int z, float us[3]) {
    const float r[3] = {(float)x - R.cf[0], (float)y - R.cf[1], (float)z - R.cf[2]};
    const int ax = R.axis;
    // u_s = Omega a x r: (a x r)_b = -r_c, (a x r)_c = r_b with (b, c) = (a+1, a+2)
    const float om = rot_omega(R);
    if (ax == 0) { us[0] = 0.f; us[1] = -om * r[2]; us[2] = om * r[1]; }
    else if (ax == 1) { us[1] = 0.f; us[2] = -om * r[0]; us[0] = om * r[2]; }
    else { us[2] = 0.f; us[0] = -om * r[1]; us[1] = om * r[0]; }
}

__device__ __forceinline__ int sel3(int ax, int a0, int a1, int a2) { return ax == 0 ? a0 : (ax == 1 ? a1 : a2); }

// ---------------------------------------------------------------------------
// fused collide and stream
// ---------------------------------------------------------------------------
template <int Q, int S, int PH, bool D0, int L>
__device__ __forceinline__ void collide_cell(const StepArgs& a, int x, int y, int z) {
    const int cell = (z * a.n[1] + y) * a.n[0] + x;
    const int ax = a.flow_axis;
    const int ca = sel3(ax, x, y, z);
    const int na = sel3(ax, a.n[0], a.n[1], a.n[2]);
    const bool inlet = a.open && a.open_lo && ca == 0;
    const bool outlet = a.open && a.open_hi && ca == na - 1;
    // every population at one offset from a per-slot base (no neighbour index
    // arithmetic): AA odd steps away from the lattice faces; esoteric twist
    // (links towards +x, +y, +z only) away from the upper faces
    constexpr bool eso = L == 1;
    // (with x halves a shift along x also crosses between the halves at
    // x = nx/2 - 1 and nx/2)
    const bool shifted = eso ? (x < a.n[0] - 1 && y < a.n[1] - 1 && z < a.n[2] - 1)
                             : (PH == 1 && x > 0 && x < a.n[0] - 1 && y > 0 && y < a.n[1] - 1 && z > 0 &&
                                z < a.n[2] - 1 && !(a.xpair && (x == a.hx - 1 || x == a.hx)));
    Offs o;
    make_offs(a, x, y, z, o);
    const int pc = o.x[1] + o.y[1] + o.z[1];   // the cell's position in a population slot
    float g[Q];
    if (!inlet && !outlet) {
        int rk = -1, bi = 0;
        for (int k = 0; k < a.nrot; ++k) {
            const unsigned dx = (unsigned)(x - a.rot[k].lo[0]), dy = (unsigned)(y - a.rot[k].lo[1]),
                           dz = (unsigned)(z - a.rot[k].lo[2]);
            if (dx < (unsigned)a.rot[k].n[0] && dy < (unsigned)a.rot[k].n[1] && dz < (unsigned)a.rot[k].n[2]) {
                rk = k;
                bi = ((int)dz * a.rot[k].n[1] + (int)dy) * a.rot[k].n[0] + (int)dx;
                break;
            }
        }
        if (a.part == 1 && rk >= 0) return;   // box cells belong to the box launch
        if (shifted) {
            using T = typename Store<S>::T;
#pragma unroll
            for (int s = 0; s < Q; ++s) g[s] = Store<S>::ld(static_cast<const T*>(a.rshift[s]) + pc);
        } else {
            load_pre<Q, S, PH, L>(a, o, g);
        }
        float u[3];
        float rho;
        if (rk >= 0) {
            const RotorDev& R = a.rot[rk];
            Band B;
            B.d = D0 ? a.d0[cell] * R.d[bi] : R.d[bi];
            const uint8_t fl = R.flags[bi];
            // u^B is the rotor's velocity on its force cells; elsewhere in the
            // box d = d0 (1 unless a static multiplier is set) with u^B = 0
            if (fl & FL_B) {
                solid_velocity(R, x, y, z, B.uB);
            } else {
                B.uB[0] = B.uB[1] = B.uB[2] = 0.0f;
            }
            // hybrid non-equilibrium on the force cells only (sigma = 1 elsewhere)
            B.sigma = (fl & FL_B) ? a.sigma_band : 1.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) B.S[k] = 0.0f;
            if (a.wall_model && (fl & FL_W)) {
                const float* wm = R.wm + bi;
                const long long bc = R.box_cells;
                B.uB[0] += wm[0];
                B.uB[1] += wm[bc];
                B.uB[2] += wm[2 * bc];
#pragma unroll
                for (int k = 0; k < 6; ++k) B.S[k] = wm[(3 + k) * bc];
                B.sigma = 0.0f;
            } else if ((fl & FL_B) && a.sigma_band < 1.0f) {
                // finite-difference strain of the band-strain kernel
                const float* wm = R.wm + bi;
                const long long bc = R.box_cells;
#pragma unroll
                for (int k = 0; k < 6; ++k) B.S[k] = wm[(3 + k) * bc];
            }
            rho = collide<Q, true>(g, B, a.tau_mo, a.Ksmag, u);
        } else if (D0) {
            // static porous medium at rest: d = d0, u^B = 0
            Band B;
            B.d = a.d0[cell];
            B.uB[0] = B.uB[1] = B.uB[2] = 0.0f;
            B.sigma = 1.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) B.S[k] = 0.0f;
            rho = collide<Q, true>(g, B, a.tau_mo, a.Ksmag, u);
        } else {
            Band B0;
            rho = collide<Q, false>(g, B0, a.tau_mo, a.Ksmag, u);
        }
        if (!(fabsf(rho) < 1e30f)) atomicOr(a.err, ERR_NONFINITE);
        if (a.open && a.open_hi && ca == na - 2) {
            const int nb = sel3(ax, a.n[1], a.n[2], a.n[0]);
            const int cb = sel3(ax, y, z, x), cc = sel3(ax, z, x, y);
            const int pl = cc * nb + cb;
            a.uplane_cur[pl] = u[0];
            a.uplane_cur[a.nplane + pl] = u[1];
            a.uplane_cur[2 * a.nplane + pl] = u[2];
        }
        if (shifted) {
            using T = typename Store<S>::T;
#pragma unroll
            for (int s = 0; s < Q; ++s) Store<S>::st(static_cast<T*>(a.wshift[s]) + pc, g[s]);
            return;
        }
#pragma unroll
        for (int s = 0; s < Q; ++s) {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            if (eso) {
                Store<S>::st(wslot_ptr<Q, S>(a, PH == 0 ? oslot(Q, s) : s) + eso_write_node(o, cx, cy, cz), g[s]);
            } else if (PH == 0) {
                Store<S>::st(wslot_ptr<Q, S>(a, oslot(Q, s)) + pc, g[s]);
            } else {
                Store<S>::st(wslot_ptr<Q, S>(a, s) + (o.x[1 + cx] + o.y[1 + cy] + o.z[1 + cz]), g[s]);
            }
        }
        return;
    }
    if (inlet && a.inflow_plane) {
        // equilibrium inflow at the caller's plane velocity
        const int nb = sel3(ax, a.n[1], a.n[2], a.n[0]);
        const int cb = sel3(ax, y, z, x), cc = sel3(ax, z, x, y);
        const int pl = cc * nb + cb;
        const float u[3] = {a.inflow_plane[pl], a.inflow_plane[a.nplane + pl], a.inflow_plane[2 * a.nplane + pl]};
        equilibrium<Q>(g, 0.0f, u);
    } else if (inlet) {
        // equilibrium inflow: U a + sum_m a_m cos(k.x') + b_m sin(k.x'), x' = x - U t a
        float u[3] = {0.f, 0.f, 0.f};
        u[ax] = a.u_in;
        float xp[3] = {(float)x, (float)y, (float)(z + a.zoff)};
        xp[ax] -= a.inflow_shift;
        for (int m = 0; m < a.n_modes; ++m) {
            const float* md = a.modes + 9 * m;
            const float ph = md[0] * xp[0] + md[1] * xp[1] + md[2] * xp[2];
            float sn, cs;
            sincosf(ph, &sn, &cs);
            u[0] += md[3] * cs + md[6] * sn;
            u[1] += md[4] * cs + md[7] * sn;
            u[2] += md[5] * cs + md[8] * sn;
        }
        equilibrium<Q>(g, 0.0f, u);
    } else {
        // equilibrium outflow at the velocity of the upstream neighbour, previous step
        const int nb = sel3(ax, a.n[1], a.n[2], a.n[0]);
        const int cb = sel3(ax, y, z, x), cc = sel3(ax, z, x, y);
        const int pl = cc * nb + cb;
        const float u[3] = {a.uplane_prev[pl], a.uplane_prev[a.nplane + pl], a.uplane_prev[2 * a.nplane + pl]};
        equilibrium<Q>(g, 0.0f, u);
    }
    // boundary planes: populations that would leave through the open face are dropped
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        if (eso) {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            const int cas = sel3(ax, cx, cy, cz);
            if ((inlet && cas < 0) || (outlet && cas > 0)) continue;
            Store<S>::st(wslot_ptr<Q, S>(a, PH == 0 ? oslot(Q, s) : s) + eso_write_node(o, cx, cy, cz), g[s]);
        } else if (PH == 0) {
            Store<S>::st(wslot_ptr<Q, S>(a, oslot(Q, s)) + pc, g[s]);
        } else {
            const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
            const int cas = sel3(ax, cx, cy, cz);
            if ((inlet && cas < 0) || (outlet && cas > 0)) continue;
            Store<S>::st(wslot_ptr<Q, S>(a, s) + (o.x[1 + cx] + o.y[1 + cy] + o.z[1 + cz]), g[s]);
        }
    }
}

// One cell per thread: the bulk launch when cell pairs are off (nx odd, a
// static porosity field), or the box launch spanning one rotor box.
template <int Q, int S, int PH, bool D0, int L>
__global__ void __launch_bounds__(128) collide_kernel(const StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (a.part == 2) {
        const RotorDev& R = a.rot[a.part_rotor];
        if (x >= R.n[0] || y >= R.n[1]) return;
        collide_cell<Q, S, PH, D0, L>(a, x + R.lo[0], y + R.lo[1], (int)blockIdx.z + R.lo[2]);
        return;
    }
    const int z = (int)blockIdx.z + a.z0;     // halo planes of a slab are not collided
    if (y >= a.n[1] || x >= a.n[0]) return;
    collide_cell<Q, S, PH, D0, L>(a, x, y, z);
}

// Bulk launches with cell pairs: a thread takes cells x and x + 1 (x even).
// A pair of plain bulk cells - outside every rotor box, off the inlet, the
// outlet and the plane that feeds the outlet, and (odd phase) off the y and z
// faces - takes the packed collision, with one access for both cells wherever
// the pair is aligned (every slot in the even phase, slots with c_x = 0 in the
// odd phase); any other pair runs the per-cell path.  The first and last pair
// of an x row take the packed path too (their odd-phase neighbours across the
// periodic x face are one row length away), so that no warp of a plain row
// diverges into the per-cell path.
// Register caps: D3Q27 at most 64 (8 blocks of 128 per SM, 8-12 bytes of
// spill), 2-3 % faster for 16-bit storage than the unbounded 72 (56, 9 blocks,
// spills 60-100 bytes and is slower on every storage); D3Q19 at most 48 (10
// blocks), 3 % faster for 16-bit storage than the unbounded 56, FP32 unchanged.
// Does the pair (x, x + 1) of row (y, z) take the packed path?
template <int Q, int S, int PH, int L>
__device__ __forceinline__ bool pair_plain(const StepArgs& a, int x, int y, int z) {
    bool plain = x + 1 < a.n[0];
    for (int k = 0; k < a.nrot; ++k) {
        const RotorDev& R = a.rot[k];
        if ((unsigned)(y - R.lo[1]) < (unsigned)R.n[1] && (unsigned)(z - R.lo[2]) < (unsigned)R.n[2] &&
            x + 1 >= R.lo[0] && x < R.lo[0] + R.n[0])
            plain = false;
    }
    if (a.open) {
        const int ca = sel3(a.flow_axis, x, y, z);
        const int ca1 = ca + (a.flow_axis == 0 ? 1 : 0);
        const int na = sel3(a.flow_axis, a.n[0], a.n[1], a.n[2]);
        if ((a.open_lo && ca == 0) || (a.open_hi && ca1 >= na - 2)) plain = false;
    }
    // the y and z neighbours the pair touches must lie inside the lattice
    if (L == 0 && PH == 1 && !(y > 0 && y < a.n[1] - 1 && z > 0 && z < a.n[2] - 1)) plain = false;
    if (L == 1 && !(y < a.n[1] - 1 && z < a.n[2] - 1)) plain = false;
    return plain;
}

// packed collision of a plain pair and its stores (x even, cell = index of x)
template <int Q, int S, int PH, int L>
__device__ __forceinline__ void pair_collide_store(const StepArgs& a, int x, int cell, F2 (&g)[Q]) {
    using T = typename Store<S>::T;
    const int lo_wrap = (L == 0 && PH == 1 && x == 0) ? a.n[0] : 0;
    const int hi_wrap = ((L == 1 || PH == 1) && x + 2 == a.n[0]) ? -a.n[0] : 0;
    F2 u[3];
    const F2 rho = collide_pair<Q>(g, a.tau_mo, a.Ksmag, u);
    if (!(fabsf(rho.v.x) < 1e30f) || !(fabsf(rho.v.y) < 1e30f)) atomicOr(a.err, ERR_NONFINITE);
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int cx = cslot(Q, s, 0);
        if (L == 1) {
            // f*_s onto the link at x + max(c_s, 0): one element off for c_x > 0
            T* dst = static_cast<T*>(a.wshift[s]) + cell;
            if (cx <= 0) {
                Store2<S>::st(dst, g[s]);
            } else {
                Store<S>::st(dst, g[s].v.x);
                Store<S>::st(dst + 1 + hi_wrap, g[s].v.y);
            }
            continue;
        }
        T* dst = PH == 0 ? wslot_ptr<Q, S>(a, oslot(Q, s)) + cell : static_cast<T*>(a.wshift[s]) + cell;
        if (PH == 0 || cx == 0) {
            Store2<S>::st(dst, g[s]);
        } else if (cx > 0) {
            Store<S>::st(dst, g[s].v.x);
            Store<S>::st(dst + 1 + hi_wrap, g[s].v.y);
        } else {
            Store<S>::st(dst + lo_wrap, g[s].v.x);
            Store<S>::st(dst + 1, g[s].v.y);
        }
    }
}

template <int Q, int S, int PH, int L>
__global__ void __launch_bounds__(128, Q == 27 ? 8 : 10) collide_pair_kernel(const StepArgs a) {
    const int x = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z + a.z0;     // halo planes of a slab are not collided
    if (y >= a.n[1] || x >= a.n[0]) return;
    if (!pair_plain<Q, S, PH, L>(a, x, y, z)) {
        collide_cell<Q, S, PH, false, L>(a, x, y, z);
        if (x + 1 < a.n[0]) collide_cell<Q, S, PH, false, L>(a, x + 1, y, z);
        return;
    }
    using T = typename Store<S>::T;
    const int cell = (z * a.n[1] + y) * a.n[0] + x;
    // periodic x: the first cell's neighbour at x - 1 (AA odd steps) and the
    // last cell's neighbour at x + 2 (AA odd steps, esoteric twist) lie one
    // row length away
    const int lo_wrap = (L == 0 && PH == 1 && x == 0) ? a.n[0] : 0;
    const int hi_wrap = ((L == 1 || PH == 1) && x + 2 == a.n[0]) ? -a.n[0] : 0;
    F2 g[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int cx = cslot(Q, s, 0);
        if (L == 1) {
            // f_s over the link at x + max(-c_s, 0): one element off for c_x < 0
            const T* src = static_cast<const T*>(a.rshift[s]) + cell;
            if (cx >= 0) g[s] = Store2<S>::ld(src);
            else g[s] = {make_float2(Store<S>::ld(src), Store<S>::ld(src + 1 + hi_wrap))};
            continue;
        }
        const T* src = PH == 0 ? slot_ptr<Q, S>(a, s) + cell : static_cast<const T*>(a.rshift[s]) + cell;
        if (PH == 0 || cx == 0) g[s] = Store2<S>::ld(src);
        else if (cx > 0) g[s] = {make_float2(Store<S>::ld(src + lo_wrap), Store<S>::ld(src + 1))};
        else g[s] = {make_float2(Store<S>::ld(src), Store<S>::ld(src + 1 + hi_wrap))};
    }
    pair_collide_store<Q, S, PH, L>(a, x, cell, g);
}

// AA layout with x halves: a thread takes cells t and t + nx/2 of a row,
// stored side by side (one 8-byte FP32 or 4-byte 16-bit access).  A shift by
// c_x = +-1 moves both cells to the neighbouring pair position, so every slot
// is one aligned access at both step parities; only at the periodic wrap
// (t = 0 reading / writing across x = 0, t = nx/2 - 1 across x = nx - 1)
// the pair lies at the other end of the row with its two cells exchanged.
// Rows on a periodic y or z face take the packed path too (D3Q19), with the
// wrapped row offsets added per slot (a branch uniform over the row's warps).
// Same cell model as collide_pair_kernel (packed FP32x2 per lane).
template <int Q, int S, int PH>
__device__ __forceinline__ bool halves_plain(const StepArgs& a, int t, int y, int z) {
    const int xs[2] = {t, t + a.hx};
    bool plain = true;
    for (int k = 0; k < a.nrot; ++k) {
        const RotorDev& R = a.rot[k];
        if ((unsigned)(y - R.lo[1]) < (unsigned)R.n[1] && (unsigned)(z - R.lo[2]) < (unsigned)R.n[2] &&
            ((unsigned)(xs[0] - R.lo[0]) < (unsigned)R.n[0] || (unsigned)(xs[1] - R.lo[0]) < (unsigned)R.n[0]))
            plain = false;
    }
    if (a.open) {
        const int na = sel3(a.flow_axis, a.n[0], a.n[1], a.n[2]);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ca = sel3(a.flow_axis, xs[c], y, z);
            if ((a.open_lo && ca == 0) || (a.open_hi && ca >= na - 2)) plain = false;
        }
    }
    return plain;
}

// Periodic offsets of one axis at odd steps: a read with c = +1 (from the
// plane below) or a write with c = -1 (onto it) crosses the lower face from
// plane 0 (lo = +n planes), a read with c = -1 or a write with c = +1 the upper
// face from plane n - 1 (hi = -n planes).
struct WrapOff {
    int lo, hi;
};
__device__ __forceinline__ int wrap_read(const WrapOff& o, int c) { return c > 0 ? o.lo : (c < 0 ? o.hi : 0); }
__device__ __forceinline__ int wrap_write(const WrapOff& o, int c) { return c > 0 ? o.hi : (c < 0 ? o.lo : 0); }

// XW: the warp holds the first or the last pair of its row (the others need
// neither the wrap offsets nor the byte permutations)
template <int Q, int S, int PH, bool YZ, bool XW>
__device__ __forceinline__ void halves_packed(const StepArgs& a, int t, int y, int z) {
    using T = typename Store<S>::T;
    const int w = (z * a.n[1] + y) * a.n[0] + 2 * t;   // the pair's position in a slot
    // x: the first pair reads (c_x = +1) and writes (c_x = -1) across x = 0,
    // the last pair reads (c_x = -1) and writes (c_x = +1) across x = nx - 1,
    // each at the row's other end with its cells exchanged
    const WrapOff ox = {XW && t == 0 ? a.n[0] : 0, XW && t == a.hx - 1 ? -a.n[0] : 0};
    const unsigned sel_lo = XW && t == 0 ? SWAP2 : KEEP2, sel_hi = XW && t == a.hx - 1 ? SWAP2 : KEEP2;
    WrapOff oy = {0, 0}, oz = {0, 0};
    if constexpr (YZ) {
        oy = {y == 0 ? a.nxy : 0, y == a.n[1] - 1 ? -a.nxy : 0};
        const int nzxy = a.n[2] * a.nxy;
        oz = {z == 0 ? nzxy : 0, z == a.n[2] - 1 ? -nzxy : 0};
    }
    F2 g[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
        if (PH == 0) {
            g[s] = Store2<S>::ld(slot_ptr<Q, S>(a, s) + w);
            continue;
        }
        int off = w;
        if constexpr (XW) off += wrap_read(ox, cx);
        if constexpr (YZ) off += wrap_read(oy, cy) + wrap_read(oz, cz);
        const T* src = static_cast<const T*>(a.rshift[s]) + off;
        if (cx == 0 || !XW) g[s] = Store2<S>::ld(src);
        else g[s] = Store2x<S>::ld(src, cx > 0 ? sel_lo : sel_hi);
    }
    F2 u[3];
    const F2 rho = collide_pair<Q>(g, a.tau_mo, a.Ksmag, u);
    if (!(fabsf(rho.v.x) < 1e30f) || !(fabsf(rho.v.y) < 1e30f)) atomicOr(a.err, ERR_NONFINITE);
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int cx = cslot(Q, s, 0), cy = cslot(Q, s, 1), cz = cslot(Q, s, 2);
        if (PH == 0) {
            Store2<S>::st(wslot_ptr<Q, S>(a, oslot(Q, s)) + w, g[s]);
            continue;
        }
        int off = w;
        if constexpr (XW) off += wrap_write(ox, cx);
        if constexpr (YZ) off += wrap_write(oy, cy) + wrap_write(oz, cz);
        T* dst = static_cast<T*>(a.wshift[s]) + off;
        if (cx == 0 || !XW) Store2<S>::st(dst, g[s]);
        else Store2x<S>::st(dst, g[s], cx > 0 ? sel_hi : sel_lo);
    }
}

// the face rows out of line: their extra offsets keep their registers to themselves
template <int Q, int S>
__device__ __noinline__ void halves_packed_faces(const StepArgs& a, int t, int y, int z) {
    halves_packed<Q, S, 1, true, true>(a, t, y, z);
}

// Register caps: D3Q19 FP16 at 56 (9 blocks of 128 per SM), 2 % faster than
// 48; BF16 (cheaper conversions) and FP32 at 48 (10 blocks); D3Q27 at 64.
template <int Q, int S, int PH>
__global__ void __launch_bounds__(128, Q == 27 ? 8 : (S == ST_F16S ? 9 : 10)) collide_halves_kernel(const __grid_constant__ StepArgs a) {
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z + a.z0;     // halo planes of a slab are not collided
    if (y >= a.n[1] || t >= a.hx) return;
    if (!halves_plain<Q, S, PH>(a, t, y, z)) {
        collide_cell<Q, S, PH, false, 0>(a, t, y, z);
        collide_cell<Q, S, PH, false, 0>(a, t + a.hx, y, z);
        return;
    }
    if (PH == 1 && (y == 0 || y == a.n[1] - 1 || z == 0 || z == a.n[2] - 1)) {
        // D3Q27: the out-of-line call costs the packed path registers (spills at
        // the 64-register cap), so its face rows take the per-cell path
        if constexpr (Q == 19) {
            halves_packed_faces<Q, S>(a, t, y, z);
        } else {
            collide_cell<Q, S, PH, false, 0>(a, t, y, z);
            collide_cell<Q, S, PH, false, 0>(a, t + a.hx, y, z);
        }
        return;
    }
    // D3Q27 (18 x-shifted slots): only the warps holding a row's first or
    // last pair take the wrap offsets and byte permutations (warps lie in
    // one row: the block's x extent is a multiple of 32 threads); FP16
    // rotor1024_q27 53.2k -> 54.6k MLUPS.  D3Q19 keeps one path for every
    // warp (the split cost it 0.8 %).
    const int t0 = t & ~31;
    if (Q == 19 || (PH == 1 && (t0 == 0 || t0 + 31 >= a.hx - 1))) halves_packed<Q, S, PH, false, true>(a, t, y, z);
    else halves_packed<Q, S, PH, false, false>(a, t, y, z);
}

// ---------------------------------------------------------------------------
// porosity embedding of the rotor boxes and the force / wall cell lists
// ---------------------------------------------------------------------------
__device__ __forceinline__ int append(int* counter, bool take, int lane) {
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    int start = 0;
    if (mask) {
        if (lane == 0) start = atomicAdd(counter, __popc(mask));
        start = __shfl_sync(0xffffffffu, start, 0);
    }
    return start + __popc(mask & ((1u << lane) - 1u));
}

// One warp per box row (x contiguous, one 32-bit divide per row); rows are
// strided over the grid's warps, so every ballot sees all 32 lanes.
__global__ void __launch_bounds__(BAND_THREADS) band_kernel(const StepArgs a) {
    const RotorDev& R = a.rot[blockIdx.y];
    const int n0 = R.n[0], n1 = R.n[1];
    const int rows = n1 * R.n[2];
    const int nbox = (int)R.box_cells;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += gridDim.x * wpb) {
        const int by = row % n1, bz = row / n1;
        const int y = R.lo[1] + by, z = R.lo[2] + bz;
        const float ry = (float)y - R.cf[1], rz = (float)z - R.cf[2];
        for (int x0 = 0; x0 < n0; x0 += 32) {
            const int bx = x0 + lane;
            const int bi = row * n0 + bx;
            bool isB = false, isW = false;
            float phi = 0.f;
            int which = -1;
            if (bx < n0) {
                const int x = R.lo[0] + bx;
                uint8_t fl = 0;
                float d = 1.0f;
                // cells beyond the rotor's reach (every blade sample out of its grid,
                // hub farther than eps/2 + 1) keep d = 1 without evaluating phi
                const float rx = (float)x - R.cf[0];
                const float ra = R.axis == 0 ? rx : (R.axis == 1 ? ry : rz);
                const float rr = rx * rx + ry * ry + rz * rz - ra * ra;
                float dd = 0.0f;
                if (rr <= R.reach_plane2 && fabsf(ra) <= R.reach_axial) {
                    phi = rotor_phi(R, R.cpD, R.spD, x, y, z, which);
                    if (phi < a.eps_half) {
                        fl |= FL_B;
                        if (phi >= 0.0f) fl |= FL_W;
                        // sets frozen: porosity and wall distance of the same component at the current pitch
                        if (R.frozen) phi = component_phi(R, which, x, y, z);
                        if (phi <= -a.eps_half) {
                            d = 0.0f;
                        } else if (phi < a.eps_half) {
                            const float tt = phi * a.inv_eps + 0.5f;
                            d = a.transition ? tt : tt * tt * (3.0f - 2.0f * tt);
                            if (a.tangent) {
                                float dphi;
                                component_phi_tan(R, which, x, y, z, dphi);
                                const float ds = a.transition ? a.inv_eps : 6.0f * tt * (1.0f - tt) * a.inv_eps;
                                dd = ds * dphi;
                            }
                        }
                    }
                }
                R.d[bi] = d;
                if (a.tangent) R.ddp[bi] = dd;
                R.flags[bi] = fl;
                isB = (fl & FL_B) != 0;
                isW = a.wall_model && (fl & FL_W);
                if (!isW) R.active[bi] = 0;
            }
            const int fslot = append(R.count, isB, lane);
            if (isB && fslot < nbox) R.list[fslot] = bi;
            const int wslot = append(R.count + 1, isW, lane);
            if (isW && wslot < nbox) {
                R.wlist[wslot] = bi;
                R.wphi[wslot] = phi;
                R.wwhich[wslot] = (signed char)which;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// wall model on the wall-cell list (Sec. 2.2.1): sample, Newton in FP64
// ---------------------------------------------------------------------------
template <int Q, int S, int PH>
__device__ void cell_velocity(const StepArgs& a, int x, int y, int z, float u[3]) {
    Offs o;
    make_offs(a, x, y, z, o);
    float g[Q];
    if (a.layout == 1) load_pre<Q, S, PH, 1>(a, o, g);
    else load_pre<Q, S, PH, 0>(a, o, g);
    float drho, j[3];
    moments01<Q>(g, drho, j);
    const float inv = 1.0f / (1.0f + drho);
    u[0] = j[0] * inv; u[1] = j[1] * inv; u[2] = j[2] * inv;
}

template <int Q, int S, int PH, int LN>
__global__ void __launch_bounds__(128) wall_kernel(const StepArgs a) {
    const RotorDev& R = a.rot[blockIdx.y];
    int count = *((volatile int*)(R.count + 1));
    if ((long long)count > R.box_cells) count = (int)R.box_cells;
    // LN lanes per wall cell (1 or 4): lane sub gathers the velocities of the
    // sample corners m = sub (mod LN); every lane of the group then runs the
    // same Newton solve and lane 0 stores the result (the group takes the
    // same list entries, so its branches are uniform)
    static_assert(LN == 1 || LN == 4, "one or four lanes per wall cell");
    const int sub = LN == 1 ? 0 : (int)(threadIdx.x & 3);
    const unsigned gm = LN == 1 ? 0u : 0xfu << (threadIdx.x & 28);
    const int gbase = threadIdx.x & 28;
    for (int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) / LN); idx < count;
         idx += (int)((gridDim.x * blockDim.x) / LN)) {
        const long long bi = R.wlist[idx];
        const float phi = R.wphi[idx];
        const int which = R.wwhich[idx];
        const int bx = (int)(bi % R.n[0]);
        const long long r2 = bi / R.n[0];
        const int by = (int)(r2 % R.n[1]);
        const int bz = (int)(r2 / R.n[1]);
        const int x = R.lo[0] + bx, y = R.lo[1] + by, z = R.lo[2] + bz;
        float n[3];
        rotor_normal(R, which, x, y, z, n);
        const float y1 = phi > 0.5f ? phi : 0.5f;
        // sampling point x_s = x + y_s n and trilinear fluid velocity there; the
        // corner and the weights come from the offset y_s n alone (x is an
        // integer), so they do not depend on where the lattice's origin lies
        const float dv[3] = {a.wmYs * n[0], a.wmYs * n[1], a.wmYs * n[2]};
        const int xc[3] = {x, y, z};
        int i0[3];
        float t[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float fl = floorf(dv[k]);
            i0[k] = xc[k] + (int)fl;
            t[k] = dv[k] - fl;
            if (a.open && k == a.flow_axis) {
                if (i0[k] < 0) { i0[k] = 0; t[k] = 0.f; }
                if (i0[k] > a.n[k] - 2) { i0[k] = a.n[k] - 2; t[k] = 1.f; }
            }
        }
        // the sample's corner cells must lie in the rotor box: the box chain
        // runs beside the bulk launch, which updates every cell outside it
        // (along z, through a slab face that cuts the box, the neighbouring
        // slab's planes in the deep halo, which only the halo exchange writes)
        bool inside = i0[2] >= R.zs_lo && i0[2] + 1 < R.zs_hi;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            inside = inside && i0[k] - R.lo[k] >= 0 && i0[k] + 1 - R.lo[k] < R.n[k];
        const long long B = R.box_cells;
        float* wm = R.wm + bi;
        if (!inside) {
            if (sub == 0) {
                atomicOr(a.err, ERR_GEOMETRY);
#pragma unroll
                for (int k = 0; k < 9; ++k) wm[k * B] = 0.f;
                R.active[bi] = 0;
                R.utau[bi] = 0.0;
            }
            continue;
        }
        constexpr int NH = 8 / LN;
        float wc[NH], uc[NH][3];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const int m = sub + LN * h;
            const int cx = m & 1, cy = (m >> 1) & 1, cz = m >> 2;
            int p[3] = {i0[0] + cx, i0[1] + cy, i0[2] + cz};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (!(a.open && k == a.flow_axis)) p[k] = ((p[k] % a.n[k]) + a.n[k]) % a.n[k];
            wc[h] = (cx ? t[0] : 1.f - t[0]) * (cy ? t[1] : 1.f - t[1]) * (cz ? t[2] : 1.f - t[2]);
            cell_velocity<Q, S, PH>(a, p[0], p[1], p[2], uc[h]);
        }
        // the trilinear sum in corner order 0..7 (m = cx + 2 cy + 4 cz)
        float us[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            float wgt, u0, u1, u2;
            if constexpr (LN == 1) {
                wgt = wc[m]; u0 = uc[m][0]; u1 = uc[m][1]; u2 = uc[m][2];
            } else {
                const int h = m >> 2, src = gbase + (m & 3);
                wgt = __shfl_sync(gm, h ? wc[1] : wc[0], src);
                u0 = __shfl_sync(gm, h ? uc[1][0] : uc[0][0], src);
                u1 = __shfl_sync(gm, h ? uc[1][1] : uc[0][1], src);
                u2 = __shfl_sync(gm, h ? uc[1][2] : uc[0][2], src);
            }
            us[0] += wgt * u0; us[1] += wgt * u1; us[2] += wgt * u2;
        }
        float usol[3];
        solid_velocity(R, x, y, z, usol);
        const float ur[3] = {us[0] - usol[0], us[1] - usol[1], us[2] - usol[2]};
        const float un = ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2];
        const float ut[3] = {ur[0] - un * n[0], ur[1] - un * n[1], ur[2] - un * n[2]};
        const float utm = sqrtf(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
        if (!(utm >= 1e-12f)) {
            if (sub == 0) {
#pragma unroll
                for (int k = 0; k < 9; ++k) wm[k * B] = 0.f;
                R.active[bi] = 0;
                R.utau[bi] = 0.0;
            }
            continue;
        }
        const float th[3] = {ut[0] / utm, ut[1] / utm, ut[2] / utm};
        const float ysamp = y1 + a.wmYs;
        const WallFn W = make_wallfn(a.wmE, a.wmK, a.nu, a.wmTol, a.wmMaxit);
        // Eq. (guess): previous value if the wall function was active last step
        // (read by lane 0, which alone writes the new value below)
        float guess = 0.f;
        if (sub == 0) guess = R.active[bi] ? (float)R.utau[bi] : sqrtf(utm / (a.wmYs * W.inv_nu));
        if constexpr (LN > 1) guess = __shfl_sync(gm, guess, gbase);
        const float utau = wall_newton_t<float>(utm, ysamp, guess, W);
        const float up = spalding_uplus_t<float>(y1 * utau * W.inv_nu, W);
        const float uw = utau * up;
        const float gs = 0.5f * (utm - uw) / a.wmYs;
        if (sub != 0) continue;
        wm[0] = uw * th[0];
        wm[B] = uw * th[1];
        wm[2 * B] = uw * th[2];
        wm[3 * B] = gs * 2.0f * th[0] * n[0];
        wm[4 * B] = gs * 2.0f * th[1] * n[1];
        wm[5 * B] = gs * 2.0f * th[2] * n[2];
        wm[6 * B] = gs * (th[0] * n[1] + n[0] * th[1]);
        wm[7 * B] = gs * (th[0] * n[2] + n[0] * th[2]);
        wm[8 * B] = gs * (th[1] * n[2] + n[1] * th[2]);
        R.active[bi] = 1;
        R.utau[bi] = (double)utau;
    }
}

// ---------------------------------------------------------------------------
// finite-difference strain across the band (Sec. 2.2, hybrid non-equilibrium
// with sigma < 1): on the force cells off the wall set, S = (grad u +
// grad u^T) / 2 by central differences of the pre-collision velocity of the
// six axis neighbours, stored in rows 3..8 (xx yy zz xy xz yz) of the cell's
// wall-model record, which the box collision reads
// ---------------------------------------------------------------------------
template <int Q, int S, int PH>
__global__ void __launch_bounds__(128) band_strain_kernel(const StepArgs a) {
    const RotorDev& R = a.rot[blockIdx.y];
    int count = *((volatile int*)R.count);
    if ((long long)count > R.box_cells) count = (int)R.box_cells;
    const long long B = R.box_cells;
    for (int idx = list_first(); idx < count; idx += list_stride()) {
        const long long bi = R.list[idx];
        if (a.wall_model && (R.flags[bi] & FL_W)) continue;
        const int bx = (int)(bi % R.n[0]);
        const long long r2 = bi / R.n[0];
        const int by = (int)(r2 % R.n[1]);
        const int bz = (int)(r2 / R.n[1]);
        float* wm = R.wm + bi;
        // the stencil must lie in the rotor box (the bulk launch updates every
        // cell outside it at the same time), or along z through a slab face
        // that cuts the box in the deep halo, which only the exchange writes
        const int zc = R.lo[2] + bz;
        if (bx < 1 || by < 1 || bx > R.n[0] - 2 || by > R.n[1] - 2 || zc - 1 < R.zs_lo || zc + 1 >= R.zs_hi) {
            atomicOr(a.err, ERR_GEOMETRY);
#pragma unroll
            for (int k = 3; k < 9; ++k) wm[k * B] = 0.f;
            continue;
        }
        const int x = R.lo[0] + bx, y = R.lo[1] + by, z = R.lo[2] + bz;
        float gr[3][3];   // gr[m][b] = d u_b / d x_m
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float up[3], um[3];
            cell_velocity<Q, S, PH>(a, x + (m == 0), y + (m == 1), z + (m == 2), up);
            cell_velocity<Q, S, PH>(a, x - (m == 0), y - (m == 1), z - (m == 2), um);
#pragma unroll
            for (int b = 0; b < 3; ++b) gr[m][b] = 0.5f * (up[b] - um[b]);
        }
        wm[3 * B] = gr[0][0];
        wm[4 * B] = gr[1][1];
        wm[5 * B] = gr[2][2];
        wm[6 * B] = 0.5f * (gr[0][1] + gr[1][0]);
        wm[7 * B] = 0.5f * (gr[0][2] + gr[2][0]);
        wm[8 * B] = 0.5f * (gr[1][2] + gr[2][1]);
    }
}

// ---------------------------------------------------------------------------
// momentum exchange (Galilean-invariant link form) over the force cells
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int Q, int S, int PH>
__global__ void __launch_bounds__(256) force_kernel(const StepArgs a) {
    const RotorDev& R = a.rot[blockIdx.y];
    int count = *((volatile int*)R.count);
    if ((long long)count > R.box_cells) count = (int)R.box_cells;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int idx = list_first(); idx < count; idx += list_stride()) {
        const long long bi = R.list[idx];
        const int bx = (int)(bi % R.n[0]);
        const long long r2 = bi / R.n[0];
        const int by = (int)(r2 % R.n[1]);
        const int bz = (int)(r2 / R.n[1]);
        const int x = R.lo[0] + bx, y = R.lo[1] + by, z = R.lo[2] + bz;
        Offs o;
        make_offs(a, x, y, z, o);
        const int cell = o.x[1] + o.y[1] + o.z[1];   // position in a population slot
        float us[3];
        solid_velocity(R, x, y, z, us);
        // per-cell link sum in FP32 on the shifted populations (the rest-weight
        // parts of the link terms cancel); cells are combined in FP64
        float Fc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int s = 1; s < Q; ++s) {
            const int c0 = cslot(Q, s, 0), c1 = cslot(Q, s, 1), c2 = cslot(Q, s, 2);
            const int o_s = oslot(Q, s);
            const int nbx = o.x[1 + c0] + o.y[1 + c1] + o.z[1 + c2];
            float out_s, in_o;   // f*_s(x) and f*_o(x + c_s)
            if (a.layout == 1) {
                // esoteric twist: both on the link between x and x + c_s
                const int nl = eso_write_node(o, c0, c1, c2);
                out_s = Store<S>::ld(wslot_ptr<Q, S>(a, PH == 0 ? o_s : s) + nl);
                in_o = Store<S>::ld(wslot_ptr<Q, S>(a, PH == 0 ? s : o_s) + nl);
            } else if (PH == 0) {
                out_s = Store<S>::ld(wslot_ptr<Q, S>(a, o_s) + cell);
                in_o = Store<S>::ld(wslot_ptr<Q, S>(a, s) + nbx);
            } else {
                out_s = Store<S>::ld(wslot_ptr<Q, S>(a, s) + nbx);
                in_o = Store<S>::ld(wslot_ptr<Q, S>(a, o_s) + cell);
            }
            Fc[0] += (float(-c0) - us[0]) * in_o - (float(c0) - us[0]) * out_s;
            Fc[1] += (float(-c1) - us[1]) * in_o - (float(c1) - us[1]) * out_s;
            Fc[2] += (float(-c2) - us[2]) * in_o - (float(c2) - us[2]) * out_s;
        }
        const double r[3] = {(double)((float)x - R.cf[0]), (double)((float)y - R.cf[1]),
                             (double)((float)z - R.cf[2])};
        const double F0 = Fc[0], F1 = Fc[1], F2 = Fc[2];
        acc[0] += F0; acc[1] += F1; acc[2] += F2;
        acc[3] += r[1] * F2 - r[2] * F1;
        acc[4] += r[2] * F0 - r[0] * F2;
        acc[5] += r[0] * F1 - r[1] * F0;
    }
    __shared__ double sh[8][6];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        R.partial[blockIdx.x * 6 + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(R.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        // combine the block partials in a fixed order: strided per thread, then a tree
        for (int k = 0; k < 6; ++k) {
            double v = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
                v += ((volatile double*)R.partial)[b * 6 + k];
            v = warp_sum(v);
            __syncthreads();
            if (lane == 0) sh[warp][0] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][0];
                R.acc[k] = t;
                R.acc[6 + k] += t;
            }
        }
        if (threadIdx.x == 0) {
            *R.done = 0u;
            R.count[0] = 0;   // force cells
            R.count[1] = 0;   // wall cells
        }
    }
}

// ---------------------------------------------------------------------------
// evolve structure (torque-driven rotors): rigid rotation about the axis,
// I dOmega/dt = M.a - Q_gen(Omega), Q_gen = q_gen0 + k_gen Omega |Omega|,
// explicit Euler (dt = 1) from this step's torque; then the next step's frames
// ---------------------------------------------------------------------------
__global__ void evolve_kernel(const StepArgs a) {
    const int k = threadIdx.x;
    if (k >= a.nrot) return;
    const RotorDev& R = a.rot[k];
    if (!R.drive) return;
    DriveDev* D = R.drive;
    const double om = D->omega;
    const double q_aero = R.acc[3 + R.axis];
    const double q_gen = D->q_gen0 + D->k_gen * om * fabs(om);
    D->theta += om;
    D->omega = om + (q_aero - q_gen) / D->inertia;
    for (int b = 0; b < R.n_blades; ++b) {
        const double ang = D->theta + 2.0 * M_PI * (double)b / (double)R.n_blades;
        D->ck[b] = (float)cos(ang);
        D->sk[b] = (float)sin(ang);
    }
    D->omegaf = (float)D->omega;
}

// ---------------------------------------------------------------------------
// FP64 mass total (deterministic two-stage reduction) and drift check
// ---------------------------------------------------------------------------
// The mass total in fixed point.  B300's FP64 pipe is narrow (one FP64
// addition per stored value ran the check at 2.5 ms on rotor256, six times
// its memory time), so each stored value is turned, with integer
// operations, into a multiple of 2^-56 and summed in 128-bit integers; a
// thread's total goes to FP64 once and the block and grid sums are FP64.  A
// value of magnitude below 8 is taken exactly down to 2^-56 (the bits below
// are dropped: at most 2^-56 per value); anything larger, and inf or NaN,
// is added in FP64 instead, so the check still sees it.
constexpr int FIX_SHIFT = 56;

// binary32 bits -> value * 2^56 as a signed 64-bit integer (|value| < 8),
// or false when the value needs the FP64 path
__device__ __forceinline__ bool f32_fixed(unsigned u, long long& out) {
    const int eb = (int)((u >> 23) & 0xffu);
    if (eb >= 130) return false;                        // |value| >= 8, inf, NaN
    const long long m = (long long)((u & 0x7fffffu) | (eb ? 0x800000u : 0u));
    const int sh = (eb ? eb : 1) - 150 + FIX_SHIFT;     // value = m * 2^((eb ? eb : 1) - 150)
    const long long mag = sh >= 0 ? (m << sh) : (sh > -24 ? (m >> -sh) : 0);
    out = (u >> 31) ? -mag : mag;
    return true;
}

template <int S>
__device__ __forceinline__ unsigned stored_bits(typename Store<S>::T v) {
    if constexpr (S == ST_F32) return __float_as_uint(v);
    else return __float_as_uint(Store<S>::ld(&v));      // exact widening of FP16 / BF16
}

// Eight consecutive stored values (one 16-byte load for 16-bit storage, two
// for FP32), loaded ahead of their summation
template <int S>
struct Group8 {
    uint4 w[S == ST_F32 ? 2 : 1];
};
template <int S>
__device__ __forceinline__ Group8<S> load8(const typename Store<S>::T* p) {
    Group8<S> g;
#pragma unroll
    for (int k = 0; k < (S == ST_F32 ? 2 : 1); ++k) g.w[k] = reinterpret_cast<const uint4*>(p)[k];
    return g;
}

// Sum of eight consecutive stored values into the thread's 128-bit
// fixed-point accumulator (and its FP64 side sum)
template <int S>
__device__ __forceinline__ void sum8_fixed(const Group8<S>& grp, __int128& acc, double& side) {
    using T = typename Store<S>::T;
    const T* h = reinterpret_cast<const T*>(grp.w);
    long long g = 0;                                    // |g| < 8 * 2^59 = 2^62
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        long long x;
        if (f32_fixed(stored_bits<S>(h[k]), x)) g += x;
        else side += (double)Store<S>::ld(h + k);
    }
    acc += (__int128)g;
}

// FP64 value of a 128-bit fixed-point total (one rounding of the low word)
__device__ __forceinline__ double fixed_to_double(__int128 acc) {
    const long long hi = (long long)(acc >> 64);
    const unsigned long long lo = (unsigned long long)acc;
    return ((double)hi * 0x1p64 + (double)lo) * 0x1p-56;
}

template <int S>
__global__ void __launch_bounds__(256, MASS_BLOCKS / 148) mass_kernel(const MassArgs m) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(m.f);
    const long long groups = m.count / 8;
    __int128 acc = 0;
    double v = 0.0;
    // four groups in flight per thread: one 16-byte load each left the
    // kernel short of requests in flight (0.47 of HBM for FP32 storage)
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < groups; i += 4 * stride) {
        Group8<S> g4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) g4[k] = load8<S>(f + 8 * (i + k * stride));
#pragma unroll
        for (int k = 0; k < 4; ++k) sum8_fixed<S>(g4[k], acc, v);
    }
    for (; i < groups; i += stride) sum8_fixed<S>(load8<S>(f + 8 * i), acc, v);
    v += fixed_to_double(acc);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (long long i = 8 * groups; i < m.count; ++i) v += (double)Store<S>::ld(f + i);
    // a slab's halo planes stand for its neighbours' cells: take them out again
    const long long nh = (long long)(m.halo_lo + m.halo_hi) * m.nxy;
    if (nh > 0) {
        const long long slots = m.count / m.N;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < slots * nh;
             i += (long long)gridDim.x * blockDim.x) {
            const long long sl = i / nh, r = i % nh;
            const long long cell = r < (long long)m.halo_lo * m.nxy ? r : m.N - nh + r;
            v -= (double)Store<S>::ld(f + sl * m.N + cell);
        }
    }
    __shared__ double sh[8];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        m.partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(m.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += ((volatile double*)m.partial)[b];
        t = warp_sum(t);
        __syncthreads();
        if (lane == 0) sh[warp] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
            s += m.shift_mass;
            *m.out = s;
            if (!(fabs(s) < 1e300)) atomicOr(m.err, ERR_NONFINITE);
            else if (m.tol >= 0.0 && fabs(s - m.ref) > m.tol * fabs(m.ref)) atomicOr(m.err, ERR_MASS);
            *m.done = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// initial state, macroscopic fields, single-cell collisions (unit checks)
// ---------------------------------------------------------------------------
template <int Q, int S>
__global__ void init_kernel(const StepArgs a, const float* rho, const float* u, float drho0, float u0x, float u0y,
                            float u0z) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= a.n[0]) return;
    const int cell = (z * a.n[1] + y) * a.n[0] + x;
    float uu[3] = {u0x, u0y, u0z};
    float drho = drho0;
    if (rho) drho = rho[cell] - 1.0f;
    if (u) { uu[0] = u[cell]; uu[1] = u[a.N + cell]; uu[2] = u[2 * a.N + cell]; }
    float g[Q];
    equilibrium<Q>(g, drho, uu);
    if (a.layout == 1) {
        // even-step layout of the esoteric twist: f_s on the link towards x - c_s
        Offs o;
        make_offs(a, x, y, z, o);
#pragma unroll
        for (int s = 0; s < Q; ++s)
            Store<S>::st(slot_ptr<Q, S>(a, s) + eso_read_node(o, cslot(Q, s, 0), cslot(Q, s, 1), cslot(Q, s, 2)),
                         g[s]);
        return;
    }
    const int pc = (z * a.n[1] + y) * a.n[0] + xmap(a, x);
#pragma unroll
    for (int s = 0; s < Q; ++s) Store<S>::st(slot_ptr<Q, S>(a, s) + pc, g[s]);
}

template <int Q, int S, int PH>
__global__ void fields_kernel(const StepArgs a, float* rho, float* u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= a.n[0]) return;
    const int cell = (z * a.n[1] + y) * a.n[0] + x;
    Offs o;
    make_offs(a, x, y, z, o);
    float g[Q];
    if (a.layout == 1) load_pre<Q, S, PH, 1>(a, o, g);
    else load_pre<Q, S, PH, 0>(a, o, g);
    float drho, j[3];
    moments01<Q>(g, drho, j);
    const float r = 1.0f + drho;
    rho[cell] = r;
    u[cell] = j[0] / r;
    u[a.N + cell] = j[1] / r;
    u[2 * a.N + cell] = j[2] / r;
}

template <int Q>
__global__ void debug_collide_kernel(int n, const float* gin, const float* d, const float* uB, const float* sigma,
                                     const float* S, float tau_mo, float Ksmag, float* gout) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float g[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) g[s] = gin[(long long)c * Q + s];
    float u[3];
    if (d) {
        Band B;
        B.d = d[c];
        B.uB[0] = uB[3 * c]; B.uB[1] = uB[3 * c + 1]; B.uB[2] = uB[3 * c + 2];
        B.sigma = sigma[c];
#pragma unroll
        for (int k = 0; k < 6; ++k) B.S[k] = S[6 * c + k];
        collide<Q, true>(g, B, tau_mo, Ksmag, u);
    } else {
        Band B0;
        collide<Q, false>(g, B0, tau_mo, Ksmag, u);
    }
#pragma unroll
    for (int s = 0; s < Q; ++s) gout[(long long)c * Q + s] = g[s];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static dim3 cell_block(int nx) {
    if (nx >= 128) return dim3(128, 1, 1);
    const int bx = ((nx + 31) / 32) * 32;
    return dim3(bx, 128 / bx >= 1 ? 128 / bx : 1, 1);
}

template <int Q, int S, int L>
static cudaError_t launch_collide_l(const StepArgs& a, cudaStream_t s) {
    const int* n = a.part == 2 ? a.rot[a.part_rotor].n : a.n;
    const dim3 blk = cell_block(n[0]);
    if (a.part != 2 && a.pairs && !a.d0) {
        const int half = (n[0] + 1) / 2;
        const dim3 pb = cell_block(half);
        const dim3 pg((half + pb.x - 1) / pb.x, (n[1] + pb.y - 1) / pb.y, a.z1 - a.z0);
        if (L == 0 && a.xpair) {
            if (a.phase == 0) collide_halves_kernel<Q, S, 0><<<pg, pb, 0, s>>>(a);
            else collide_halves_kernel<Q, S, 1><<<pg, pb, 0, s>>>(a);
        } else {
            if (a.phase == 0) collide_pair_kernel<Q, S, 0, L><<<pg, pb, 0, s>>>(a);
            else collide_pair_kernel<Q, S, 1, L><<<pg, pb, 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    const dim3 grd((n[0] + blk.x - 1) / blk.x, (n[1] + blk.y - 1) / blk.y, a.part == 2 ? n[2] : a.z1 - a.z0);
    if (a.d0) {
        if (a.phase == 0) collide_kernel<Q, S, 0, true, L><<<grd, blk, 0, s>>>(a);
        else collide_kernel<Q, S, 1, true, L><<<grd, blk, 0, s>>>(a);
    } else {
        if (a.phase == 0) collide_kernel<Q, S, 0, false, L><<<grd, blk, 0, s>>>(a);
        else collide_kernel<Q, S, 1, false, L><<<grd, blk, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t launch_collide_t(const StepArgs& a, cudaStream_t s) {
    return a.layout == 1 ? launch_collide_l<Q, S, 1>(a, s) : launch_collide_l<Q, S, 0>(a, s);
}

template <int Q, int S>
static cudaError_t launch_band_t(const StepArgs& a, cudaStream_t s) {
    if (a.nrot == 0) return cudaSuccess;
    long long maxrows = 0;
    for (int k = 0; k < a.nrot; ++k) {
        const long long r = (long long)a.rot[k].n[1] * a.rot[k].n[2];
        maxrows = r > maxrows ? r : maxrows;
    }
    constexpr int WPB = BAND_THREADS / 32;
    long long blocks = (maxrows + WPB - 1) / WPB;
    // at most four 128-thread blocks per SM: the embedding runs beside the
    // bulk launch, and fewer blocks leave it more of the GPU (rotor256 step
    // 0.797 -> 0.790 ms with two 256-thread blocks); a 128-thread block of 48
    // registers fits what one retiring bulk block frees (rotor128 40 -> 33 us)
    if (blocks > 148 * 4) blocks = 148 * 4;
    if (blocks < 1) blocks = 1;
    band_kernel<<<dim3((unsigned)blocks, a.nrot), BAND_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t launch_wall_t(const StepArgs& a, cudaStream_t s) {
    if (a.nrot == 0 || !a.wall_model) return cudaSuccess;
    // small rotor boxes (few wall cells): four lanes per cell, so the corner
    // gathers of a short list spread over more SMs; large boxes: one lane per
    // cell (four lanes would repeat each FP64 Newton solve four times)
    long long box = 0;
    for (int k = 0; k < a.nrot; ++k) box = a.rot[k].box_cells > box ? a.rot[k].box_cells : box;
    if (box <= WALL_SMALL_BOX) {
        const dim3 grd(WALL_GROUP_BLOCKS, a.nrot);
        if (a.phase == 0) wall_kernel<Q, S, 0, 4><<<grd, WALL_THREADS, 0, s>>>(a);
        else wall_kernel<Q, S, 1, 4><<<grd, WALL_THREADS, 0, s>>>(a);
    } else {
        const dim3 grd(WALL_BLOCKS, a.nrot);
        if (a.phase == 0) wall_kernel<Q, S, 0, 1><<<grd, WALL_THREADS, 0, s>>>(a);
        else wall_kernel<Q, S, 1, 1><<<grd, WALL_THREADS, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t launch_band_strain_t(const StepArgs& a, cudaStream_t s) {
    if (a.nrot == 0 || !(a.sigma_band < 1.0f)) return cudaSuccess;
    const dim3 grd(WALL_BLOCKS, a.nrot);
    if (a.phase == 0) band_strain_kernel<Q, S, 0><<<grd, WALL_THREADS, 0, s>>>(a);
    else band_strain_kernel<Q, S, 1><<<grd, WALL_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t launch_force_t(const StepArgs& a, cudaStream_t s) {
    if (a.nrot == 0) return cudaSuccess;
    const dim3 grd(FORCE_BLOCKS, a.nrot);
    if (a.phase == 0) force_kernel<Q, S, 0><<<grd, 256, 0, s>>>(a);
    else force_kernel<Q, S, 1><<<grd, 256, 0, s>>>(a);
    return cudaGetLastError();
}

#define HL_DISPATCH(Q, S, FN, ...)                                                   \
    do {                                                                             \
        if (Q == 19 && S == ST_F32) return FN<19, ST_F32>(__VA_ARGS__);              \
        if (Q == 19 && S == ST_F16S) return FN<19, ST_F16S>(__VA_ARGS__);            \
        if (Q == 19 && S == ST_BF16S) return FN<19, ST_BF16S>(__VA_ARGS__);          \
        if (Q == 27 && S == ST_F32) return FN<27, ST_F32>(__VA_ARGS__);              \
        if (Q == 27 && S == ST_F16S) return FN<27, ST_F16S>(__VA_ARGS__);            \
        if (Q == 27 && S == ST_BF16S) return FN<27, ST_BF16S>(__VA_ARGS__);          \
        return cudaErrorInvalidValue;                                                \
    } while (0)

cudaError_t launch_collide(int Q, int S, const StepArgs& a, cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_collide_t, a, s);
}
cudaError_t launch_band(int Q, int S, const StepArgs& a, cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_band_t, a, s);
}
cudaError_t launch_wall(int Q, int S, const StepArgs& a, cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_wall_t, a, s);
}
cudaError_t launch_band_strain(int Q, int S, const StepArgs& a, cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_band_strain_t, a, s);
}
cudaError_t launch_force(int Q, int S, const StepArgs& a, cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_force_t, a, s);
}

cudaError_t launch_evolve(const StepArgs& a, cudaStream_t s) {
    bool any = false;
    for (int k = 0; k < a.nrot; ++k) any = any || a.rot[k].drive;
    if (!any) return cudaSuccess;
    evolve_kernel<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mass(int Q, int S, const MassArgs& m, cudaStream_t s) {
    (void)Q;
    switch (S) {
        case ST_F32: mass_kernel<ST_F32><<<MASS_BLOCKS, 256, 0, s>>>(m); break;
        case ST_F16S: mass_kernel<ST_F16S><<<MASS_BLOCKS, 256, 0, s>>>(m); break;
        case ST_BF16S: mass_kernel<ST_BF16S><<<MASS_BLOCKS, 256, 0, s>>>(m); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t launch_init_t(const StepArgs& a, const float* rho, const float* u, float drho0,
                                 const float u0[3], cudaStream_t s) {
    const dim3 grd((a.n[0] + 127) / 128, a.n[1], a.n[2]);
    init_kernel<Q, S><<<grd, 128, 0, s>>>(a, rho, u, drho0, u0[0], u0[1], u0[2]);
    return cudaGetLastError();
}
cudaError_t launch_init(int Q, int S, const StepArgs& a, const float* rho, const float* u, float drho0,
                        const float u0[3], cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_init_t, a, rho, u, drho0, u0, s);
}

template <int Q, int S>
static cudaError_t launch_fields_t(const StepArgs& a, float* rho, float* u, cudaStream_t s) {
    const dim3 grd((a.n[0] + 127) / 128, a.n[1], a.n[2]);
    if (a.phase == 0) fields_kernel<Q, S, 0><<<grd, 128, 0, s>>>(a, rho, u);
    else fields_kernel<Q, S, 1><<<grd, 128, 0, s>>>(a, rho, u);
    return cudaGetLastError();
}
cudaError_t launch_fields(int Q, int S, const StepArgs& a, float* rho, float* u, cudaStream_t s) {
    HL_DISPATCH(Q, S, launch_fields_t, a, rho, u, s);
}

// halo message: slot list x consecutive planes, raw stored values (no conversion)
template <typename T>
__global__ void __launch_bounds__(256) halo_kernel(const HaloArgs h) {
    const long long per_slot = (long long)h.nplanes * h.nxy;
    const long long n = (long long)h.nslot * per_slot;
    T* f = static_cast<T*>(h.f);
    T* b = static_cast<T*>(h.buf);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / per_slot);
        const long long c = (long long)h.plane * h.nxy + (i - (long long)k * per_slot);
        T* p = f + (long long)h.slots[k] * h.N + c;
        if (h.import_) *p = b[i];
        else b[i] = *p;
    }
}

cudaError_t launch_halo(int storage, const HaloArgs& h, cudaStream_t s) {
    const long long n = (long long)h.nslot * h.nplanes * h.nxy;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (blocks < 1) blocks = 1;
    if (storage == ST_F32) halo_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(h);
    else halo_kernel<unsigned short><<<(unsigned)blocks, 256, 0, s>>>(h);
    return cudaGetLastError();
}

cudaError_t launch_debug_collide(int Q, int n, const float* g_in, const float* d, const float* uB,
                                 const float* sigma, const float* S, float tau_mo, float Ksmag, float* g_out,
                                 cudaStream_t s) {
    const int blocks = (n + 127) / 128;
    if (n <= 0) return cudaSuccess;
    if (Q == 19)
        debug_collide_kernel<19><<<blocks, 128, 0, s>>>(n, g_in, d, uB, sigma, S, tau_mo, Ksmag, g_out);
    else if (Q == 27)
        debug_collide_kernel<27><<<blocks, 128, 0, s>>>(n, g_in, d, uB, sigma, S, tau_mo, Ksmag, g_out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace hl
