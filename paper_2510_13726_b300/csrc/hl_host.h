// Host-side internals shared by the C ABI (hl_api.cu) and the reverse
// sweep (hl_grad.cu): workspace layouts, the lattice handle, error helpers
// and the step issue.  Not part of the public header.
#pragma once

#include <cstdio>
#include <vector>

#include "hl_internal.h"
#include "hlbm.h"

namespace hl {
namespace host {

constexpr size_t ALIGN = 256;

inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t f, uplane0, uplane1, modes, err, mpartial, mdone, mout, total;
};

inline int store_bytes(int storage) { return storage == HL_STORE_F32 ? 4 : 2; }

inline long long plane_cells(const hl_config& c) {
    const int n[3] = {c.nx, c.ny, c.nz};
    return (long long)n[(c.flow_axis + 1) % 3] * n[(c.flow_axis + 2) % 3];
}

inline Layout lattice_layout(const hl_config& c) {
    Layout L{};
    const long long N = (long long)c.nx * c.ny * c.nz;
    size_t o = 0;
    L.f = o; o = align_up(o + (size_t)c.q * N * store_bytes(c.storage));
    L.uplane0 = o; o = align_up(o + sizeof(float) * 3 * plane_cells(c));
    L.uplane1 = o; o = align_up(o + sizeof(float) * 3 * plane_cells(c));
    L.modes = o; o = align_up(o + sizeof(float) * 9 * (c.n_modes > 0 ? c.n_modes : 1));
    L.err = o; o = align_up(o + sizeof(unsigned));
    L.mpartial = o; o = align_up(o + sizeof(double) * MASS_BLOCKS);
    L.mdone = o; o = align_up(o + sizeof(unsigned));
    L.mout = o; o = align_up(o + sizeof(double));
    L.total = o;
    return L;
}

struct RotorLayout {
    size_t sdf, d, flags, wm, utau, active, list[2], wlist[2], wphi[2], wwhich[2], count, done, partial, acc, drive,
        total;
};

// The cell lists of the embedding (force cells, wall cells and their data)
// are kept twice, by step parity, so that the next step's embedding can run
// while this step's force reduction still reads its lists; the counters of
// both sets are four ints from `count` (set p at count + 2 p).
constexpr size_t COUNT_BYTES = 4 * sizeof(int);

inline RotorLayout rotor_layout(long long ngrid, long long box) {
    RotorLayout L{};
    size_t o = 0;
    L.sdf = o; o = align_up(o + sizeof(float) * ngrid);
    L.d = o; o = align_up(o + sizeof(float) * box);
    L.flags = o; o = align_up(o + box);
    L.wm = o; o = align_up(o + sizeof(float) * 9 * box);
    L.utau = o; o = align_up(o + sizeof(double) * box);
    L.active = o; o = align_up(o + box);
    for (int p = 0; p < 2; ++p) {
        L.list[p] = o; o = align_up(o + sizeof(int) * box);
        L.wlist[p] = o; o = align_up(o + sizeof(int) * box);
        L.wphi[p] = o; o = align_up(o + sizeof(float) * box);
        L.wwhich[p] = o; o = align_up(o + box);
    }
    L.count = o; o = align_up(o + COUNT_BYTES);
    L.done = o; o = align_up(o + sizeof(unsigned));
    L.partial = o; o = align_up(o + sizeof(double) * 6 * FORCE_BLOCKS);
    L.acc = o; o = align_up(o + sizeof(double) * 12);
    L.drive = o; o = align_up(o + sizeof(DriveDev));
    L.total = o;
    return L;
}

struct RotorHost {
    hl_rotor_geometry geom;
    double omega, pitch;
    double pitch_sets;       // pitch that decides the cell sets while they are frozen
    bool driven;             // torque-driven rotation (device state at dev.drive)
    bool clip[2];            // the box is cut by the slab's lower / upper halo face
    RotorDev dev;
    char* ws;
    RotorLayout L;
};

}  // namespace host
}  // namespace hl

struct hl_lattice {
    hl_config cfg;
    long long N;
    cudaStream_t stream;
    char* ws;
    hl::host::Layout L;
    void* f;
    float* uplane[2];
    float* modes;
    unsigned* err;
    double mass_ref;
    long long t;
    long long n_avg;
    int nrot;
    hl::host::RotorHost rot[hl::MAXROT];
    const float* d0;         // caller's static porosity multiplier [N], or null
    const float* inflow;     // caller's inflow velocity plane [3][plane], or null (synthetic modes)
    long long halo_t[2];     // slab: time of the last halo import of the lower / upper face (-1: none)
    long long deep_t[2];     // slab: time of the last deep halo import of each face (-1: none)
    bool clip_face[2];       // a rotor box is cut by the lower / upper halo face
    // a rotor box cut by a halo face: the force reduction of a step reads the
    // neighbouring slab's cells, so it runs after the halo exchange, at the
    // start of the next step or before the next load query
    bool force_pending;
    hl::StepArgs pending;
    bool frozen;             // cell sets decided by RotorHost::pitch_sets
    char msg[256];
    // second stream for the rotor-box chain, and the events that order it
    cudaStream_t aux;
    cudaEvent_t ev_bulk[2], ev_box[2], ev_fork, ev_join;
    bool have_aux;
    // third stream: the force reduction (and the driven-rotor update) of a
    // step, beside the next step's embedding and wall model
    cudaStream_t fst;
    cudaEvent_t ev_force[2], ev_join_f;
    // per-kernel event timing (hl_profile_begin / hl_profile_end)
    bool prof_on;
    int prof_cap;
    std::vector<cudaEvent_t> prof_ev[6];   // start/stop pairs per kernel kind
};

namespace hl {
namespace host {

hl_status fail(hl_lattice* lat, hl_status code, const char* what);
hl_status cuda_fail(hl_lattice* lat, cudaError_t e, const char* where);

#define HL_CUDA(lat, call)                                                   \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::hl::host::cuda_fail(lat, e_, #call); \
    } while (0)

// kernel arguments of the lattice's current step (in-place populations)
StepArgs make_args(const hl_lattice* lat);
// odd-step shifted bases from slot / wslot (call after changing either)
void set_shifted_bases(StepArgs* a, int q, int esize);
// issue one step with the given arguments: serial, or bulk / box chain on two
// streams; with_force = false skips the force reduction (and resets the
// cell-list counters it would reset)
hl_status issue_step(hl_lattice* lat, const StepArgs& a, bool with_force);
hl_status read_error_word(hl_lattice* lat);

}  // namespace host
}  // namespace hl
