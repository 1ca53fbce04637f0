// Host side of the C ABI declared in include/hlbm.h.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hl_host.h"

using namespace hl;
using namespace hl::host;

namespace hl {
namespace host {

hl_status fail(hl_lattice* lat, hl_status code, const char* what) {
    if (lat) std::snprintf(lat->msg, sizeof lat->msg, "%s", what);
    return code;
}

hl_status cuda_fail(hl_lattice* lat, cudaError_t e, const char* where) {
    if (lat) std::snprintf(lat->msg, sizeof lat->msg, "%s: %s", where, cudaGetErrorString(e));
    return HL_ERR_CUDA;
}

}  // namespace host
}  // namespace hl

namespace {

bool valid_config(const hl_config* c) {
    if (!c) return false;
    if (c->nx < 3 || c->ny < 3 || c->nz < 3) return false;
    if ((long long)c->nx * c->ny * c->nz > (1LL << 31) - 1) return false;
    if (c->nx > 65535 * 128 || c->ny > 65535 || c->nz > 65535) return false;
    if (c->q != 19 && c->q != 27) return false;
    if (c->storage < 0 || c->storage > 2) return false;
    if (c->flow_axis < 0 || c->flow_axis > 2) return false;
    if (!(c->tau_mo > 0.5) || !(c->c_smag >= 0.0) || !(c->eps_h > 0.0)) return false;
    if (!(c->sigma_band >= 0.0 && c->sigma_band <= 1.0)) return false;
    if (c->n_modes < 0 || (c->n_modes > 0 && !c->modes)) return false;
    if (c->wm_maxit < 0 || c->wm_maxit > 1000 || !(c->wm_ysample > 0.0)) return false;
    if (c->mass_check_every < 0) return false;
    if (c->layout < 0 || c->layout > 2) return false;
    if (c->layout == 2 && c->nx % 2) return false;                      // x halves need nx even
    // z_offset may be -1: the first slab of a periodic z decomposition starts with the last slab's plane
    if (c->halo_lo < 0 || c->halo_lo > HALO_MAX || c->halo_hi < 0 || c->halo_hi > HALO_MAX) return false;
    if ((c->halo_lo || c->halo_hi) && c->layout == 1) return false;   // slabs use the AA pattern
    // the owned planes fill a neighbour's deep halo
    const int owned = c->nz - c->halo_lo - c->halo_hi;
    if (owned < 1 || owned < c->halo_lo || owned < c->halo_hi) return false;
    return true;
}

}  // namespace

namespace hl {
namespace host {

void set_shifted_bases(StepArgs* a, int q, int esize) {
    std::vector<int> c(3 * q);
    std::vector<double> w(q);
    hl_velocity_set(q, c.data(), w.data());
    const int P = (q - 1) / 2;
    for (int s = 0; s < q; ++s) {
        const int sbar = s == 0 ? 0 : (s <= P ? s + P : s - P);
        // integer arithmetic on the addresses: the shifted bases may lie
        // outside the buffer, every address formed from them lies inside
        if (a->layout == 1) {
            // esoteric twist: the link between x and x + c_s lives at cell
            // x + max(c_s, 0); a cell reads f_s over the link to x - c_s (at
            // x + max(-c_s, 0)) and writes f*_s onto the link to x + c_s, in
            // slot s / sbar (reads) and sbar / s (writes) at even / odd steps
            long long Dp = 0, Dn = 0;
            const long long stride[3] = {1, a->n[0], a->nxy};
            for (int k = 0; k < 3; ++k) {
                Dp += (c[3 * s + k] > 0 ? 1 : 0) * stride[k];
                Dn += (c[3 * s + k] < 0 ? 1 : 0) * stride[k];
            }
            const int rs = a->phase == 0 ? s : sbar, ws = a->phase == 0 ? sbar : s;
            a->rshift[s] = reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(a->slot[rs]) + Dn * esize);
            a->wshift[s] = reinterpret_cast<void*>(reinterpret_cast<uintptr_t>(a->wslot[ws]) + Dp * esize);
        } else {
            // with x halves a cell's x neighbours sit two positions away
            // (away from the wrap and the seam between the halves)
            const long long D = (a->xpair ? 2 : 1) * (long long)c[3 * s] + (long long)c[3 * s + 1] * a->n[0] +
                                (long long)c[3 * s + 2] * a->nxy;
            a->rshift[s] = reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(a->slot[sbar]) - D * esize);
            a->wshift[s] = reinterpret_cast<void*>(reinterpret_cast<uintptr_t>(a->wslot[s]) + D * esize);
        }
    }
    // packed cell pairs need two-element alignment of every pair they touch:
    // x even, and with nx (hence nx * ny) even a shift by c_s keeps the parity of c_x
    bool pairs = a->n[0] % 2 == 0;
    for (int s = 0; s < q; ++s)
        pairs = pairs && reinterpret_cast<uintptr_t>(a->slot[s]) % (2 * esize) == 0 &&
                reinterpret_cast<uintptr_t>(a->wslot[s]) % (2 * esize) == 0;
    a->pairs = pairs ? 1 : 0;
}

StepArgs make_args(const hl_lattice* lat) {
    const hl_config& c = lat->cfg;
    StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.f = lat->f;
    a.N = lat->N;
    for (int q = 0; q < c.q; ++q) {
        a.slot[q] = static_cast<char*>(lat->f) + (size_t)q * lat->N * store_bytes(c.storage);
        a.wslot[q] = a.slot[q];
    }
    a.d0 = lat->d0;
    a.inflow_plane = lat->inflow;
    a.n[0] = c.nx; a.n[1] = c.ny; a.n[2] = c.nz;
    a.nxy = c.nx * c.ny;
    a.nplane = (int)plane_cells(c);
    a.phase = (int)(lat->t & 1);
    a.layout = c.layout == 1 ? 1 : 0;
    a.xpair = c.layout == 2 ? 1 : 0;
    a.hx = c.nx / 2;
    a.t = lat->t;
    a.flow_axis = c.flow_axis;
    a.open = c.open_boundaries;
    // a slab (halo planes along z) has the inlet / outlet of a z flow only where it has no halo
    a.open_lo = (c.flow_axis == 2 && c.halo_lo) ? 0 : 1;
    a.open_hi = (c.flow_axis == 2 && c.halo_hi) ? 0 : 1;
    a.z0 = c.halo_lo;
    a.z1 = c.nz - c.halo_hi;
    a.zoff = c.z_offset;
    a.tau_mo = (float)c.tau_mo;
    a.Ksmag = (float)(18.0 * std::sqrt(2.0) * c.c_smag * c.c_smag);
    a.u_in = (float)c.u_in;
    a.inflow_shift = (float)(c.u_in * (double)lat->t);
    a.eps_half = (float)(0.5 * c.eps_h);
    a.inv_eps = (float)(1.0 / c.eps_h);
    a.transition = c.transition;
    a.wall_model = c.wall_model;
    a.wmE = c.wm_E;
    a.wmK = c.wm_kappa;
    a.wmYs = (float)c.wm_ysample;
    a.wmTol = c.wm_tol;
    a.wmMaxit = c.wm_maxit;
    a.nu = (c.tau_mo - 0.5) / 3.0;
    a.sigma_band = (float)c.sigma_band;
    a.modes = lat->modes;
    a.n_modes = c.n_modes;
    a.uplane_prev = lat->uplane[(lat->t + 1) & 1];
    a.uplane_cur = lat->uplane[lat->t & 1];
    a.err = lat->err;
    a.nrot = lat->nrot;
    for (int k = 0; k < lat->nrot; ++k) {
        const RotorHost& R = lat->rot[k];
        a.rot[k] = R.dev;
        // rotor kinematics: theta = theta0 + Omega t, blade k at theta + 2 pi k / n_blades;
        // the binary32 frames are rounded once from FP64
        const double th = R.geom.phase0 + R.omega * (double)lat->t;
        for (int b = 0; b < R.geom.n_blades; ++b) {
            const double ang = th + 2.0 * M_PI * (double)b / (double)R.geom.n_blades;
            a.rot[k].ck[b] = (float)std::cos(ang);
            a.rot[k].sk[b] = (float)std::sin(ang);
        }
        a.rot[k].cp = (float)std::cos(R.pitch);
        a.rot[k].sp = (float)std::sin(R.pitch);
        const double ps = lat->frozen ? R.pitch_sets : R.pitch;
        a.rot[k].cpD = (float)std::cos(ps);
        a.rot[k].spD = (float)std::sin(ps);
        a.rot[k].frozen = lat->frozen ? 1 : 0;
        // the cell lists and counters of this step's parity
        const int p = (int)(lat->t & 1);
        a.rot[k].list = reinterpret_cast<int*>(R.ws + R.L.list[p]);
        a.rot[k].wlist = reinterpret_cast<int*>(R.ws + R.L.wlist[p]);
        a.rot[k].wphi = reinterpret_cast<float*>(R.ws + R.L.wphi[p]);
        a.rot[k].wwhich = reinterpret_cast<signed char*>(R.ws + R.L.wwhich[p]);
        a.rot[k].count = R.dev.count + 2 * p;
    }
    set_shifted_bases(&a, c.q, store_bytes(c.storage));   // needs n and nxy
    return a;
}

hl_status read_error_word(hl_lattice* lat) {
    unsigned e = 0;
    HL_CUDA(lat, cudaMemcpyAsync(&e, lat->err, sizeof e, cudaMemcpyDeviceToHost, lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    if (e & ERR_NONFINITE) return fail(lat, HL_ERR_NONFINITE, "non-finite density on the device");
    if (e & ERR_MASS) return fail(lat, HL_ERR_MASS, "total mass drifted beyond mass_tol");
    if (e & ERR_GEOMETRY)
        return fail(lat, HL_ERR_GEOMETRY, "a wall-model sample or a band-strain stencil left the rotor box: pad the blade grid");
    return HL_OK;
}

}  // namespace host
}  // namespace hl

namespace {

// N_owned * sum_i w_i: the mass of the storage shift over the cells the
// lattice owns (a slab's halo planes excluded)
double shift_mass(const hl_lattice* lat) {
    std::vector<int> c(3 * lat->cfg.q);
    std::vector<double> w(lat->cfg.q);
    hl_velocity_set(lat->cfg.q, c.data(), w.data());
    double s = 0.0;
    for (double v : w) s += v;
    const long long nxy = (long long)lat->cfg.nx * lat->cfg.ny;
    return s * (double)(lat->N - (long long)(lat->cfg.halo_lo + lat->cfg.halo_hi) * nxy);
}

hl_status compute_mass(hl_lattice* lat, double tol, double* out) {
    MassArgs m;
    m.f = lat->f;
    m.count = (long long)lat->cfg.q * lat->N;
    m.N = lat->N;
    m.nxy = lat->cfg.nx * lat->cfg.ny;
    m.halo_lo = lat->cfg.halo_lo;
    m.halo_hi = lat->cfg.halo_hi;
    m.shift_mass = shift_mass(lat);
    m.ref = lat->mass_ref;
    m.tol = tol;
    m.partial = reinterpret_cast<double*>(lat->ws + lat->L.mpartial);
    m.done = reinterpret_cast<unsigned*>(lat->ws + lat->L.mdone);
    m.out = reinterpret_cast<double*>(lat->ws + lat->L.mout);
    m.err = lat->err;
    HL_CUDA(lat, launch_mass(lat->cfg.q, lat->cfg.storage, m, lat->stream));
    if (out) {
        HL_CUDA(lat, cudaMemcpyAsync(out, m.out, sizeof(double), cudaMemcpyDeviceToHost, lat->stream));
        HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    }
    return HL_OK;
}

hl_status reset_outlet_plane(hl_lattice* lat, const float u0[3]) {
    const long long np = plane_cells(lat->cfg);
    std::vector<float> h(3 * np);
    for (int k = 0; k < 3; ++k)
        for (long long p = 0; p < np; ++p) h[k * np + p] = u0[k];
    for (int b = 0; b < 2; ++b)
        HL_CUDA(lat, cudaMemcpyAsync(lat->uplane[b], h.data(), sizeof(float) * h.size(),
                                     cudaMemcpyHostToDevice, lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    return HL_OK;
}

}  // namespace

extern "C" {

void hl_config_defaults(hl_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->q = 19;
    c->storage = HL_STORE_F32;
    c->flow_axis = 2;
    c->open_boundaries = 1;
    c->tau_mo = 0.5005;
    c->c_smag = 0.1;
    c->u_in = 0.05;
    c->sigma_band = 1.0;
    c->eps_h = 2.0;
    c->transition = 0;
    c->wall_model = 1;
    c->wm_E = 9.8;
    c->wm_kappa = 0.41;
    c->wm_ysample = 2.0;
    c->wm_tol = 1e-4;
    c->wm_maxit = 10;
    c->mass_check_every = 100;
    c->mass_tol = 0.05;
    c->overlap = 1;
}

hl_status hl_workspace_size(const hl_config* cfg, size_t* bytes) {
    if (!valid_config(cfg) || !bytes) return HL_ERR_ARG;
    *bytes = lattice_layout(*cfg).total;
    return HL_OK;
}

hl_status hl_lattice_init(hl_lattice** out, const hl_config* cfg, void* d_workspace, size_t bytes,
                          void* stream) {
    if (!out || !valid_config(cfg) || !d_workspace) return HL_ERR_ARG;
    if (reinterpret_cast<size_t>(d_workspace) % ALIGN) return HL_ERR_ARG;
    const Layout L = lattice_layout(*cfg);
    if (bytes < L.total) return HL_ERR_WORKSPACE;
    hl_lattice* lat = new (std::nothrow) hl_lattice();
    if (!lat) return HL_ERR_ARG;
    lat->cfg = *cfg;
    lat->cfg.modes = nullptr;
    lat->N = (long long)cfg->nx * cfg->ny * cfg->nz;
    lat->stream = static_cast<cudaStream_t>(stream);
    lat->ws = static_cast<char*>(d_workspace);
    lat->L = L;
    lat->f = lat->ws + L.f;
    lat->uplane[0] = reinterpret_cast<float*>(lat->ws + L.uplane0);
    lat->uplane[1] = reinterpret_cast<float*>(lat->ws + L.uplane1);
    lat->modes = reinterpret_cast<float*>(lat->ws + L.modes);
    lat->err = reinterpret_cast<unsigned*>(lat->ws + L.err);
    std::snprintf(lat->msg, sizeof lat->msg, "no error");
    lat->halo_t[0] = lat->halo_t[1] = -1;
    lat->deep_t[0] = lat->deep_t[1] = -1;
    hl_status st;
    if (cfg->n_modes > 0) {
        std::vector<float> m(9 * cfg->n_modes);
        for (size_t i = 0; i < m.size(); ++i) m[i] = (float)cfg->modes[i];
        cudaError_t e = cudaMemcpyAsync(lat->modes, m.data(), sizeof(float) * m.size(),
                                        cudaMemcpyHostToDevice, lat->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
        if (e != cudaSuccess) { delete lat; return HL_ERR_CUDA; }
    }
    cudaError_t e = cudaMemsetAsync(lat->ws + L.err, 0, L.total - L.err, lat->stream);
    if (e != cudaSuccess) { delete lat; return HL_ERR_CUDA; }
    float u0[3] = {0.f, 0.f, 0.f};
    u0[cfg->flow_axis] = (float)cfg->u_in;
    e = launch_init(cfg->q, cfg->storage, make_args(lat), nullptr, nullptr, 0.0f, u0, lat->stream);
    if (e != cudaSuccess) { delete lat; return HL_ERR_CUDA; }
    if ((st = reset_outlet_plane(lat, u0)) != HL_OK) { delete lat; return st; }
    double m0 = 0.0;
    if ((st = compute_mass(lat, -1.0, &m0)) != HL_OK) { delete lat; return st; }
    lat->mass_ref = m0;
    if (cfg->overlap) {
        int lo = 0, hi = 0;
        bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
                  cudaStreamCreateWithPriority(&lat->aux, cudaStreamNonBlocking, hi) == cudaSuccess;
        for (int k = 0; ok && k < 2; ++k)
            ok = cudaEventCreateWithFlags(&lat->ev_bulk[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&lat->ev_box[k], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&lat->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&lat->ev_join, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaStreamCreateWithPriority(&lat->fst, cudaStreamNonBlocking, hi) == cudaSuccess;
        for (int k = 0; ok && k < 2; ++k)
            ok = cudaEventCreateWithFlags(&lat->ev_force[k], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&lat->ev_join_f, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) { hl_destroy(lat); return HL_ERR_CUDA; }
        lat->have_aux = true;
    }
    *out = lat;
    return HL_OK;
}

// reach of a rotor: every cell from which a blade sample can land inside the
// blade grid (any angle, any pitch) lies within reach_plane of the axis and
// reach_axial along it; the hub sphere is included up to eps/2 beyond it
static void rotor_reach(const hl_lattice* lat, const hl_rotor_geometry* g, double* reach_plane, double* reach_axial) {
    const double h = g->spacing;
    const double R0 = g->origin[0], R1 = g->origin[0] + h * (g->gx - 1);
    const double T0 = g->origin[1], T1 = g->origin[1] + h * (g->gy - 1);
    const double A0 = g->origin[2], A1 = g->origin[2] + h * (g->gz - 1);
    const double rmax = std::fmax(std::fabs(R0), std::fabs(R1));
    const double tmax = std::fmax(std::fabs(T0), std::fabs(T1));
    const double amax = std::fmax(std::fabs(A0), std::fabs(A1));
    const double w = std::hypot(tmax, amax);     // the pitch rotation mixes T and A
    const double hubr = g->hub_radius > 0 ? g->hub_radius + 0.5 * lat->cfg.eps_h : 0.0;
    *reach_plane = std::fmax(g->n_blades > 0 ? std::hypot(rmax, w) : 0.0, hubr);
    *reach_axial = std::fmax(g->n_blades > 0 ? w : 0.0, hubr);
}

// halo planes a face needs when it cuts a rotor box: the wall-model sample
// (y_s along the normal, trilinear corners) and, at odd steps, the one more
// plane its corner velocities are gathered from
static int deep_halo_min(const hl_config& c) { return (int)std::ceil(c.wm_ysample) + 2; }

// The rotor's box of cells.  A slab's box lies in its own planes; where it
// reaches through a halo face of at least deep_halo_min planes it is cut
// there (clip[f]) and the slab beyond takes the rest.  Returns an error text
// or null.
static const char* rotor_box(const hl_lattice* lat, const hl_rotor_geometry* g, int lo[3], int nn[3],
                             bool clip[2]) {
    double rp, ra;
    rotor_reach(lat, g, &rp, &ra);
    const double reach_plane = rp + 2.0, reach_axial = ra + 2.0;
    const int dims[3] = {lat->cfg.nx, lat->cfg.ny, lat->cfg.nz};
    const int halo[2] = {lat->cfg.halo_lo, lat->cfg.halo_hi};
    clip[0] = clip[1] = false;
    for (int k = 0; k < 3; ++k) {
        const double r = (k == g->axis) ? reach_axial : reach_plane;
        int a = (int)std::floor(g->center[k] - r);
        int b = (int)std::ceil(g->center[k] + r);
        const bool open = lat->cfg.open_boundaries && k == lat->cfg.flow_axis;
        if (k == 2 && (halo[0] || halo[1])) {
            // owned planes halo_lo .. nz - 1 - halo_hi; a face without halo is open or periodic
            const int z0 = halo[0], z1 = dims[2] - 1 - halo[1];
            for (int f = 0; f < 2; ++f) {
                const bool beyond = f == 0 ? a < z0 : b > z1;
                if (!beyond) continue;
                if (!halo[f]) return "rotor box leaves the lattice or touches an open boundary";
                if (halo[f] < deep_halo_min(lat->cfg))
                    return "rotor box cut by a slab face with fewer halo planes than the wall-model sample needs";
                clip[f] = true;
                if (f == 0) a = z0;
                else b = z1;
            }
            const bool open_lo = open && !halo[0], open_hi = open && !halo[1];
            if ((open_lo && a < 4) || (open_hi && b > dims[2] - 5)) return "rotor box touches an open boundary";
            if (a > b) return "rotor box outside the slab's planes";
        } else {
            // 4 cells from an open face
            const int m = open ? 4 : 0;
            if (a < m || b > dims[k] - 1 - m) return "rotor box leaves the lattice or touches an open boundary";
        }
        lo[k] = a;
        nn[k] = b - a + 1;
    }
    return nullptr;
}

static bool valid_geometry(const hl_rotor_geometry* g) {
    if (!g) return false;
    if (g->axis < 0 || g->axis > 2 || g->n_blades < 0 || g->n_blades > MAXBLADES) return false;
    if (g->n_blades > 0 && (!g->sdf || g->gx < 2 || g->gy < 2 || g->gz < 2)) return false;
    if (!(g->spacing > 0.0) || !(g->hub_radius >= 0.0)) return false;
    if (g->n_blades == 0 && !(g->hub_radius > 0.0)) return false;
    return true;
}

hl_status hl_rotor_workspace_size(const hl_lattice* lat, const hl_rotor_geometry* geom, size_t* bytes) {
    if (!lat || !valid_geometry(geom) || !bytes) return HL_ERR_ARG;
    int lo[3], nn[3];
    bool clip[2];
    if (rotor_box(lat, geom, lo, nn, clip)) return HL_ERR_ARG;
    const long long box = (long long)nn[0] * nn[1] * nn[2];
    const long long ng = geom->n_blades > 0 ? (long long)geom->gx * geom->gy * geom->gz : 1;
    *bytes = rotor_layout(ng, box).total;
    return HL_OK;
}

hl_status hl_set_rotor(hl_lattice* lat, int* rotor_id, const hl_rotor_geometry* geom, double omega,
                       double pitch, void* d_workspace, size_t bytes) {
    if (!lat) return HL_ERR_ARG;
    if (!valid_geometry(geom) || !d_workspace || !std::isfinite(omega) || !std::isfinite(pitch))
        return fail(lat, HL_ERR_ARG, "hl_set_rotor: invalid geometry or arguments");
    if (reinterpret_cast<size_t>(d_workspace) % ALIGN) return fail(lat, HL_ERR_ARG, "workspace not aligned");
    if (lat->nrot >= MAXROT) return fail(lat, HL_ERR_ARG, "too many rotors");
    int lo[3], nn[3];
    bool clip[2];
    if (const char* why = rotor_box(lat, geom, lo, nn, clip)) return fail(lat, HL_ERR_ARG, why);
    for (int k = 0; k < lat->nrot; ++k) {
        const RotorDev& o = lat->rot[k].dev;
        bool overlap = true;
        for (int d = 0; d < 3; ++d)
            if (lo[d] + nn[d] <= o.lo[d] || o.lo[d] + o.n[d] <= lo[d]) overlap = false;
        if (overlap) return fail(lat, HL_ERR_ARG, "rotor boxes overlap");
    }
    const long long box = (long long)nn[0] * nn[1] * nn[2];
    const long long ng = geom->n_blades > 0 ? (long long)geom->gx * geom->gy * geom->gz : 1;
    const RotorLayout L = rotor_layout(ng, box);
    if (bytes < L.total) return fail(lat, HL_ERR_WORKSPACE, "rotor workspace too small");
    RotorHost& R = lat->rot[lat->nrot];
    std::memset(&R, 0, sizeof R);
    R.geom = *geom;
    R.geom.sdf = nullptr;
    R.omega = omega;
    R.pitch = pitch;
    R.pitch_sets = pitch;
    R.ws = static_cast<char*>(d_workspace);
    R.L = L;
    RotorDev& D = R.dev;
    for (int k = 0; k < 3; ++k) {
        D.lo[k] = lo[k];
        D.n[k] = nn[k];
        D.cf[k] = (float)geom->center[k];
        D.g[k] = k == 0 ? geom->gx : (k == 1 ? geom->gy : geom->gz);
        D.origin[k] = (float)geom->origin[k];
    }
    if (geom->n_blades == 0) D.g[0] = D.g[1] = D.g[2] = 2;
    // wall-model samples stay in the box, or cross a cut face into the halo
    // (one plane short of its end: odd steps gather a corner's populations
    // from its neighbours)
    R.clip[0] = clip[0];
    R.clip[1] = clip[1];
    D.zs_lo = clip[0] ? 1 : lo[2];
    D.zs_hi = clip[1] ? lat->cfg.nz - 1 : lo[2] + nn[2];
    D.box_cells = box;
    D.omega = (float)omega;
    D.axis = geom->axis;
    D.n_blades = geom->n_blades;
    D.hub = (float)geom->hub_radius;
    D.inv_h = (float)(1.0 / geom->spacing);
    D.h = (float)geom->spacing;
    {
        double rp, ra;
        rotor_reach(lat, geom, &rp, &ra);
        rp += 1.0;   // one cell of margin covers every binary32 rounding of the test
        ra += 1.0;
        D.reach_plane2 = (float)(rp * rp);
        D.reach_axial = (float)ra;
    }
    D.sdf = reinterpret_cast<const float*>(R.ws + L.sdf);
    D.d = reinterpret_cast<float*>(R.ws + L.d);
    D.flags = reinterpret_cast<uint8_t*>(R.ws + L.flags);
    D.wm = reinterpret_cast<float*>(R.ws + L.wm);
    D.utau = reinterpret_cast<double*>(R.ws + L.utau);
    D.active = reinterpret_cast<uint8_t*>(R.ws + L.active);
    // set 0 of the cell lists; make_args selects the set of the step's parity
    D.list = reinterpret_cast<int*>(R.ws + L.list[0]);
    D.wlist = reinterpret_cast<int*>(R.ws + L.wlist[0]);
    D.wphi = reinterpret_cast<float*>(R.ws + L.wphi[0]);
    D.wwhich = reinterpret_cast<signed char*>(R.ws + L.wwhich[0]);
    D.count = reinterpret_cast<int*>(R.ws + L.count);
    D.done = reinterpret_cast<unsigned*>(R.ws + L.done);
    D.partial = reinterpret_cast<double*>(R.ws + L.partial);
    D.acc = reinterpret_cast<double*>(R.ws + L.acc);
    D.drive = nullptr;
    HL_CUDA(lat, cudaMemsetAsync(R.ws, 0, L.total, lat->stream));
    if (geom->n_blades > 0)
        HL_CUDA(lat, cudaMemcpyAsync(R.ws + L.sdf, geom->sdf, sizeof(float) * ng, cudaMemcpyHostToDevice,
                                     lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    if (rotor_id) *rotor_id = lat->nrot;
    lat->nrot += 1;
    lat->clip_face[0] = lat->clip_face[0] || clip[0];
    lat->clip_face[1] = lat->clip_face[1] || clip[1];
    return HL_OK;
}

// records one event of kind k when profiling (start: even index, stop: odd)
static cudaError_t prof_mark(hl_lattice* lat, int k, cudaStream_t st) {
    if (!lat->prof_on) return cudaSuccess;
    std::vector<cudaEvent_t>& v = lat->prof_ev[k];
    if ((int)v.size() >= 2 * lat->prof_cap) return cudaSuccess;
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    v.push_back(e);
    return cudaEventRecord(e, st);
}

}  // extern "C"

// a rotor box cut by a halo face: the force reduction of a step waits for
// the halo exchange that follows it
static bool defers_force(const hl_lattice* lat) { return lat->clip_face[0] || lat->clip_face[1]; }

// the deferred force reduction (and driven-rotor update) of the last step,
// on the lattice stream
static hl_status flush_force(hl_lattice* lat) {
    if (!lat->force_pending) return HL_OK;
    lat->force_pending = false;
    const int Q = lat->cfg.q, S = lat->cfg.storage;
    HL_CUDA(lat, prof_mark(lat, 2, lat->stream));
    HL_CUDA(lat, launch_force(Q, S, lat->pending, lat->stream));
    HL_CUDA(lat, prof_mark(lat, 2, lat->stream));
    HL_CUDA(lat, launch_evolve(lat->pending, lat->stream));
    return HL_OK;
}

// one step on a single stream
static hl_status step_serial(hl_lattice* lat, const StepArgs& a0, bool with_force) {
    const int Q = lat->cfg.q, S = lat->cfg.storage;
    cudaStream_t st = lat->stream;
    StepArgs a = a0;
    a.part = 0;
    if (lat->nrot > 0) {
        HL_CUDA(lat, prof_mark(lat, 0, st));
        HL_CUDA(lat, launch_band(Q, S, a, st));
        HL_CUDA(lat, launch_band_strain(Q, S, a, st));
        HL_CUDA(lat, prof_mark(lat, 0, st));
        if (lat->cfg.wall_model) {
            HL_CUDA(lat, prof_mark(lat, 4, st));
            HL_CUDA(lat, launch_wall(Q, S, a, st));
            HL_CUDA(lat, prof_mark(lat, 4, st));
        }
    }
    HL_CUDA(lat, prof_mark(lat, 1, st));
    HL_CUDA(lat, launch_collide(Q, S, a, st));
    HL_CUDA(lat, prof_mark(lat, 1, st));
    if (lat->nrot > 0) {
        if (with_force && !defers_force(lat)) {
            HL_CUDA(lat, prof_mark(lat, 2, st));
            HL_CUDA(lat, launch_force(Q, S, a, st));
            HL_CUDA(lat, prof_mark(lat, 2, st));
            HL_CUDA(lat, launch_evolve(a, st));
        } else if (!with_force) {
            for (int k = 0; k < lat->nrot; ++k)
                HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.count, 0, COUNT_BYTES, st));
        }
    }
    return HL_OK;
}

// One step on two streams.  The AA pattern gives every memory location to
// exactly one cell's thread, and the wall model and force only read cells
// deep inside a rotor box, so within a step the bulk launch (cells outside
// every box, lattice stream) and the box chain (embedding, wall model, box
// collision, force; aux stream) touch disjoint memory.  Across steps:
// box(t) waits for bulk(t-1), bulk(t) waits for box(t-1).
static hl_status step_overlap(hl_lattice* lat, const StepArgs& a0, bool with_force) {
    const int Q = lat->cfg.q, S = lat->cfg.storage;
    const int p = (int)(a0.t & 1), q = p ^ 1;
    cudaStream_t us = lat->stream, ax = lat->aux;
    StepArgs a = a0;
    // lattice stream: cells outside every rotor box
    HL_CUDA(lat, cudaStreamWaitEvent(us, lat->ev_box[q], 0));
    a.part = 1;
    HL_CUDA(lat, prof_mark(lat, 1, us));
    HL_CUDA(lat, launch_collide(Q, S, a, us));
    HL_CUDA(lat, prof_mark(lat, 1, us));
    HL_CUDA(lat, cudaEventRecord(lat->ev_bulk[p], us));
    // aux stream: embedding, wall model, box collision; the force reduction
    // and the driven-rotor update follow on the third stream.  A driven
    // rotor's frames come from the previous step's update.
    bool driven = false;
    for (int k = 0; k < lat->nrot; ++k) driven = driven || lat->rot[k].driven;
    if (driven) HL_CUDA(lat, cudaStreamWaitEvent(ax, lat->ev_force[q], 0));
    HL_CUDA(lat, prof_mark(lat, 0, ax));
    HL_CUDA(lat, launch_band(Q, S, a, ax));
    HL_CUDA(lat, launch_band_strain(Q, S, a, ax));
    HL_CUDA(lat, prof_mark(lat, 0, ax));
    if (lat->cfg.wall_model) {
        HL_CUDA(lat, prof_mark(lat, 4, ax));
        HL_CUDA(lat, launch_wall(Q, S, a, ax));
        HL_CUDA(lat, prof_mark(lat, 4, ax));
    }
    // the box collision overwrites the populations the previous step's force
    // reduction reads (and the bulk launch's boundary slots)
    HL_CUDA(lat, cudaStreamWaitEvent(ax, lat->ev_bulk[q], 0));
    HL_CUDA(lat, cudaStreamWaitEvent(ax, lat->ev_force[q], 0));
    a.part = 2;
    for (int k = 0; k < lat->nrot; ++k) {
        a.part_rotor = k;
        HL_CUDA(lat, prof_mark(lat, 5, ax));
        HL_CUDA(lat, launch_collide(Q, S, a, ax));
        HL_CUDA(lat, prof_mark(lat, 5, ax));
    }
    HL_CUDA(lat, cudaEventRecord(lat->ev_box[p], ax));
    a.part = 0;
    if (with_force && defers_force(lat)) {
        // taken after the halo exchange (flush_force)
    } else if (with_force) {
        cudaStream_t fs = lat->fst;
        HL_CUDA(lat, cudaStreamWaitEvent(fs, lat->ev_box[p], 0));
        HL_CUDA(lat, prof_mark(lat, 2, fs));
        HL_CUDA(lat, launch_force(Q, S, a, fs));
        HL_CUDA(lat, prof_mark(lat, 2, fs));
        HL_CUDA(lat, launch_evolve(a, fs));
        HL_CUDA(lat, cudaEventRecord(lat->ev_force[p], fs));
    } else {
        for (int k = 0; k < lat->nrot; ++k)
            HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.count, 0, COUNT_BYTES, ax));
    }
    return HL_OK;
}

namespace hl {
namespace host {

hl_status issue_step(hl_lattice* lat, const StepArgs& a, bool with_force) {
    const bool two = lat->have_aux && lat->nrot > 0;
    return two ? step_overlap(lat, a, with_force) : step_serial(lat, a, with_force);
}

}  // namespace host
}  // namespace hl

extern "C" {

hl_status hl_step_async(hl_lattice* lat, int n) {
    if (!lat || n < 0) return HL_ERR_ARG;
    if (lat->cfg.halo_lo || lat->cfg.halo_hi) {
        // a slab steps once per call, after the halo exchange of its parity
        if (n > 1) return fail(lat, HL_ERR_ARG, "a slab (halo planes) advances one step per call");
        for (int f = 0; f < 2 && n > 0; ++f) {
            if ((f == 0 ? lat->cfg.halo_lo : lat->cfg.halo_hi) && lat->t > 0 && lat->halo_t[f] != lat->t)
                return fail(lat, HL_ERR_STATE, "halo face not imported at the current time step");
            // a face that cuts a rotor box: its deep halo holds the neighbour's state
            // of this step, also at t = 0 (the wall model samples through it)
            if (lat->clip_face[f] && lat->deep_t[f] != lat->t)
                return fail(lat, HL_ERR_STATE, "deep halo of a face that cuts a rotor box not imported at this step");
        }
        if (n > 0) {
            hl_status fst_ = flush_force(lat);
            if (fst_ != HL_OK) return fst_;
        }
    }
    const bool two = lat->have_aux && lat->nrot > 0;
    if (two && n > 0) {
        // everything issued on the lattice stream so far precedes the aux work
        HL_CUDA(lat, cudaEventRecord(lat->ev_fork, lat->stream));
        HL_CUDA(lat, cudaStreamWaitEvent(lat->aux, lat->ev_fork, 0));
    }
    for (int s = 0; s < n; ++s) {
        const StepArgs a = make_args(lat);
        hl_status st = issue_step(lat, a, true);
        if (st != HL_OK) return st;
        if (defers_force(lat) && lat->nrot > 0) {
            lat->pending = a;
            lat->pending.part = 0;
            lat->force_pending = true;
        }
        const long long t_done = lat->t;
        lat->t += 1;
        lat->n_avg += 1;
        const int K = lat->cfg.mass_check_every;
        if (K > 0 && lat->t % K == 0) {
            const int p = (int)(t_done & 1);
            if (two) HL_CUDA(lat, cudaStreamWaitEvent(lat->stream, lat->ev_box[p], 0));
            HL_CUDA(lat, prof_mark(lat, 3, lat->stream));
            st = compute_mass(lat, lat->cfg.mass_tol, nullptr);
            if (st != HL_OK) return st;
            HL_CUDA(lat, prof_mark(lat, 3, lat->stream));
            // the next box collision must also wait for the mass total
            if (two) HL_CUDA(lat, cudaEventRecord(lat->ev_bulk[p], lat->stream));
        }
    }
    if (two && n > 0) {
        // the lattice stream sees the completed aux and force-stream work
        HL_CUDA(lat, cudaEventRecord(lat->ev_join, lat->aux));
        HL_CUDA(lat, cudaStreamWaitEvent(lat->stream, lat->ev_join, 0));
        HL_CUDA(lat, cudaEventRecord(lat->ev_join_f, lat->fst));
        HL_CUDA(lat, cudaStreamWaitEvent(lat->stream, lat->ev_join_f, 0));
    }
    return HL_OK;
}

hl_status hl_profile_begin(hl_lattice* lat, int capacity) {
    if (!lat || capacity < 0) return HL_ERR_ARG;
    for (auto& v : lat->prof_ev) {
        for (cudaEvent_t e : v) cudaEventDestroy(e);
        v.clear();
    }
    lat->prof_cap = capacity;
    lat->prof_on = true;
    return HL_OK;
}

hl_status hl_profile_end(hl_lattice* lat, double* ms, long long* launches) {
    if (!lat) return HL_ERR_ARG;
    lat->prof_on = false;
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    hl_status st = HL_OK;
    for (int k = 0; k < 6; ++k) {
        std::vector<cudaEvent_t>& v = lat->prof_ev[k];
        double sum = 0.0;
        const size_t pairs = v.size() / 2;
        for (size_t i = 0; i < pairs; ++i) {
            float t = 0.f;
            cudaError_t e = cudaEventElapsedTime(&t, v[2 * i], v[2 * i + 1]);
            if (e != cudaSuccess && st == HL_OK) st = cuda_fail(lat, e, "cudaEventElapsedTime");
            sum += t;
        }
        if (ms) ms[k] = sum;
        if (launches) launches[k] = (long long)pairs;
        for (cudaEvent_t e : v) cudaEventDestroy(e);
        v.clear();
    }
    return st;
}

hl_status hl_check(hl_lattice* lat) {
    if (!lat) return HL_ERR_ARG;
    return read_error_word(lat);
}

hl_status hl_step(hl_lattice* lat, int n) {
    hl_status st = hl_step_async(lat, n);
    if (st != HL_OK) return st;
    return read_error_word(lat);
}

static hl_status read_acc(hl_lattice* lat, std::vector<double>& acc) {
    if (hl_status st = flush_force(lat); st != HL_OK) return st;
    acc.assign(12 * (size_t)lat->nrot, 0.0);
    for (int k = 0; k < lat->nrot; ++k)
        HL_CUDA(lat, cudaMemcpyAsync(acc.data() + 12 * k, lat->rot[k].dev.acc, 12 * sizeof(double),
                                     cudaMemcpyDeviceToHost, lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    return HL_OK;
}

hl_status hl_loads_async(hl_lattice* lat, double* h_loads) {
    if (!lat || !h_loads) return HL_ERR_ARG;
    if (hl_status st = flush_force(lat); st != HL_OK) return st;
    for (int k = 0; k < lat->nrot; ++k)
        HL_CUDA(lat, cudaMemcpyAsync(h_loads + 6 * k, lat->rot[k].dev.acc, 6 * sizeof(double),
                                     cudaMemcpyDeviceToHost, lat->stream));
    return HL_OK;
}

hl_status hl_forces(hl_lattice* lat, double* F, double* F_avg, int reset_avg) {
    if (!lat) return HL_ERR_ARG;
    std::vector<double> acc;
    hl_status st = read_acc(lat, acc);
    if (st != HL_OK) return st;
    const double na = lat->n_avg > 0 ? (double)lat->n_avg : 1.0;
    for (int k = 0; k < lat->nrot; ++k)
        for (int a = 0; a < 3; ++a) {
            if (F) F[3 * k + a] = acc[12 * k + a];
            if (F_avg) F_avg[3 * k + a] = lat->n_avg > 0 ? acc[12 * k + 6 + a] / na : 0.0;
        }
    if (reset_avg) {
        for (int k = 0; k < lat->nrot; ++k)
            HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.acc + 6, 0, 6 * sizeof(double), lat->stream));
        HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
        lat->n_avg = 0;
    }
    return HL_OK;
}

hl_status hl_moments(hl_lattice* lat, double* M, double* M_avg) {
    if (!lat) return HL_ERR_ARG;
    std::vector<double> acc;
    hl_status st = read_acc(lat, acc);
    if (st != HL_OK) return st;
    const double na = lat->n_avg > 0 ? (double)lat->n_avg : 1.0;
    for (int k = 0; k < lat->nrot; ++k)
        for (int a = 0; a < 3; ++a) {
            if (M) M[3 * k + a] = acc[12 * k + 3 + a];
            if (M_avg) M_avg[3 * k + a] = lat->n_avg > 0 ? acc[12 * k + 9 + a] / na : 0.0;
        }
    return HL_OK;
}

hl_status hl_fields(hl_lattice* lat, float* d_rho, float* d_u) {
    if (!lat || !d_rho || !d_u) return HL_ERR_ARG;
    const StepArgs a = make_args(lat);
    HL_CUDA(lat, launch_fields(lat->cfg.q, lat->cfg.storage, a, d_rho, d_u, lat->stream));
    return HL_OK;
}

hl_status hl_init_fields(hl_lattice* lat, const float* d_rho, const float* d_u) {
    if (!lat) return HL_ERR_ARG;
    const float u0[3] = {0.f, 0.f, 0.f};
    HL_CUDA(lat, launch_init(lat->cfg.q, lat->cfg.storage, make_args(lat), d_rho, d_u, 0.0f, u0,
                             lat->stream));
    lat->t = 0;
    lat->n_avg = 0;
    HL_CUDA(lat, cudaMemsetAsync(lat->err, 0, sizeof(unsigned), lat->stream));
    for (int k = 0; k < lat->nrot; ++k)
        HL_CUDA(lat, cudaMemsetAsync(lat->rot[k].dev.acc, 0, 12 * sizeof(double), lat->stream));
    double m0 = 0.0;
    hl_status st = compute_mass(lat, -1.0, &m0);
    if (st != HL_OK) return st;
    lat->mass_ref = m0;
    return HL_OK;
}

// ---- slabs: halo exchange (AA pattern, decomposition along z) ----
// The message of a face is one plane of the slots whose velocity crosses
// that face, chosen by the step parity (see include/hlbm.h); with D_lo /
// D_hi halo planes the plane next to the lower face is D_lo - 1 and the
// lower boundary plane D_lo (upper: nz - D_hi and nz - D_hi - 1):
//   export  face 0: t odd boundary plane (c_z = +1),  t even halo plane (c_z = -1)
//           face 1: t odd boundary plane (c_z = -1),  t even halo plane (c_z = +1)
//   import  face 0: t odd halo plane (c_z = -1),      t even boundary plane (c_z = +1)
//           face 1: t odd halo plane (c_z = +1),      t even boundary plane (c_z = -1)
static int halo_slot_list(int q, int sign, int* out) {
    std::vector<int> c(3 * q);
    std::vector<double> w(q);
    hl_velocity_set(q, c.data(), w.data());
    int n = 0;
    for (int s = 0; s < q; ++s)
        if (c[3 * s + 2] == sign) out[n++] = s;
    return n;
}

static hl_status halo_copy(hl_lattice* lat, int face, void* buf, bool import_) {
    if (!lat || face < 0 || face > 1 || !buf) return HL_ERR_ARG;
    if (!(face == 0 ? lat->cfg.halo_lo : lat->cfg.halo_hi))
        return fail(lat, HL_ERR_ARG, "hl_halo_export/import: the face is not a halo face");
    // the halo plane next to the face and the slab's own boundary plane
    const int nz = lat->cfg.nz;
    const int h_lo = lat->cfg.halo_lo - 1, b_lo = lat->cfg.halo_lo;
    const int h_hi = nz - lat->cfg.halo_hi, b_hi = nz - lat->cfg.halo_hi - 1;
    const bool odd = (lat->t & 1) != 0;
    int plane, sign;
    if (!import_) {
        if (face == 0) { plane = odd ? b_lo : h_lo; sign = odd ? +1 : -1; }
        else { plane = odd ? b_hi : h_hi; sign = odd ? -1 : +1; }
    } else {
        if (face == 0) { plane = odd ? h_lo : b_lo; sign = odd ? -1 : +1; }
        else { plane = odd ? h_hi : b_hi; sign = odd ? +1 : -1; }
    }
    HaloArgs h;
    std::memset(&h, 0, sizeof h);
    h.f = lat->f;
    h.N = lat->N;
    h.nxy = lat->cfg.nx * lat->cfg.ny;
    h.plane = plane;
    h.nplanes = 1;
    h.nslot = halo_slot_list(lat->cfg.q, sign, h.slots);
    h.buf = buf;
    h.import_ = import_ ? 1 : 0;
    HL_CUDA(lat, launch_halo(lat->cfg.storage, h, lat->stream));
    if (import_) lat->halo_t[face] = lat->t;
    return HL_OK;
}

hl_status hl_halo_size(const hl_lattice* lat, size_t* bytes) {
    if (!lat || !bytes || !(lat->cfg.halo_lo || lat->cfg.halo_hi)) return HL_ERR_ARG;
    const int nslot = lat->cfg.q == 19 ? 5 : 9;
    *bytes = (size_t)nslot * lat->cfg.nx * lat->cfg.ny * store_bytes(lat->cfg.storage);
    return HL_OK;
}

hl_status hl_halo_export(hl_lattice* lat, int face, void* d_buf) { return halo_copy(lat, face, d_buf, false); }

hl_status hl_halo_import(hl_lattice* lat, int face, const void* d_buf) {
    return halo_copy(lat, face, const_cast<void*>(d_buf), true);
}

// Deep halo: every slot of the D planes next to a face.  Export: the slab's
// own D planes next to the face; import: its D halo planes beyond it.  Runs
// after the one-plane exchange of the same step, so the neighbour's planes
// are complete.
static hl_status deep_copy(hl_lattice* lat, int face, void* buf, bool import_) {
    if (!lat || face < 0 || face > 1 || !buf) return HL_ERR_ARG;
    const int D = face == 0 ? lat->cfg.halo_lo : lat->cfg.halo_hi;
    if (D < 1) return fail(lat, HL_ERR_ARG, "hl_halo_deep_export/import: the face is not a halo face");
    const int nz = lat->cfg.nz;
    HaloArgs h;
    std::memset(&h, 0, sizeof h);
    h.f = lat->f;
    h.N = lat->N;
    h.nxy = lat->cfg.nx * lat->cfg.ny;
    if (face == 0) h.plane = import_ ? 0 : D;
    else h.plane = import_ ? nz - D : nz - 2 * D;
    h.nplanes = D;
    h.nslot = lat->cfg.q;
    for (int s = 0; s < lat->cfg.q; ++s) h.slots[s] = s;
    h.buf = buf;
    h.import_ = import_ ? 1 : 0;
    HL_CUDA(lat, launch_halo(lat->cfg.storage, h, lat->stream));
    if (import_) lat->deep_t[face] = lat->t;
    return HL_OK;
}

hl_status hl_halo_deep_size(const hl_lattice* lat, int face, size_t* bytes) {
    if (!lat || !bytes || face < 0 || face > 1) return HL_ERR_ARG;
    const int D = face == 0 ? lat->cfg.halo_lo : lat->cfg.halo_hi;
    if (D < 1) return HL_ERR_ARG;
    *bytes = (size_t)D * lat->cfg.q * lat->cfg.nx * lat->cfg.ny * store_bytes(lat->cfg.storage);
    return HL_OK;
}

hl_status hl_halo_deep_export(hl_lattice* lat, int face, void* d_buf) { return deep_copy(lat, face, d_buf, false); }

hl_status hl_halo_deep_import(hl_lattice* lat, int face, const void* d_buf) {
    return deep_copy(lat, face, const_cast<void*>(d_buf), true);
}

hl_status hl_mass(hl_lattice* lat, double* mass) {
    if (!lat || !mass) return HL_ERR_ARG;
    return compute_mass(lat, -1.0, mass);
}

hl_status hl_get_time(const hl_lattice* lat, long long* t) {
    if (!lat || !t) return HL_ERR_ARG;
    *t = lat->t;
    return HL_OK;
}

// snapshot layout: header | populations | outlet planes | per rotor: utau, active, acc
struct StateHeader {
    long long magic, t, n_avg, N;
    int q, storage, nrot, pad;
    double mass_ref;
};
static const long long STATE_MAGIC = 0x484c424d53544154LL;

static size_t state_bytes(const hl_lattice* lat) {
    size_t o = align_up(sizeof(StateHeader));
    o = align_up(o + (size_t)lat->cfg.q * lat->N * store_bytes(lat->cfg.storage));
    o = align_up(o + 2 * sizeof(float) * 3 * plane_cells(lat->cfg));
    for (int k = 0; k < lat->nrot; ++k) {
        const long long b = lat->rot[k].dev.box_cells;
        o = align_up(o + sizeof(double) * b);
        o = align_up(o + b);
        o = align_up(o + sizeof(double) * 12);
        o = align_up(o + sizeof(DriveDev));
    }
    return o;
}

hl_status hl_state_size(const hl_lattice* lat, size_t* bytes) {
    if (!lat || !bytes) return HL_ERR_ARG;
    *bytes = state_bytes(lat);
    return HL_OK;
}

static hl_status state_copy(hl_lattice* lat, char* buf, bool save) {
    const cudaMemcpyKind kd = cudaMemcpyDeviceToDevice;
    size_t o = align_up(sizeof(StateHeader));
    auto cp = [&](void* dev, size_t n) -> cudaError_t {
        cudaError_t e = save ? cudaMemcpyAsync(buf + o, dev, n, kd, lat->stream)
                             : cudaMemcpyAsync(dev, buf + o, n, kd, lat->stream);
        o = align_up(o + n);
        return e;
    };
    HL_CUDA(lat, cp(lat->f, (size_t)lat->cfg.q * lat->N * store_bytes(lat->cfg.storage)));
    const size_t pb = sizeof(float) * 3 * plane_cells(lat->cfg);
    // both outlet planes, in the order (previous, current) of the saved time
    {
        float* first = lat->uplane[(lat->t + 1) & 1];
        float* second = lat->uplane[lat->t & 1];
        cudaError_t e = save ? cudaMemcpyAsync(buf + o, first, pb, kd, lat->stream)
                             : cudaMemcpyAsync(first, buf + o, pb, kd, lat->stream);
        HL_CUDA(lat, e);
        e = save ? cudaMemcpyAsync(buf + o + pb, second, pb, kd, lat->stream)
                 : cudaMemcpyAsync(second, buf + o + pb, pb, kd, lat->stream);
        HL_CUDA(lat, e);
        o = align_up(o + 2 * pb);
    }
    for (int k = 0; k < lat->nrot; ++k) {
        RotorDev& D = lat->rot[k].dev;
        HL_CUDA(lat, cp(D.utau, sizeof(double) * D.box_cells));
        HL_CUDA(lat, cp(D.active, (size_t)D.box_cells));
        HL_CUDA(lat, cp(D.acc, sizeof(double) * 12));
        HL_CUDA(lat, cp(lat->rot[k].ws + lat->rot[k].L.drive, sizeof(DriveDev)));
    }
    return HL_OK;
}

hl_status hl_save_state(hl_lattice* lat, void* d_buf, size_t bytes) {
    if (!lat || !d_buf) return HL_ERR_ARG;
    if (bytes < state_bytes(lat)) return fail(lat, HL_ERR_WORKSPACE, "state buffer too small");
    if (hl_status fs = flush_force(lat); fs != HL_OK) return fs;
    StateHeader h{STATE_MAGIC, lat->t, lat->n_avg, lat->N, lat->cfg.q, lat->cfg.storage, lat->nrot, 0,
                  lat->mass_ref};
    HL_CUDA(lat, cudaMemcpyAsync(d_buf, &h, sizeof h, cudaMemcpyHostToDevice, lat->stream));
    hl_status st = state_copy(lat, static_cast<char*>(d_buf), true);
    if (st != HL_OK) return st;
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    return HL_OK;
}

hl_status hl_load_state(hl_lattice* lat, const void* d_buf, size_t bytes) {
    if (!lat || !d_buf) return HL_ERR_ARG;
    if (bytes < state_bytes(lat)) return fail(lat, HL_ERR_WORKSPACE, "state buffer too small");
    StateHeader h;
    HL_CUDA(lat, cudaMemcpyAsync(&h, d_buf, sizeof h, cudaMemcpyDeviceToHost, lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    if (h.magic != STATE_MAGIC || h.N != lat->N || h.q != lat->cfg.q || h.storage != lat->cfg.storage ||
        h.nrot != lat->nrot)
        return fail(lat, HL_ERR_STATE, "state snapshot does not match this lattice");
    lat->t = h.t;
    lat->n_avg = h.n_avg;
    lat->mass_ref = h.mass_ref;
    lat->halo_t[0] = lat->halo_t[1] = -1;   // a slab exchanges again before its next step
    lat->deep_t[0] = lat->deep_t[1] = -1;
    lat->force_pending = false;             // the snapshot's loads are complete
    hl_status st = state_copy(lat, const_cast<char*>(static_cast<const char*>(d_buf)), false);
    if (st != HL_OK) return st;
    HL_CUDA(lat, cudaMemsetAsync(lat->err, 0, sizeof(unsigned), lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    return HL_OK;
}

hl_status hl_set_drive(hl_lattice* lat, int rotor, double inertia, double k_gen, double q_gen0) {
    if (!lat || rotor < 0 || rotor >= lat->nrot) return HL_ERR_ARG;
    if (!(inertia > 0.0) || !std::isfinite(inertia) || !std::isfinite(k_gen) || !std::isfinite(q_gen0))
        return fail(lat, HL_ERR_ARG, "hl_set_drive: inertia must be positive and finite");
    RotorHost& R = lat->rot[rotor];
    if (R.clip[0] || R.clip[1])
        return fail(lat, HL_ERR_STATE, "hl_set_drive: the rotor's box is cut by a slab face (its torque is split)");
    DriveDev h;
    std::memset(&h, 0, sizeof h);
    double th, om;
    if (R.driven) {
        HL_CUDA(lat, cudaMemcpyAsync(&h, R.ws + R.L.drive, sizeof h, cudaMemcpyDeviceToHost, lat->stream));
        HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
        th = h.theta;
        om = h.omega;
    } else {
        th = R.geom.phase0 + R.omega * (double)lat->t;
        om = R.omega;
    }
    h.theta = th;
    h.omega = om;
    h.inertia = inertia;
    h.k_gen = k_gen;
    h.q_gen0 = q_gen0;
    for (int b = 0; b < R.geom.n_blades; ++b) {
        const double ang = th + 2.0 * M_PI * (double)b / (double)R.geom.n_blades;
        h.ck[b] = (float)std::cos(ang);
        h.sk[b] = (float)std::sin(ang);
    }
    h.omegaf = (float)om;
    HL_CUDA(lat, cudaMemcpyAsync(R.ws + R.L.drive, &h, sizeof h, cudaMemcpyHostToDevice, lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    R.driven = true;
    R.dev.drive = reinterpret_cast<DriveDev*>(R.ws + R.L.drive);
    return HL_OK;
}

hl_status hl_drive_state(hl_lattice* lat, int rotor, double* theta, double* omega) {
    if (!lat || rotor < 0 || rotor >= lat->nrot || !theta || !omega) return HL_ERR_ARG;
    RotorHost& R = lat->rot[rotor];
    if (!R.driven) {
        *theta = R.geom.phase0 + R.omega * (double)lat->t;
        *omega = R.omega;
        return HL_OK;
    }
    DriveDev h;
    HL_CUDA(lat, cudaMemcpyAsync(&h, R.ws + R.L.drive, sizeof h, cudaMemcpyDeviceToHost, lat->stream));
    HL_CUDA(lat, cudaStreamSynchronize(lat->stream));
    *theta = h.theta;
    *omega = h.omega;
    return HL_OK;
}

hl_status hl_rotor_box(const hl_lattice* lat, int rotor, int* lo, int* n) {
    if (!lat || rotor < 0 || rotor >= lat->nrot || !lo || !n) return HL_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
        lo[k] = lat->rot[rotor].dev.lo[k];
        n[k] = lat->rot[rotor].dev.n[k];
    }
    return HL_OK;
}

hl_status hl_rotor_band(hl_lattice* lat, int rotor, float* d_d, unsigned char* d_flags, float* d_wm,
                        double* d_utau) {
    if (!lat || rotor < 0 || rotor >= lat->nrot) return HL_ERR_ARG;
    const RotorDev& D = lat->rot[rotor].dev;
    const size_t b = (size_t)D.box_cells;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (d_d) HL_CUDA(lat, cudaMemcpyAsync(d_d, D.d, sizeof(float) * b, k, lat->stream));
    if (d_flags) HL_CUDA(lat, cudaMemcpyAsync(d_flags, D.flags, b, k, lat->stream));
    if (d_wm) HL_CUDA(lat, cudaMemcpyAsync(d_wm, D.wm, sizeof(float) * 9 * b, k, lat->stream));
    if (d_utau) HL_CUDA(lat, cudaMemcpyAsync(d_utau, D.utau, sizeof(double) * b, k, lat->stream));
    return HL_OK;
}

hl_status hl_velocity_set(int q, int* c, double* w) {
    if ((q != 19 && q != 27) || !c) return HL_ERR_ARG;
    const int P = (q - 1) / 2;
    for (int s = 0; s < q; ++s)
        for (int a = 0; a < 3; ++a) {
            int v = 0;
            if (s >= 1) {
                const int p = s <= P ? s - 1 : s - 1 - P;
                v = cpos(q, p, a);
                if (s > P) v = -v;
            }
            c[3 * s + a] = v;
        }
    // exact rational weights by shell |c|^2
    if (w)
        for (int s = 0; s < q; ++s) {
            const int sh = c[3 * s] * c[3 * s] + c[3 * s + 1] * c[3 * s + 1] + c[3 * s + 2] * c[3 * s + 2];
            if (q == 19) w[s] = sh == 0 ? 1.0 / 3.0 : (sh == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
            else w[s] = sh == 0 ? 8.0 / 27.0 : (sh == 1 ? 2.0 / 27.0 : (sh == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
        }
    return HL_OK;
}

hl_status hl_debug_collide(int q, int n, const float* d_g_in, const float* d_d, const float* d_uB,
                           const float* d_sigma, const float* d_S, double tau_mo, double c_smag,
                           float* d_g_out, void* stream) {
    if ((q != 19 && q != 27) || n < 0 || (n > 0 && (!d_g_in || !d_g_out))) return HL_ERR_ARG;
    const bool band = d_d || d_uB || d_sigma || d_S;
    if (band && !(d_d && d_uB && d_sigma && d_S)) return HL_ERR_ARG;
    const float K = (float)(18.0 * std::sqrt(2.0) * c_smag * c_smag);
    cudaError_t e = launch_debug_collide(q, n, d_g_in, d_d, d_uB, d_sigma, d_S, (float)tau_mo, K, d_g_out,
                                         static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HL_OK : HL_ERR_CUDA;
}

const char* hl_last_error(const hl_lattice* lat) { return lat ? lat->msg : "null handle"; }

void hl_destroy(hl_lattice* lat) {
    if (!lat) return;
    for (auto& v : lat->prof_ev)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    if (lat->aux) cudaStreamSynchronize(lat->aux);
    if (lat->fst) cudaStreamSynchronize(lat->fst);
    for (int k = 0; k < 2; ++k) {
        if (lat->ev_bulk[k]) cudaEventDestroy(lat->ev_bulk[k]);
        if (lat->ev_box[k]) cudaEventDestroy(lat->ev_box[k]);
        if (lat->ev_force[k]) cudaEventDestroy(lat->ev_force[k]);
    }
    if (lat->ev_fork) cudaEventDestroy(lat->ev_fork);
    if (lat->ev_join) cudaEventDestroy(lat->ev_join);
    if (lat->ev_join_f) cudaEventDestroy(lat->ev_join_f);
    if (lat->aux) cudaStreamDestroy(lat->aux);
    if (lat->fst) cudaStreamDestroy(lat->fst);
    delete lat;
}

}  // extern "C"
