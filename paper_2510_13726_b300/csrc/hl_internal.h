// Launch-side interface between the C ABI (hl_api.cu) and the kernels
// (hl_kernels.cu).  Not part of the public header.
#pragma once

#include <cuda_runtime.h>

#include "hl_device.cuh"

namespace hl {

constexpr int FORCE_BLOCKS = 64;     // blocks per rotor in the force reduction (few: they start beside the bulk launch)
constexpr int WALL_BLOCKS = 148;     // blocks per rotor in the wall model
constexpr int WALL_THREADS = 128;    // four warps per block
// the wall-model kernels take four lanes per wall cell: up to 37,888 wall
// cells per rotor in one pass (blocks whose lanes find no entry exit at once)
constexpr int WALL_GROUP_BLOCKS = 148 * 8;
// rotor boxes up to this many cells take four lanes per wall cell in the
// forward wall model (the 128x128x256 rotor's box: 0.26M cells; rotor256's: 1.3M)
constexpr long long WALL_SMALL_BOX = 1LL << 20;

// Cell lists (force cells, wall cells): consecutive entries (neighbouring
// cells) go to consecutive threads, so each warp's gathers share cache lines
// and each warp carries a full set of lanes through the FP64 wall-function
// solve, whose pipe bounds the wall kernel (spreading the entries one per
// warp lane across all SMs left most lanes idle and ran 3.4x slower).
__device__ __forceinline__ int list_first(void) { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int list_stride(void) { return gridDim.x * blockDim.x; }
constexpr int MASS_BLOCKS = 592;     // 4 x 148 SMs
constexpr int BAND_THREADS = 128;

// device error word; ERR_GEOMETRY: a wall cell's velocity sample reached
// outside its rotor box (the blade grid needs more padding around the blade)
enum ErrBits : unsigned { ERR_NONFINITE = 1u, ERR_MASS = 2u, ERR_GEOMETRY = 4u };

struct StepArgs {
    void* f;                 // populations [Q][N], storage type
    void* slot[27];          // base of slot s of the pre-collision state (read)
    void* wslot[27];         // base of slot s of the post-collision state (written; = slot in place)
    // odd-step bases shifted by the slot's velocity: f_s(x) is read at
    // rshift[s] + x (slot sbar of x - c_s) and f*_s(x) written at wshift[s] + x
    // (slot s of x + c_s); valid for cells whose neighbours need no periodic wrap
    const void* rshift[27];
    void* wshift[27];
    long long N;
    int n[3];
    int nxy, nplane;         // nx * ny; cells of an inlet/outlet plane
    int phase;               // t & 1: AA layout of the pre-collision state
    long long t;
    int flow_axis, open;
    int open_lo, open_hi;    // the open faces of the flow axis that this lattice has (a slab may lack one)
    int z0, z1;              // planes the bulk launches collide: z0 <= z < z1 (halo planes excluded)
    int zoff;                // global z of local plane 0 (synthetic inflow)
    float tau_mo, Ksmag;     // Ksmag = 18 sqrt(2) C_S^2
    float u_in, inflow_shift;   // inflow_shift = u_in * t
    float eps_half, inv_eps;
    int transition, wall_model;
    float wmYs;
    double wmE, wmK, wmTol, nu;      // wall-function constants (rounded to FP32 by make_wallfn)
    int wmMaxit;
    float sigma_band;        // hybridisation factor of the force cells off the wall set
    const float* modes;      // [n_modes][9]
    int n_modes;
    const float* uplane_prev;  // [3][plane]
    float* uplane_cur;
    unsigned* err;
    int part;                // collide cells: 0 all, 1 outside every rotor box, 2 the box of part_rotor
    int part_rotor;
    const float* d0;         // [N] static porosity multiplier, null = 1
    const float* inflow_plane;  // [3][plane] caller's inflow velocity, null = the synthetic modes
    int tangent;             // band kernel also writes d(porosity)/d(pitch) (reverse sweep)
    int pairs;               // bulk launches take x-adjacent cell pairs (nx even, slot bases 2-element aligned)
    int layout;              // 0 AA pattern, 1 esoteric twist (an AA lattice with x halves has 0 here)
    int xpair;               // AA with x halves: cell x of a row stored at 2x (x < hx), 2(x - hx) + 1 (x >= hx)
    int hx;                  // nx / 2
    int nrot;
    RotorDev rot[MAXROT];
};

struct MassArgs {
    const void* f;
    long long count;         // Q * N stored values
    long long N;             // cells per slot
    int nxy;                 // cells per z plane
    int halo_lo, halo_hi;    // halo planes (z < halo_lo, z >= nz - halo_hi) excluded from the total
    double shift_mass;       // N * sum_i w_i (the storage shift)
    double ref, tol;         // reference mass and allowed relative drift (tol < 0: no check)
    double* partial;         // [MASS_BLOCKS]
    unsigned* done;
    double* out;
    unsigned* err;
};

// launchers: return the launch error of the last kernel
cudaError_t launch_band(int Q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_collide(int Q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_wall(int Q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_band_strain(int Q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_force(int Q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_mass(int Q, int storage, const MassArgs& m, cudaStream_t s);
cudaError_t launch_evolve(const StepArgs& a, cudaStream_t s);
cudaError_t launch_init(int Q, int storage, const StepArgs& a, const float* rho, const float* u, float drho0,
                        const float u0[3], cudaStream_t s);
cudaError_t launch_fields(int Q, int storage, const StepArgs& a, float* rho, float* u,
                          cudaStream_t s);
// halo message of a slab: nslot slots (list) of nplanes consecutive planes,
// [nslot][nplanes][nxy] stored values; export = planes -> buffer, import =
// buffer -> planes
struct HaloArgs {
    void* f;
    long long N;
    int nxy, plane, nplanes, nslot;   // planes plane .. plane + nplanes - 1
    int slots[27];
    void* buf;                        // [nslot][nplanes][nxy]
    int import_;
};
constexpr int HALO_MAX = 8;           // halo planes per face at most
cudaError_t launch_halo(int storage, const HaloArgs& h, cudaStream_t s);
cudaError_t launch_debug_collide(int Q, int n, const float* g_in, const float* d, const float* uB,
                                 const float* sigma, const float* S, float tau_mo, float Ksmag,
                                 float* g_out, cudaStream_t s);

}  // namespace hl
