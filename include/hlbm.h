/*
 * hlbm.h -- C ABI of the B300 (sm_103a) homogenized lattice Boltzmann rotor
 * library: wall-modelled LES of rotating blades with the hybrid
 * recursive-regularized collision (HHRRLBM-LES) of arXiv 2510.13726.
 *
 * The calls follow the statement of the problem in the paper: a lattice
 * (Sec. 2.2), rotors given by a voxelised reference grid and prescribed
 * rotation (Sec. 3.1), the time loop of the listing "HHRRLBM-FSI" (Sec. 3.2),
 * and the per-rotor integral forces (Sec. 2.2.2).
 *
 * Conventions
 *  - Lattice units: spacing 1, time step 1, cs^2 = 1/3.  Cells (x, y, z) with
 *    x fastest in memory; cell index = (z * ny + y) * nx + x.
 *  - Ownership: the caller allocates every device buffer (workspace, outputs,
 *    state snapshots) and keeps it alive while the handle uses it.  The handle
 *    itself is a small host object released by hl_destroy.  Host arrays passed
 *    in (blade grid, inflow modes) are copied during the call.
 *  - Streams: every device operation runs on the stream given to
 *    hl_lattice_init (a cudaStream_t passed as void*; NULL = legacy default).
 *  - Errors: every call returns an hl_status; none aborts, traps or exits.
 *    hl_last_error() describes the last failure of a handle.
 *  - Not thread-safe: one handle must not be used from two threads at once.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hl_lattice hl_lattice;

typedef int hl_status;
#define HL_OK 0
#define HL_ERR_ARG (-1)         /* invalid argument or unsupported combination */
#define HL_ERR_CUDA (-2)        /* a CUDA runtime call failed (see hl_last_error) */
#define HL_ERR_NONFINITE (-3)   /* a non-finite density appeared on the device */
#define HL_ERR_WORKSPACE (-4)   /* workspace or buffer smaller than required */
#define HL_ERR_STATE (-5)       /* call not valid in the current state */
#define HL_ERR_MASS (-8)        /* total mass drifted beyond mass_tol */
#define HL_ERR_GEOMETRY (-9)    /* a wall-model sample point or a band-strain stencil left its
                                   rotor's box: the blade grid needs more padding (the cell
                                   was left unmodelled) */

#define HL_STORE_F32 0          /* populations stored as FP32 of f_i - w_i */
#define HL_STORE_F16S 1         /* populations stored as FP16 of f_i - w_i */
#define HL_STORE_BF16S 2        /* populations stored as BF16 of f_i - w_i */

/* Lattice and model parameters.  Fill with hl_config_defaults() first.
 *  q               19 (D3Q19, Fig. "D3Q19") or 27 (D3Q27)
 *  storage         HL_STORE_*; arithmetic is FP32 in every case
 *  flow_axis       streamwise axis 0/1/2; with open_boundaries the inlet is
 *                  the plane at index 0 and the outlet the last plane
 *  open_boundaries 1: equilibrium inlet (u_in + turbulence) and equilibrium
 *                  outlet (velocity of the upstream neighbour of the previous
 *                  step) on flow_axis, periodic laterally; 0: fully periodic
 *  tau_mo, c_smag  molecular relaxation time and Smagorinsky constant,
 *                  Eqs. (turbVisc), (tauEff)
 *  u_in            inflow speed along +flow_axis (the initial state is the
 *                  equilibrium at this velocity)
 *  sigma_band      hybridisation factor of the band cells off the wall set,
 *                  0 <= sigma_band <= 1 (Sec. 2.2, hybrid non-equilibrium):
 *                  below 1 their non-equilibrium part mixes in the
 *                  Chapman-Enskog term of the finite-difference strain
 *                  (central differences of the pre-collision velocity of
 *                  the six axis neighbours); wall cells use sigma = 0 with
 *                  the wall model's strain
 *  eps_h           width of the porosity transition (Definition "Lattice Porosity")
 *  transition      0 smoothstep t^2 (3 - 2t), 1 linear s = phi/eps + 1/2
 *  wall_model      1: Spalding wall function on the wall cells (Sec. 2.2.1)
 *  wm_E, wm_kappa  Eq. (spalding) constants (9.8, 0.41)
 *  wm_ysample      sampling distance along the wall normal (cells)
 *  wm_tol, wm_maxit  Newton stopping rule (1e-4, 10)
 *  n_modes, modes  synthetic inflow turbulence: host array [n_modes][9] of
 *                  k(3), a(3), b(3); u = U a + sum a cos(k.x') + b sin(k.x'),
 *                  x' = x - U t a
 *  mass_check_every  every K steps an FP64 mass total is taken (0 = never)
 *  mass_tol        relative drift of the total mass that fails the check
 *  overlap         1: with rotors, the cells outside every rotor box are
 *                  collided on the lattice's stream while the embedding,
 *                  wall model, box collision and force reduction run on an
 *                  internal high-priority stream (ordered by events; same
 *                  results bit for bit); 0: everything on one stream
 *  layout          population layout of the single buffer: 0 the AA pattern
 *                  (even steps read and write each cell's own slots, odd
 *                  steps its neighbours'), 1 the esoteric twist (every step
 *                  a cell reads and writes the links to its +x/+y/+z
 *                  neighbours, the slot of each link alternating with the
 *                  step parity), 2 the AA pattern with each x row of a slot
 *                  stored as its two halves interleaved (cell x < nx/2 at
 *                  position 2x, cell x >= nx/2 at 2(x - nx/2) + 1; nx even):
 *                  the bulk launch then moves the cell pair (x, x + nx/2)
 *                  with one aligned access per slot at both step parities.
 *                  Same cell model; hl_grad permutes layouts 1 and 2 into
 *                  the AA layout of the same step for its sweep and back
 *  halo_lo, halo_hi  slab of a lattice decomposed along z (the domain
 *                  decomposition of the paper's multi-GPU runs, Sec. 5):
 *                  D > 0 makes the planes z < D (halo_lo) or z >= nz - D
 *                  (halo_hi) halo planes that stand for the neighbouring
 *                  slab's planes next to the face (0 <= D <= 8; the owned
 *                  planes number at least max(halo_lo, halo_hi)).  One plane
 *                  carries the streaming across the face; a face that cuts a
 *                  rotor's box needs at least ceil(wm_ysample) + 2 (the
 *                  wall-model sample reaches through it).  Halo planes are
 *                  never collided, take no part in the mass total, and their
 *                  fields are undefined;
 *                  with flow_axis 2 the open face on that side is absent (the
 *                  inlet belongs to the first slab, the outlet to the last).
 *                  Every odd step is bracketed by hl_halo_export /
 *                  hl_halo_import of each halo face (see there).  Needs
 *                  layout 0 or 2; hl_grad rejects slabs (HL_ERR_STATE).
 *  z_offset        global z index of local plane 0 (the synthetic inflow is
 *                  evaluated at global coordinates); 0 for a whole lattice,
 *                  -1 for the first slab of a periodic decomposition
 */
typedef struct hl_config {
    int nx, ny, nz;
    int q;
    int storage;
    int flow_axis;
    int open_boundaries;
    double tau_mo, c_smag, u_in;
    double sigma_band, eps_h;
    int transition;
    int wall_model;
    double wm_E, wm_kappa, wm_ysample, wm_tol;
    int wm_maxit;
    int n_modes;
    const double* modes;
    int mass_check_every;
    double mass_tol;
    int overlap;
    int layout;
    int halo_lo, halo_hi;
    int z_offset;
} hl_config;

/* A rotor: n_blades copies of one blade grid plus a hub sphere (Sec. 3.1).
 *  center          rotor centre (lattice coordinates, may be fractional)
 *  axis            rotation axis 0/1/2 (positive rotation right-handed about +axis)
 *  n_blades        1..8; blade k sits at azimuth phase0 + 2 pi k / n_blades
 *  hub_radius      hub sphere radius (0: none)
 *  phase0          rotor angle at t = 0
 *  sdf             host pointer, float [gz][gy][gx]: signed distance of ONE
 *                  blade, negative inside, on a grid in the blade frame
 *                  (R = span, T = tangential, A = axial), node (i,j,k) at
 *                  origin + spacing * (i, j, k); copied by hl_set_rotor
 */
typedef struct hl_rotor_geometry {
    double center[3];
    int axis;
    int n_blades;
    double hub_radius;
    double phase0;
    const float* sdf;
    int gx, gy, gz;
    double origin[3];
    double spacing;
} hl_rotor_geometry;

/* Default parameters (D3Q19, FP32 storage, z streamwise, open boundaries,
 * tau_mo 0.5005, C_S 0.1, u_in 0.05, smoothstep over eps_h = 2, wall model on
 * with E 9.8, kappa 0.41, y_s 2, tol 1e-4, 10 iterations; mass check every 100
 * steps with 5 % tolerance; overlap on).  The grid size is left at 0 and must be set. */
void hl_config_defaults(hl_config* cfg);

/* Bytes of device workspace hl_lattice_init needs for cfg.  Host only. */
hl_status hl_workspace_size(const hl_config* cfg, size_t* bytes);

/* Create a lattice in the caller's device workspace (>= hl_workspace_size,
 * 256-byte aligned) and set the initial state f = f^eq(1, u_in a), t = 0.
 * stream: cudaStream_t (as void*) used by every later call.  Asynchronous. */
hl_status hl_lattice_init(hl_lattice** out, const hl_config* cfg, void* d_workspace, size_t bytes,
                          void* stream);

/* Bytes of device workspace hl_set_rotor needs for this geometry: the blade
 * grid copy plus the band arrays of the rotor's box of cells. */
hl_status hl_rotor_workspace_size(const hl_lattice* lat, const hl_rotor_geometry* geom, size_t* bytes);

/* Add a rotor turning at omega (rad per step) with blade pitch `pitch` (rad,
 * a rigid rotation of each blade about its span axis that increases the
 * section angle to the rotor plane).  The rotor's box of cells (every cell
 * the blades or the hub can reach at any angle) must lie inside the lattice,
 * at least 4 cells from the inlet/outlet planes, and not overlap another
 * rotor's box; otherwise HL_ERR_ARG.  At most 8 rotors. */
hl_status hl_set_rotor(hl_lattice* lat, int* rotor_id, const hl_rotor_geometry* geom, double omega,
                       double pitch, void* d_workspace, size_t bytes);

/* Advance n time steps in the order of the listing "HHRRLBM-FSI": porosity
 * embedding of every rotor box and wall model on the wall cells; fused
 * collide-and-stream; momentum-exchange force and torque per rotor; evolve
 * the rotor angle.  Then synchronises the stream and reports the device
 * error word (HL_ERR_NONFINITE, HL_ERR_MASS, HL_ERR_GEOMETRY; sticky until hl_load_state or
 * hl_lattice_init). */
hl_status hl_step(hl_lattice* lat, int n);

/* As hl_step without the final synchronisation; call hl_check later. */
hl_status hl_step_async(hl_lattice* lat, int n);

/* Synchronise the stream and report the device error word. */
hl_status hl_check(hl_lattice* lat);

/* Force on each rotor (FP64, lattice units, [n_rotors][3]) from the
 * momentum exchange of the last step, and its mean over the steps since the
 * last reset (Sec. 2.2.2).  Thrust = F . axis.  Either pointer may be NULL.
 * reset_avg != 0 restarts the mean after reading.  Synchronises. */
hl_status hl_forces(hl_lattice* lat, double* F, double* F_avg, int reset_avg);

/* Enqueue on the lattice's stream, without synchronising, a copy of the last
 * enqueued step's loads into h_loads (host, [n_rotors][6] doubles: F(3) then
 * M(3), as hl_forces / hl_moments report them; page-locked memory keeps the
 * copy asynchronous).  The values are there once the stream has passed the
 * copy (an event recorded after this call, or hl_check).  Lets a time loop
 * read every step's thrust and torque while the next steps run. */
hl_status hl_loads_async(hl_lattice* lat, double* h_loads);

/* Torque about each rotor centre, [n_rotors][3], last step and mean. */
hl_status hl_moments(hl_lattice* lat, double* M, double* M_avg);

/* Density d_rho[N] and velocity d_u[3][N] (device, FP32) of the current
 * populations.  Values on open boundary planes are not defined by the scheme. */
hl_status hl_fields(hl_lattice* lat, float* d_rho, float* d_u);

/* Replace the state by f = f^eq(rho, u) from device arrays d_rho[N] and
 * d_u[3][N] (either may be NULL: rho = 1, u = 0); resets t to 0. */
hl_status hl_init_fields(hl_lattice* lat, const float* d_rho, const float* d_u);

/* FP64 total mass sum_x sum_i f_i of the stored populations (every stored
 * value converted to FP64 before it is added).  Synchronises. */
hl_status hl_mass(hl_lattice* lat, double* mass);

/* Number of steps taken since init (or since the loaded state's time). */
hl_status hl_get_time(const hl_lattice* lat, long long* t);

/* Bytes of a state snapshot, and device-to-device save / restore of the
 * complete dynamic state (populations, outlet plane, wall-model state, force
 * accumulators, time).  Restoring reproduces later steps bit for bit. */
hl_status hl_state_size(const hl_lattice* lat, size_t* bytes);
hl_status hl_save_state(hl_lattice* lat, void* d_buf, size_t bytes);
hl_status hl_load_state(hl_lattice* lat, const void* d_buf, size_t bytes);

/* Torque-driven rotation ("evolve structure" of the listing "HHRRLBM-FSI"
 * as a rigid rotor): from the next step on, rotor `rotor` turns with the
 * angle and angular velocity it has now, advanced after every step by
 *   theta += Omega;  Omega += (M . a - Q_gen(Omega)) / inertia,
 *   Q_gen = q_gen0 + k_gen Omega |Omega|   (lattice units, dt = 1),
 * with M the step's momentum-exchange torque about the rotor centre.  The
 * state lives on the device (no host round trip per step) and is part of
 * state snapshots.  inertia > 0 (HL_ERR_ARG otherwise).  Calling it again
 * changes the parameters and keeps the state.  hl_grad rejects driven
 * rotors (HL_ERR_STATE).  Synchronises. */
hl_status hl_set_drive(hl_lattice* lat, int rotor, double inertia, double k_gen, double q_gen0);

/* Angle (rad) and angular velocity (rad per step) of rotor `rotor` at the
 * current step (host outputs); prescribed rotors report theta0 + Omega t.
 * Synchronises. */
hl_status hl_drive_state(hl_lattice* lat, int rotor, double* theta, double* omega);

/* Box of rotor `rotor`: lo[3] first cell, n[3] extent (host outputs). */
hl_status hl_rotor_box(const hl_lattice* lat, int rotor, int* lo, int* n);

/* Copy the rotor's band arrays of the last porosity update into device
 * buffers of box size: porosity d (float), flags (uint8: bit 0 force cell
 * d < 1, bit 1 wall cell), wall-model output wm (float [9][box]: modelled
 * velocity xyz, strain xx yy zz xy xz yz), friction velocity utau (double).
 * Any pointer may be NULL. */
hl_status hl_rotor_band(hl_lattice* lat, int rotor, float* d_d, unsigned char* d_flags, float* d_wm,
                        double* d_utau);

/* Velocity set of the library's slot order: c[q][3] and w[q] (host). */
hl_status hl_velocity_set(int q, int* c, double* w);

/* Collide n independent cells on the device (unit checks of Eq. (hlbm)).
 * d_g_in / d_g_out: [n][q] shifted populations f_i - w_i in the slot order
 * of hl_velocity_set.  Band data d_d[n], d_uB[n][3], d_sigma[n],
 * d_S[n][6] (xx yy zz xy xz yz) select the homogenized branch; pass all four
 * NULL for the bulk branch.  Runs on `stream`; does not synchronise. */
hl_status hl_debug_collide(int q, int n, const float* d_g_in, const float* d_d, const float* d_uB,
                           const float* d_sigma, const float* d_S, double tau_mo, double c_smag,
                           float* d_g_out, void* stream);

/* As hl_debug_collide for the bulk branch, through the packed two-cell
 * collision of the bulk launch (cells 2k and 2k+1 share a thread's FP32x2
 * operations); n even (HL_ERR_ARG otherwise).  Runs on `stream`. */
hl_status hl_debug_collide_pair(int q, int n, const float* d_g_in, double tau_mo, double c_smag, float* d_g_out,
                                void* stream);

/* ---- gradients (discrete adjoint of the step) ----
 *
 * Objective over the next `steps` steps from the current state:
 *   J = (1/avg_last) sum over the last avg_last steps of
 *       sum_k [ w_thrust[k] F_k . a_k + w_torque[k] M_k . a_k ]
 * (F, M: the momentum-exchange force and torque of Sec. 2.2.2, a_k the rotor
 * axis).  Its gradient is taken with respect to each rotor's pitch and to a
 * static porosity multiplier d0 (d = d0 d_rotor in Eq. (convexVelocity),
 * d0 = 1 unless set by hl_set_d0), with the step's cell sets (force cells,
 * wall cells, closest blade) held at their forward values; the wall-model
 * Newton solves are differentiated through the iterations they took. */

/* Static porosity multiplier d0[N] (device FP32, caller-owned, read by every
 * later step while set; NULL restores d0 = 1).  Cells outside the rotors'
 * force sets then relax towards rest with weight 1 - d0. */
hl_status hl_set_d0(hl_lattice* lat, const float* d_d0);

/* Inflow from the caller (a precursor run, measured data): d_plane is a
 * device FP32 array [3][n_c][n_b] of inlet velocities (components x, y, z;
 * (b, c) = the two axes after flow_axis in cyclic order, b fastest - the
 * layout of the outlet plane), caller-owned and read by the inlet cells of
 * every later step while set, so the caller may overwrite it between steps
 * on the lattice's stream; NULL restores the synthetic inflow of the
 * configuration (u_in and its Fourier modes, Sec. 4 inflow condition).
 * HL_ERR_STATE without open boundaries.  hl_grad reads the plane in every
 * step of its sweep (forward pass and recompute), so the inflow over the
 * sweep is the plane's content at the call; the inlet equilibrium does not
 * depend on the state, so the plane enters no derivative. */
hl_status hl_set_inflow_plane(hl_lattice* lat, const float* d_plane);

/* Change the pitch of rotor `rotor` (rad) for the following steps. */
hl_status hl_set_pitch(hl_lattice* lat, int rotor, double pitch);

/* on != 0: from now on the cell sets follow the pitches the rotors have at
 * this call while porosity, normals and wall distances follow later
 * hl_set_pitch calls (finite-difference checks of the pitch gradient with
 * the sets frozen, as the gradient has them); on = 0: both follow the pitch. */
hl_status hl_freeze_sets(hl_lattice* lat, int on);

/* Bytes of device workspace hl_grad needs: (ceil(steps / ckpt_every) + 1)
 * state checkpoints, ckpt_every - 1 population buffers of a recomputed
 * segment, two adjoint population arrays and small per-rotor arrays. */
hl_status hl_grad_workspace_size(const hl_lattice* lat, int steps, int ckpt_every, size_t* bytes);

/* Run `steps` steps (the lattice ends exactly where hl_step(lat, steps)
 * leaves it, force averages included) and return J (host double, may be
 * NULL), dJ/dpitch[n_rotors] (host double, may be NULL) and dJ/dd0 (device
 * float [N], overwritten; may be NULL).  w_thrust, w_torque: host
 * [n_rotors]; 1 <= avg_last <= steps; ckpt_every >= 1 sets the checkpoint
 * spacing (memory vs. one recomputed forward step per step).  d_work:
 * caller's device workspace of hl_grad_workspace_size bytes, 256-byte
 * aligned, overwritten.  Synchronises; HL_ERR_NONFINITE / HL_ERR_MASS as
 * hl_step; HL_ERR_STATE for a torque-driven rotor (the derivative covers
 * prescribed rotation; with sigma_band < 1 it includes the finite-difference
 * strain of the band cells, transposed onto their neighbours' populations;
 * a caller's inflow plane is held at its content for the whole sweep).  With the esoteric-twist
 * layout the state is permuted into the AA layout of the same step for the
 * sweep (the two layouts give the same trajectory; the copy lives in
 * d_work) and back at the end, also when the sweep fails. */
hl_status hl_grad(hl_lattice* lat, int steps, int avg_last, int ckpt_every, const double* w_thrust,
                  const double* w_torque, double* J, double* dJ_dpitch, float* d_dJ_dd0, void* d_work,
                  size_t bytes);

/* Vector-Jacobian product of the collision of n independent cells (unit
 * checks): arguments as hl_debug_collide, plus d_lam_star[n][q] (adjoint of
 * the post-collision populations) -> d_lam[n][q] (adjoint of the
 * pre-collision populations) and, for the homogenized branch, the adjoint
 * of the band data d_gd[n], d_guB[n][3], d_gS[n][6] (each may be NULL).
 * Runs on `stream`; does not synchronise. */
hl_status hl_debug_collide_vjp(int q, int n, const float* d_g_in, const float* d_d, const float* d_uB,
                               const float* d_sigma, const float* d_S, double tau_mo, double c_smag,
                               const float* d_lam_star, float* d_lam, float* d_gd, float* d_guB, float* d_gS,
                               void* stream);

/* Per-kernel timing with CUDA events recorded on the lattice's stream around
 * each launch of the time loop.  hl_profile_begin(lat, capacity) starts
 * recording (at most `capacity` launches per kernel kind; it creates CUDA
 * events, it allocates no device memory); hl_profile_end synchronises,
 * returns for each kind (0 porosity embedding, 1 collide-and-stream of all
 * cells, or of the cells outside every rotor box when overlap is on, 2 force
 * reduction, 3 mass check, 4 wall model, 5 collide-and-stream of rotor boxes
 * when overlap is on) the summed duration in ms and the number of launches
 * ([6] each), and releases the events.  Either output may be NULL. */
hl_status hl_profile_begin(hl_lattice* lat, int capacity);
hl_status hl_profile_end(hl_lattice* lat, double* ms, long long* launches);

/* ---- slabs: halo exchange of a lattice decomposed along z ----
 *
 * In the AA pattern only odd steps move populations between cells.  A slab's
 * boundary cells then read and write the populations with c_z = -1 (lower
 * face) or c_z = +1 (upper face) on the adjacent halo plane, 5 slots on D3Q19
 * and 9 on D3Q27.  Before an odd step the halo plane must hold the
 * neighbour's values of those slots, and after it the values the slab wrote
 * there belong to the neighbour.  So around every odd step, for each halo
 * face, the caller moves one message from each slab to its neighbour:
 *   t odd (before the step):  hl_halo_export(A, 1) -> hl_halo_import(B, 0) and
 *                             hl_halo_export(B, 0) -> hl_halo_import(A, 1);
 *   then the step of every slab;
 *   t even (after the odd step): the same two exchanges again;
 * A the slab below B (its upper neighbour; with z periodic the last slab is
 * below the first).  The library picks the plane and the slot set from the
 * face and the parity of t.  A message is [nslots][nx * ny] stored values
 * (storage type, hl_halo_size bytes); the caller carries it (a device copy
 * on one GPU, a send/receive between ranks).  hl_step on a slab advances one
 * step per call and returns HL_ERR_STATE if a halo face has not imported at
 * the current t (t > 0).
 *
 * A rotor's box may be cut by a halo face of enough planes (see halo_lo):
 * each slab then embeds, models and collides the box cells in its own
 * planes, and the wall-model samples of cells next to the face read the
 * neighbour's planes in the deep halo.  After every step, once both one-plane
 * messages of every face have been imported, each such face also moves its
 * deep message (every slot of the D planes next to it) with
 * hl_halo_deep_export / hl_halo_deep_import; before the first step too.  The
 * force and torque of a cut rotor are this slab's share (sum them over the
 * slabs); its force reduction of a step runs at the next hl_step_async or
 * the next load query (hl_forces, hl_moments, hl_loads_async,
 * hl_save_state), which must come after the deep exchange.  A cut rotor
 * takes no hl_set_drive (HL_ERR_STATE: its torque is split over the slabs). */

/* Bytes of one halo message of this lattice (HL_ERR_ARG without halo planes). */
hl_status hl_halo_size(const hl_lattice* lat, size_t* bytes);

/* Copy the outgoing message of face `face` (0 lower, 1 upper; must be a halo
 * face, HL_ERR_ARG otherwise) into the caller's device buffer d_buf
 * (hl_halo_size bytes).  Asynchronous on the lattice stream. */
hl_status hl_halo_export(hl_lattice* lat, int face, void* d_buf);

/* Store the neighbour's message for face `face` (d_buf, device, as written
 * by the neighbour's hl_halo_export of the opposite face at the same t) and
 * record that the face is up to date at the current t.  Asynchronous on the
 * lattice stream: the caller orders it after the neighbour's export. */
hl_status hl_halo_import(hl_lattice* lat, int face, const void* d_buf);

/* Bytes of the deep message of face `face`: every slot of its D halo planes,
 * [q][D][nx * ny] stored values (HL_ERR_ARG if the face has no halo). */
hl_status hl_halo_deep_size(const hl_lattice* lat, int face, size_t* bytes);

/* Copy every slot of the slab's own D planes next to face `face` into d_buf
 * (hl_halo_deep_size bytes, device).  Asynchronous on the lattice stream;
 * call after the one-plane imports of the current t on both sides. */
hl_status hl_halo_deep_export(hl_lattice* lat, int face, void* d_buf);

/* Store the neighbour's deep message (its hl_halo_deep_export of the opposite
 * face at the same t; both faces have the same D) into the D halo planes of
 * face `face` and record the face as up to date at the current t. */
hl_status hl_halo_deep_import(hl_lattice* lat, int face, const void* d_buf);

/* Total mass of a population array, without allocating anything.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory when they need the total (code inside a memory pool
 * that forbids new allocations, a driver that has given all device memory to
 * the lattice, a callback whose allocator is not re-entrant).  The block
 * partial sums live in a fixed array in the library's own static device
 * memory (4096 doubles plus a counter, held by every GPU that loads the
 * library until the process exits); nothing is allocated, by the library or
 * by any library it calls.
 *  q, storage  lattice (19 or 27) and storage kind (HL_STORE_*) of d_f
 *  d_f         device populations [q][n_cells], stored as f_i - w_i
 *  d_mass      device output: sum_x sum_i f_i in FP64
 *  stream      cudaStream_t as void*; the call is asynchronous
 * At most 2^32 stored values (q * n_cells) are accepted: larger arrays return
 * HL_ERR_WORKSPACE.  The first call on a device looks up the array's device
 * address (once per device, with that device current), so make that first
 * call before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (two streams, or two threads) race and must be ordered
 * by the caller.  An error still pending on the calling thread from earlier
 * CUDA work is reported as HL_ERR_CUDA before anything is launched (reading
 * it clears it, as for any CUDA runtime call). */
hl_status hl_mass_noalloc(int q, int storage, const void* d_f, long long n_cells, double* d_mass,
                          void* stream);

/* Text of the last error of the handle (never NULL). */
const char* hl_last_error(const hl_lattice* lat);

/* Release the handle (host memory).  Device buffers stay the caller's. */
void hl_destroy(hl_lattice* lat);

#ifdef __cplusplus
}
#endif

#endif /* HLBM_H */
