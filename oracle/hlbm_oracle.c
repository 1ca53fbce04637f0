/*
 * FP64 CPU oracle of the homogenized hybrid recursive-regularized lattice
 * Boltzmann rotor scheme (HHRRLBM-LES with Smagorinsky closure and a
 * Spalding wall model), arXiv 2510.13726.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct
 * statement of what the CUDA library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the library
 * never does.  It shares no code, header or table with the library.
 *
 * Every formula is written out in its textbook/tensor form in FP64: Hermite
 * tensors as full 3x3 and 3x3x3 arrays, contractions as explicit loops, two
 * population buffers with pull streaming.  Section / equation references are
 * to the paper:
 *   Eq. (hlbm)            homogenized LB update, Sec. 2.2
 *   hybrid f~(1)          Sec. 2.2, after Eq. (hlbm)
 *   f(1), a1(n)           Hermite expansion of the non-equilibrium, Sec. 2.2
 *   f(1,FD)               finite-difference non-equilibrium, Sec. 2.2
 *   f eq                  third-order equilibrium, Sec. 2.2
 *   Eq. (convexVelocity)  homogenized velocity
 *   Eq. (tauEff), (turbVisc)  Smagorinsky effective relaxation time
 *   Eqs. (u+), (y+), (spalding), (implicitWF), (guess)  wall model, Sec. 2.2.1
 *   Definition "Lattice Porosity"  and momentum exchange, Sec. 2.2.2
 *   Listing "HHRRLBM-FSI"  per-step order of operations, Sec. 3.2
 *
 * Readings where the paper is ambiguous (all mirrored by the library):
 *  - the convex velocity is u^ = d u + (1-d) u^B with d = 1 in fluid
 *    (the printed Eq. (convexVelocity) has the weights the other way round,
 *    which contradicts the porosity definition d = 1 for phi >= eps/2);
 *  - the third-order equilibrium term is the full tensor contraction divided
 *    by 3! cs^6, and a0^(n) = rho u^(x)n;
 *  - a1^(3) follows the recursion a1_abg = u_a a1_bg + u_b a1_ag + u_g a1_ab
 *    with a1^(2) = Pi_neq taken against the fluid velocity u;
 *  - f(1,FD) = w_i rho tau_eff / cs^2 H2 : S_FD;
 *  - away from wall cells, S_FD of a band cell with sigma < 1 is the
 *    symmetric part of the velocity gradient by central differences of the
 *    pre-collision velocity j/rho of the six axis neighbours (periodic
 *    wrap laterally; one-sided where a neighbour is across an open face);
 *  - tau_eff is the positive root of tau = tau_mo + 3 C_S^2 |S| with
 *    S = -Pi_neq / (2 rho cs^2 tau) and |S| = sqrt(2 S:S);
 *  - the transition function is a smoothstep t^2 (3 - 2t), t = phi/eps + 1/2
 *    (linear on request, as printed);
 *  - momentum exchange uses the Galilean-invariant link form
 *    F = sum_{x: d<1} sum_{i>0} [(c_ibar - u_s) f*_ibar(x+c_i) - (c_i - u_s) f*_i(x)]
 *    on post-collision populations (the printed formula lost the opposite
 *    index; its literal sign pattern is kept as option force_form = 1);
 *  - wall cells are W = {0 <= phi < eps/2}; y1 = max(phi, 1/2) n; the wall
 *    function is sampled at x + y_s n, and its result (modelled velocity
 *    added to u^B, FD strain, sigma = 0) is used by the same step's
 *    collision; the wall model runs after the porosity update and before
 *    collide-and-stream (the listing's cyclic order with the porosity update
 *    first, so the modelled velocity is defined on the step's own wall set);
 *  - the geometry decision value phi is evaluated in binary32 with a fixed
 *    operation order (the kernel's precision), because it decides discrete
 *    cell sets (solid, wall, force cells); everything downstream is FP64.
 */
#include <complex.h>
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXQ 27
#define OR_MAXROT 16

/* ------------------------------------------------------------------ */
/* lattice: velocities, weights, Hermite tensors                       */
/* ------------------------------------------------------------------ */

typedef struct {
    int q;
    int c[OR_MAXQ][3];
    double w[OR_MAXQ];
    int opp[OR_MAXQ];
    double H2[OR_MAXQ][3][3];
    double H3[OR_MAXQ][3][3][3];
} or_lattice;

static const double CS2 = 1.0 / 3.0;

static int delta(int a, int b) { return a == b ? 1 : 0; }

/* D3Q19 / D3Q27 velocity sets (Fig. "D3Q19"); weights by shell |c|^2. */
static int lattice_init(or_lattice* L, int q)
{
    if (q != 19 && q != 27) return -1;
    L->q = q;
    int n = 0;
    for (int shell = 0; shell <= 3; ++shell) {
        for (int cx = -1; cx <= 1; ++cx)
            for (int cy = -1; cy <= 1; ++cy)
                for (int cz = -1; cz <= 1; ++cz) {
                    int s = cx * cx + cy * cy + cz * cz;
                    if (s != shell) continue;
                    if (q == 19 && s == 3) continue;
                    L->c[n][0] = cx; L->c[n][1] = cy; L->c[n][2] = cz;
                    double w;
                    if (q == 19) w = (s == 0) ? 1.0 / 3.0 : (s == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                    else w = (s == 0) ? 8.0 / 27.0 : (s == 1) ? 2.0 / 27.0 : (s == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
                    L->w[n] = w;
                    ++n;
                }
    }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    /* Hermite polynomials of the discrete velocities (cs^2 = 1/3):
       H2_ab = c_a c_b - cs2 d_ab,
       H3_abg = c_a c_b c_g - cs2 (c_a d_bg + c_b d_ag + c_g d_ab). */
    for (int i = 0; i < q; ++i) {
        const int* c = L->c[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                L->H2[i][a][b] = c[a] * c[b] - CS2 * delta(a, b);
                for (int g = 0; g < 3; ++g)
                    L->H3[i][a][b][g] = (double)(c[a] * c[b] * c[g])
                        - CS2 * (c[a] * delta(b, g) + c[b] * delta(a, g) + c[g] * delta(a, b));
            }
    }
    return 0;
}

static double contract2(const double H[3][3], const double A[3][3])
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += H[a][b] * A[a][b];
    return s;
}

static double contract3(const double H[3][3][3], const double A[3][3][3])
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int g = 0; g < 3; ++g) s += H[a][b][g] * A[a][b][g];
    return s;
}

/* ------------------------------------------------------------------ */
/* local cell model                                                    */
/* ------------------------------------------------------------------ */

/* Third-order equilibrium (Sec. 2.2):
   f_i^eq = w_i ( rho + c_i.rho u / cs2 + H2:a0^(2) / (2 cs4) + H3:a0^(3) / (6 cs6) ),
   a0^(2) = rho u u, a0^(3) = rho u u u. */
static void equilibrium(const or_lattice* L, double rho, const double u[3], double* feq)
{
    double A2[3][3], A3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            A2[a][b] = rho * u[a] * u[b];
            for (int g = 0; g < 3; ++g) A3[a][b][g] = rho * u[a] * u[b] * u[g];
        }
    for (int i = 0; i < L->q; ++i) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        feq[i] = L->w[i] * (rho + rho * cu / CS2
                            + contract2(L->H2[i], A2) / (2.0 * CS2 * CS2)
                            + contract3(L->H3[i], A3) / (6.0 * CS2 * CS2 * CS2));
    }
}

/* Moments: rho = sum f, j = sum c f, Pi = sum c c f. */
static void moments(const or_lattice* L, const double* f, double* rho, double j[3], double Pi[3][3])
{
    double r = 0.0;
    double m[3] = {0, 0, 0};
    double P[3][3] = {{0}};
    for (int i = 0; i < L->q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) {
            m[a] += L->c[i][a] * f[i];
            for (int b = 0; b < 3; ++b) P[a][b] += L->c[i][a] * L->c[i][b] * f[i];
        }
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) {
        j[a] = m[a];
        for (int b = 0; b < 3; ++b) Pi[a][b] = P[a][b];
    }
}

/* Smagorinsky effective relaxation time, Eqs. (turbVisc), (tauEff) with
   dx = dt = 1: tau = tau_mo + 3 C_S^2 |S|, S = -Pi_neq / (2 rho cs2 tau),
   |S| = sqrt(2 S:S).  The positive root of the resulting quadratic is
   tau = (tau_mo + sqrt(tau_mo^2 + 18 sqrt(2) C_S^2 sqrt(Pi_neq:Pi_neq) / rho)) / 2. */
static double smagorinsky_tau(double tau_mo, double c_smag, double rho, const double Pneq[3][3])
{
    double Q = contract2(Pneq, Pneq);
    return 0.5 * (tau_mo + sqrt(tau_mo * tau_mo + 18.0 * sqrt(2.0) * c_smag * c_smag * sqrt(Q) / rho));
}

/* Regularized non-equilibrium (Sec. 2.2): f_i^(1) = w_i ( H2:a1^(2) / (2 cs4)
   + H3:a1^(3) / (6 cs6) ), a1^(0) = a1^(1) = 0, a1^(2) = Pi_neq,
   a1^(3)_abg = u_a a1_bg + u_b a1_ag + u_g a1_ab  (recursive, with u^). */
static void regularized_neq(const or_lattice* L, const double a2[3][3], const double u[3], double* f1)
{
    double a3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int g = 0; g < 3; ++g)
                a3[a][b][g] = u[a] * a2[b][g] + u[b] * a2[a][g] + u[g] * a2[a][b];
    for (int i = 0; i < L->q; ++i)
        f1[i] = L->w[i] * (contract2(L->H2[i], a2) / (2.0 * CS2 * CS2)
                           + contract3(L->H3[i], a3) / (6.0 * CS2 * CS2 * CS2));
}

/* Finite-difference non-equilibrium (Sec. 2.2): f_i^(1,FD) = w_i rho tau / cs2 H2:S_FD. */
static void fd_neq(const or_lattice* L, double rho, double tau, const double S[3][3], double* f1fd)
{
    for (int i = 0; i < L->q; ++i) f1fd[i] = L->w[i] * rho * tau / CS2 * contract2(L->H2[i], S);
}

typedef struct {
    double d;        /* lattice porosity (1 = fluid) */
    double uB[3];    /* solid (boundary) velocity incl. wall-model correction */
    double sigma;    /* hybridisation factor */
    double Sfd[3][3];/* finite-difference strain rate */
} cell_band;

/* One HHRRLBM-LES collision, Eq. (hlbm):
   f_i* = f_i^eq(rho, u^) + (1 - 1/tau_eff) ( sigma f_i^(1) - (1 - sigma) f_i^(1,FD) ).
   Returns tau_eff. */
static double collide(const or_lattice* L, const double* f, const cell_band* B,
                      double tau_mo, double c_smag, double* fout, double u_out[3])
{
    double rho, j[3], Pi[3][3];
    moments(L, f, &rho, j, Pi);
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double Pneq[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Pneq[a][b] = Pi[a][b] - rho * CS2 * delta(a, b) - rho * u[a] * u[b];
    double tau = smagorinsky_tau(tau_mo, c_smag, rho, Pneq);
    /* Eq. (convexVelocity), read with d = 1 in the fluid */
    double uh[3];
    for (int a = 0; a < 3; ++a) uh[a] = B->d * u[a] + (1.0 - B->d) * B->uB[a];
    double feq[OR_MAXQ], f1[OR_MAXQ], f1fd[OR_MAXQ];
    equilibrium(L, rho, uh, feq);
    regularized_neq(L, Pneq, uh, f1);
    fd_neq(L, rho, tau, B->Sfd, f1fd);
    for (int i = 0; i < L->q; ++i) {
        double ft = B->sigma * f1[i] - (1.0 - B->sigma) * f1fd[i];
        fout[i] = feq[i] + (1.0 - 1.0 / tau) * ft;
    }
    if (u_out) { u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2]; }
    return tau;
}

/* ------------------------------------------------------------------ */
/* wall function, Sec. 2.2.1                                           */
/* ------------------------------------------------------------------ */

/* Truncated Spalding law, Eq. (spalding): y+ as a function of u+. */
static double spalding_yplus(double up, double E, double kappa)
{
    double k = kappa * up;
    return up + (exp(k) - 1.0 - k - 0.5 * k * k - k * k * k / 6.0) / E;
}

/* dy+/du+ */
static double spalding_dyplus(double up, double E, double kappa)
{
    double k = kappa * up;
    return 1.0 + kappa / E * (exp(k) - 1.0 - k - 0.5 * k * k);
}

/* Eq. (implicitWF): f(u_tau) = y+(u/u_tau) - y u_tau / nu. */
static double wf_residual(double ut, double u, double y, double nu, double E, double kappa)
{
    return spalding_yplus(u / ut, E, kappa) - y * ut / nu;
}

/* The Newton step f/f' of Eq. (implicitWF) at u_tau = ut, with numerator and
   denominator both multiplied by exp(-kappa u+) before the division: the
   same quotient, but neither factor overflows when the iterate lies far
   below the root (f and f' both grow like exp(kappa u+); f' leaves the FP64
   range for kappa u+ above ~700, where the plain quotient would be 0 and
   the iterate would stop moving).  There the step tends to -ut/(kappa u+). */
static double wf_step(double ut, double u, double y, double nu, double E, double kappa)
{
    double up = u / ut, k = kappa * up, s = exp(-k);
    double P2 = 1.0 + k + 0.5 * k * k, P3 = P2 + k * k * k / 6.0;
    double fs = (up - y * ut / nu) * s + (1.0 - P3 * s) / E;
    double fps = -(s + kappa / E * (1.0 - P2 * s)) * up / ut - y / nu * s;
    return fs / fps;
}

/* Newton-Raphson for u_tau (Sec. 2.2.1): iterate until the residual changes by
   less than tol between iterates, at most maxit iterations; a non-positive
   iterate is replaced by half the previous one. */
static double wf_newton(double u, double y, double nu, double guess, double E, double kappa,
                        double tol, int maxit, int* iters)
{
    double ut = guess;
    double fv = wf_residual(ut, u, y, nu, E, kappa);
    int it = 0;
    while (it < maxit) {
        double un = ut - wf_step(ut, u, y, nu, E, kappa);
        if (!(un > 0.0)) un = 0.5 * ut;
        double fn = wf_residual(un, u, y, nu, E, kappa);
        ut = un;
        ++it;
        if (fabs(fn - fv) < tol) break;
        fv = fn;
    }
    if (iters) *iters = it;
    return ut;
}

/* Inverse of Eq. (spalding): u+ for a given y+, by Newton from the right of
   the root (y+ is convex and increasing in u+), same stopping rule. */
static double spalding_uplus(double yp, double E, double kappa, double tol, int maxit)
{
    double lg = log(1.0 + E * yp) / kappa;
    double up = yp < lg ? yp : lg;
    double g = spalding_yplus(up, E, kappa) - yp;
    for (int it = 0; it < maxit; ++it) {
        double un = up - g / spalding_dyplus(up, E, kappa);
        if (!(un > 0.0)) un = 0.5 * up;
        double gn = spalding_yplus(un, E, kappa) - yp;
        up = un;
        if (fabs(gn - g) < tol) break;
        g = gn;
    }
    return up;
}

/* ------------------------------------------------------------------ */
/* rotor geometry and porosity, Sec. 2.2.2 / 3.1                       */
/* ------------------------------------------------------------------ */

typedef struct {
    double center[3];
    int axis;            /* rotor axis = one lattice axis */
    int n_blades;
    double hub_radius;
    double phase0;       /* theta at t = 0 */
    double omega;        /* angular velocity, positive right-handed about +axis */
    double pitch;        /* blade pitch (rad), rigid rotation about the span axis */
    const float* sdf;    /* one blade, [gz][gy][gx], blade frame (R, T, A) */
    int gx, gy, gz;
    double origin[3];
    double spacing;
} or_rotor;

typedef struct {
    or_rotor r;
    float* sdf;          /* owned copy */
    /* torque-driven rotation (listing "HHRRLBM-FSI", evolve structure):
       angle and angular velocity are state, r.omega follows the state */
    int driven;
    double theta;        /* rotor angle of the current step */
    double inertia, k_gen, q_gen0;
} rotor_store;

/* Per-blade binary32 frame: cos/sin of (theta + 2 pi k / n_blades) and of the
   pitch, rounded once from FP64. */
typedef struct { float ck[8], sk[8], cp, sp; double ckd[8], skd[8], cpd, spd; } blade_frames;

/* frames at rotor angle th (blade k at th + 2 pi k / n_blades) */
static void blade_frames_theta(const or_rotor* R, double th, blade_frames* B)
{
    for (int k = 0; k < R->n_blades; ++k) {
        double ang = th + 2.0 * M_PI * (double)k / (double)R->n_blades;
        B->ckd[k] = cos(ang); B->skd[k] = sin(ang);
        B->ck[k] = (float)B->ckd[k]; B->sk[k] = (float)B->skd[k];
    }
    B->cpd = cos(R->pitch); B->spd = sin(R->pitch);
    B->cp = (float)B->cpd; B->sp = (float)B->spd;
}

/* prescribed rotation: theta = theta0 + Omega t */
static void blade_frames_at(const or_rotor* R, long t, blade_frames* B)
{
    blade_frames_theta(R, R->phase0 + R->omega * (double)t, B);
}

/* angle of rotor k at the current step: its state when torque-driven */
static double rotor_angle(const rotor_store* rs, long t)
{
    return rs->driven ? rs->theta : rs->r.phase0 + rs->r.omega * (double)t;
}

static float lerpf_(float a, float b, float t) { return fmaf(t, b - a, a); }

/* Trilinear sample of the blade grid at blade-frame point (pR, qT, qA), in
   binary32 with a fixed order (x, then y, then z).  Returns +inf outside. */
static float blade_sample_f32(const or_rotor* R, float pR, float qT, float qA)
{
    float inv_h = (float)(1.0 / R->spacing);
    float g0 = (pR - (float)R->origin[0]) * inv_h;
    float g1 = (qT - (float)R->origin[1]) * inv_h;
    float g2 = (qA - (float)R->origin[2]) * inv_h;
    float f0 = floorf(g0), f1 = floorf(g1), f2 = floorf(g2);
    if (!(f0 >= 0.0f && f0 <= (float)(R->gx - 2) && f1 >= 0.0f && f1 <= (float)(R->gy - 2)
          && f2 >= 0.0f && f2 <= (float)(R->gz - 2)))
        return INFINITY;
    int i0 = (int)f0, j0 = (int)f1, k0 = (int)f2;
    float tx = g0 - f0, ty = g1 - f1, tz = g2 - f2;
    const float* s = R->sdf;
    size_t sx = 1, sy = (size_t)R->gx, sz = (size_t)R->gx * (size_t)R->gy;
    size_t o = (size_t)k0 * sz + (size_t)j0 * sy + (size_t)i0;
    float v00 = lerpf_(s[o], s[o + sx], tx);
    float v10 = lerpf_(s[o + sy], s[o + sy + sx], tx);
    float v01 = lerpf_(s[o + sz], s[o + sz + sx], tx);
    float v11 = lerpf_(s[o + sz + sy], s[o + sz + sy + sx], tx);
    float w0 = lerpf_(v00, v10, ty);
    float w1 = lerpf_(v01, v11, ty);
    return lerpf_(w0, w1, tz);
}

/* Signed distance of lattice cell (ix, iy, iz) to rotor R at the frames B,
   binary32, fixed order.  which = blade index, or n_blades for the hub. */
static float rotor_phi_f32(const or_rotor* R, const blade_frames* B, int ix, int iy, int iz,
                           int* which)
{
    int a = R->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    int ii[3] = {ix, iy, iz};
    float rl[3];
    for (int k = 0; k < 3; ++k) rl[k] = (float)ii[k] - (float)R->center[k];
    float rb = rl[b], rc = rl[c], ra = rl[a];
    float best = INFINITY;
    int wb = -1;
    for (int k = 0; k < R->n_blades; ++k) {
        float pR = fmaf(B->ck[k], rb, B->sk[k] * rc);
        float pT = fmaf(B->ck[k], rc, -(B->sk[k] * rb));
        float qT = fmaf(B->cp, pT, -(B->sp * ra));
        float qA = fmaf(B->cp, ra, B->sp * pT);
        float v = blade_sample_f32(R, pR, qT, qA);
        if (v < best) { best = v; wb = k; }
    }
    if (R->hub_radius > 0.0) {
        float r2 = fmaf(rb, rb, fmaf(rc, rc, ra * ra));
        float v = sqrtf(r2) - (float)R->hub_radius;
        if (v < best) { best = v; wb = R->n_blades; }
    }
    if (which) *which = wb;
    return best;
}

/* Signed distance of one component (blade `which`, or the hub when which =
   n_blades) at the frames B, with the same binary32 operations as
   rotor_phi_f32: for the component that attains the minimum the two agree
   bit for bit. */
static float component_phi_f32(const or_rotor* R, const blade_frames* B, int which, int ix, int iy, int iz)
{
    int a = R->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    int ii[3] = {ix, iy, iz};
    float rl[3];
    for (int k = 0; k < 3; ++k) rl[k] = (float)ii[k] - (float)R->center[k];
    float rb = rl[b], rc = rl[c], ra = rl[a];
    if (which >= R->n_blades) {
        float r2 = fmaf(rb, rb, fmaf(rc, rc, ra * ra));
        return sqrtf(r2) - (float)R->hub_radius;
    }
    int k = which;
    float pR = fmaf(B->ck[k], rb, B->sk[k] * rc);
    float pT = fmaf(B->ck[k], rc, -(B->sk[k] * rb));
    float qT = fmaf(B->cp, pT, -(B->sp * ra));
    float qA = fmaf(B->cp, ra, B->sp * pT);
    return blade_sample_f32(R, pR, qT, qA);
}

/* Outward unit normal (lab frame, FP64) of the component `which` of rotor R
   at cell (ix, iy, iz): trilinear interpolation of the central-difference
   gradient of the blade grid, rotated back through pitch and azimuth; the
   hub sphere normal is radial. */
static void rotor_normal(const or_rotor* R, const blade_frames* B, int which, int ix, int iy, int iz,
                         double n_out[3])
{
    int a = R->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    double rl[3] = {ix - R->center[0], iy - R->center[1], iz - R->center[2]};
    double v[3] = {0, 0, 0};
    if (which >= R->n_blades) {
        v[0] = rl[0]; v[1] = rl[1]; v[2] = rl[2];
    } else {
        int k = which;
        double rb = rl[b], rc = rl[c], ra = rl[a];
        double ck = B->ckd[k], sk = B->skd[k], cp = B->cpd, sp = B->spd;
        double pR = ck * rb + sk * rc, pT = ck * rc - sk * rb;
        double qT = cp * pT - sp * ra, qA = cp * ra + sp * pT;
        double h = R->spacing;
        double g[3] = {(pR - R->origin[0]) / h, (qT - R->origin[1]) / h, (qA - R->origin[2]) / h};
        int i0 = (int)floor(g[0]), j0 = (int)floor(g[1]), k0 = (int)floor(g[2]);
        if (i0 < 0) i0 = 0;
        if (i0 > R->gx - 2) i0 = R->gx - 2;
        if (j0 < 0) j0 = 0;
        if (j0 > R->gy - 2) j0 = R->gy - 2;
        if (k0 < 0) k0 = 0;
        if (k0 > R->gz - 2) k0 = R->gz - 2;
        double t[3] = {g[0] - i0, g[1] - j0, g[2] - k0};
        double gb[3] = {0, 0, 0};   /* gradient in blade frame (R, T, A) */
        int dims[3] = {R->gx, R->gy, R->gz};
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    int node[3] = {i0 + cx, j0 + cy, k0 + cz};
                    double wgt = (cx ? t[0] : 1 - t[0]) * (cy ? t[1] : 1 - t[1]) * (cz ? t[2] : 1 - t[2]);
                    for (int d = 0; d < 3; ++d) {
                        int lo[3] = {node[0], node[1], node[2]}, hi[3] = {node[0], node[1], node[2]};
                        lo[d] = node[d] > 0 ? node[d] - 1 : node[d];
                        hi[d] = node[d] < dims[d] - 1 ? node[d] + 1 : node[d];
                        size_t olo = ((size_t)lo[2] * R->gy + lo[1]) * R->gx + lo[0];
                        size_t ohi = ((size_t)hi[2] * R->gy + hi[1]) * R->gx + hi[0];
                        double der = ((double)R->sdf[ohi] - (double)R->sdf[olo]) / ((hi[d] - lo[d]) * h);
                        gb[d] += wgt * der;
                    }
                }
        /* undo the pitch rotation, then the azimuth rotation */
        double vT = cp * gb[1] + sp * gb[2];
        double vA = -sp * gb[1] + cp * gb[2];
        double vR = gb[0];
        double lab[3];
        lab[b] = ck * vR - sk * vT;
        lab[c] = sk * vR + ck * vT;
        lab[a] = vA;
        v[0] = lab[0]; v[1] = lab[1]; v[2] = lab[2];
    }
    double nrm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (nrm > 0.0) { n_out[0] = v[0] / nrm; n_out[1] = v[1] / nrm; n_out[2] = v[2] / nrm; }
    else { n_out[0] = n_out[1] = n_out[2] = 0.0; }
}

/* Definition "Lattice Porosity": d = 0 for phi <= -eps/2, s(phi) inside the
   transition, 1 for phi >= eps/2; s = smoothstep(t), t = phi/eps + 1/2, or the
   printed linear s = t. */
static double porosity_of_phi(double phi, double eps, int linear)
{
    if (phi <= -0.5 * eps) return 0.0;
    if (phi >= 0.5 * eps) return 1.0;
    double t = phi / eps + 0.5;
    return linear ? t : t * t * (3.0 - 2.0 * t);
}

/* solid velocity of a rigid rotation: u_s = Omega a x (x - c) */
static void solid_velocity(const or_rotor* R, int ix, int iy, int iz, double us[3])
{
    int a = R->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    double rl[3] = {ix - R->center[0], iy - R->center[1], iz - R->center[2]};
    us[a] = 0.0;
    us[b] = -R->omega * rl[c];
    us[c] = R->omega * rl[b];
}

/* ------------------------------------------------------------------ */
/* whole-lattice state                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz, q;
    int flow_axis;
    int open_boundaries;
    double tau_mo, c_smag, u_in;
    double sigma_band, eps_h;
    int transition;
    int wall_model;
    double wm_E, wm_kappa, wm_ysample, wm_tol;
    int wm_maxit;
    int force_form;
    int n_modes;
    const double* modes;      /* [n_modes][9]: k(3), a(3), b(3) */
} or_params;

enum { FL_B = 1, FL_W = 2 };

typedef struct {
    or_params P;
    double* modes;
    or_lattice L;
    int nrot;
    rotor_store rot[OR_MAXROT];
    size_t N;
    double* f;       /* [q][N] pre-collision populations at the current time */
    double* fpost;   /* [q][N] post-collision */
    float* phi;      /* [N] binary32 decision value */
    double* d;       /* [N] porosity */
    signed char* tag;
    signed char* which; /* [N] component (blade k, n_blades = hub) of force-set cells */
    unsigned char* flags;
    double* nrm;     /* [N][3] */
    double* y1;      /* [N][3] */
    double* wm_du;   /* [N][3] modelled velocity added to u^B */
    double* wm_S;    /* [N][9] modelled strain rate */
    double* wm_ut;   /* [N] friction velocity of the last evaluation */
    unsigned char* wm_active;
    double* uplane[2];
    long step;
    double* d0;      /* [N] static porosity multiplier, NULL = 1 */
    int frozen;      /* 1: cell sets from decision_pitch, porosity and normals from pitch */
    double decision_pitch[OR_MAXROT];
    double F[OR_MAXROT][3], M[OR_MAXROT][3];
    double Fsum[OR_MAXROT][3], Msum[OR_MAXROT][3];
    long navg;
    long wm_newton_iters, wm_evals;
} or_state;

static size_t cidx(const or_state* S, int x, int y, int z)
{
    return ((size_t)z * S->P.ny + (size_t)y) * S->P.nx + (size_t)x;
}

static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* neighbour along c with periodic lateral axes; returns 0 when it leaves
   the domain through an open (inlet/outlet) face */
static int neighbour(const or_state* S, const int x[3], const int c[3], int sgn, int out[3])
{
    int n[3] = {S->P.nx, S->P.ny, S->P.nz};
    for (int k = 0; k < 3; ++k) {
        int v = x[k] + sgn * c[k];
        if (S->P.open_boundaries && k == S->P.flow_axis) {
            if (v < 0 || v >= n[k]) return 0;
            out[k] = v;
        } else {
            out[k] = wrap(v, n[k]);
        }
    }
    return 1;
}

/* inflow velocity at inlet cell x, time t: U a + sum_m a_m cos(k.x') + b_m sin(k.x'),
   x' = x - U t a (frozen turbulence) */
static void inflow_velocity(const or_state* S, int x, int y, int z, long t, double u[3])
{
    int a = S->P.flow_axis;
    double xp[3] = {x, y, z};
    xp[a] -= S->P.u_in * (double)t;
    u[0] = u[1] = u[2] = 0.0;
    u[a] = S->P.u_in;
    for (int m = 0; m < S->P.n_modes; ++m) {
        const double* md = S->modes + 9 * m;
        double ph = md[0] * xp[0] + md[1] * xp[1] + md[2] * xp[2];
        double cph = cos(ph), sph = sin(ph);
        for (int k = 0; k < 3; ++k) u[k] += md[3 + k] * cph + md[6 + k] * sph;
    }
}

static void cell_velocity(const or_state* S, size_t x, double u[3], double* rho_out)
{
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < S->L.q; ++i) {
        double fi = S->f[(size_t)i * S->N + x];
        rho += fi;
        for (int k = 0; k < 3; ++k) j[k] += S->L.c[i][k] * fi;
    }
    for (int k = 0; k < 3; ++k) u[k] = j[k] / rho;
    if (rho_out) *rho_out = rho;
}

/* ---- step parts in the order of the listing "HHRRLBM-FSI" ---- */

static void update_porosity(or_state* S)
{
    const or_params* P = &S->P;
    /* BF: frames of the rotor's pitch; BD: frames that decide the cell sets
       (the same unless the sets are frozen for a finite-difference check) */
    blade_frames BF[OR_MAXROT], BD[OR_MAXROT];
    for (int k = 0; k < S->nrot; ++k) {
        const double th = rotor_angle(&S->rot[k], S->step);
        blade_frames_theta(&S->rot[k].r, th, &BF[k]);
        or_rotor rd = S->rot[k].r;
        if (S->frozen) rd.pitch = S->decision_pitch[k];
        blade_frames_theta(&rd, th, &BD[k]);
    }
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                float best = INFINITY;
                int tag = -1, which = -1;
                for (int k = 0; k < S->nrot; ++k) {
                    int w;
                    float v = rotor_phi_f32(&S->rot[k].r, &BD[k], x, y, z, &w);
                    if (v < best) { best = v; tag = k; which = w; }
                }
                S->phi[o] = best;
                float half = (float)(0.5 * P->eps_h);
                unsigned char fl = 0;
                if (best < half) fl |= FL_B;
                if (best >= 0.0f && best < half) fl |= FL_W;
                S->flags[o] = fl;
                S->tag[o] = (fl & FL_B) ? (signed char)tag : -1;
                S->which[o] = (fl & FL_B) ? (signed char)which : -1;
                float val = best;
                if (S->frozen && (fl & FL_B)) val = component_phi_f32(&S->rot[tag].r, &BF[tag], which, x, y, z);
                S->d[o] = (fl & FL_B) ? porosity_of_phi((double)val, P->eps_h, P->transition) : 1.0;
                if (fl & FL_W) {
                    double n[3];
                    rotor_normal(&S->rot[tag].r, &BF[tag], which, x, y, z, n);
                    double y1 = (double)val > 0.5 ? (double)val : 0.5;
                    for (int k = 0; k < 3; ++k) { S->nrm[3 * o + k] = n[k]; S->y1[3 * o + k] = y1 * n[k]; }
                }
            }
}

/* Wall model on W (Sec. 2.2.1, 3.2) from the current (pre-collision) populations. */
static void wall_model(or_state* S)
{
    const or_params* P = &S->P;
    double nu = (P->tau_mo - 0.5) * CS2;
    int dims[3] = {P->nx, P->ny, P->nz};
    long iters_total = 0, evals = 0;
    #pragma omp parallel for schedule(static) reduction(+:iters_total, evals)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                double* du = S->wm_du + 3 * o;
                double* Sm = S->wm_S + 9 * o;
                if (!(P->wall_model && (S->flags[o] & FL_W))) {
                    du[0] = du[1] = du[2] = 0.0;
                    for (int k = 0; k < 9; ++k) Sm[k] = 0.0;
                    S->wm_active[o] = 0;
                    S->wm_ut[o] = 0.0;
                    continue;
                }
                const double* n = S->nrm + 3 * o;
                const double* y1v = S->y1 + 3 * o;
                double y1 = sqrt(y1v[0] * y1v[0] + y1v[1] * y1v[1] + y1v[2] * y1v[2]);
                /* sampling point x_s = x + y_s n; trilinear fluid velocity there */
                double xs[3] = {x + P->wm_ysample * n[0], y + P->wm_ysample * n[1], z + P->wm_ysample * n[2]};
                int i0[3];
                double t[3];
                for (int k = 0; k < 3; ++k) {
                    double fl = floor(xs[k]);
                    i0[k] = (int)fl;
                    t[k] = xs[k] - fl;
                    if (P->open_boundaries && k == P->flow_axis) {
                        if (i0[k] < 0) { i0[k] = 0; t[k] = 0.0; }
                        if (i0[k] > dims[k] - 2) { i0[k] = dims[k] - 2; t[k] = 1.0; }
                    }
                }
                double us_[3] = {0, 0, 0};
                for (int cz = 0; cz < 2; ++cz)
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            int p[3] = {i0[0] + cx, i0[1] + cy, i0[2] + cz};
                            for (int k = 0; k < 3; ++k)
                                if (!(P->open_boundaries && k == P->flow_axis)) p[k] = wrap(p[k], dims[k]);
                            double wgt = (cx ? t[0] : 1 - t[0]) * (cy ? t[1] : 1 - t[1]) * (cz ? t[2] : 1 - t[2]);
                            double uc[3];
                            cell_velocity(S, cidx(S, p[0], p[1], p[2]), uc, NULL);
                            for (int k = 0; k < 3; ++k) us_[k] += wgt * uc[k];
                        }
                double usol[3];
                solid_velocity(&S->rot[S->tag[o]].r, x, y, z, usol);
                double ur[3] = {us_[0] - usol[0], us_[1] - usol[1], us_[2] - usol[2]};
                double un = ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2];
                double ut[3] = {ur[0] - un * n[0], ur[1] - un * n[1], ur[2] - un * n[2]};
                double utm = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
                if (utm < 1e-12) {
                    du[0] = du[1] = du[2] = 0.0;
                    for (int k = 0; k < 9; ++k) Sm[k] = 0.0;
                    S->wm_active[o] = 0;
                    S->wm_ut[o] = 0.0;
                    continue;
                }
                double th[3] = {ut[0] / utm, ut[1] / utm, ut[2] / utm};
                double ysamp = y1 + P->wm_ysample;
                /* Eq. (guess) */
                double guess = S->wm_active[o] ? S->wm_ut[o] : sqrt(nu * utm / P->wm_ysample);
                int its = 0;
                double utau = wf_newton(utm, ysamp, nu, guess, P->wm_E, P->wm_kappa, P->wm_tol, P->wm_maxit, &its);
                iters_total += its;
                evals += 1;
                double y1p = y1 * utau / nu;
                double up = spalding_uplus(y1p, P->wm_E, P->wm_kappa, P->wm_tol, P->wm_maxit);
                double uwall = utau * up;
                for (int k = 0; k < 3; ++k) du[k] = uwall * th[k];
                double g = (utm - uwall) / P->wm_ysample;
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) Sm[3 * p + q] = 0.5 * g * (th[p] * n[q] + n[p] * th[q]);
                S->wm_active[o] = 1;
                S->wm_ut[o] = utau;
            }
    S->wm_newton_iters += iters_total;
    S->wm_evals += evals;
}

/* Band parameters of interior cell o at (x, y, z) for this step's collision:
   d = d0 d_rotor (d0 = static multiplier, 1 unless set), u^B = u_s + du_WM,
   sigma, S^FD (Sec. 2.2, 2.2.1; d_rotor = 1 and u^B = 0 outside the force set). */
/* Finite-difference rate of strain of the fluid velocity at (x, y, z):
   S = (grad u + grad u^T) / 2 with central differences of u = j / rho of the
   pre-collision populations of the six axis neighbours (one-sided where a
   neighbour lies across an open face); the non-local strain of the hybrid
   non-equilibrium part (Sec. 2.2, f^(1,FD)). */
static void fd_strain(const or_state* S, int x, int y, int z, double Sfd[3][3])
{
    const int xi[3] = {x, y, z};
    double u0[3];
    cell_velocity(S, cidx(S, x, y, z), u0, NULL);
    double g[3][3];
    for (int a = 0; a < 3; ++a) {
        int e[3] = {0, 0, 0};
        e[a] = 1;
        int xp[3], xm[3];
        const int okp = neighbour(S, xi, e, +1, xp), okm = neighbour(S, xi, e, -1, xm);
        double up[3], um[3];
        if (okp) cell_velocity(S, cidx(S, xp[0], xp[1], xp[2]), up, NULL);
        else for (int b = 0; b < 3; ++b) up[b] = u0[b];
        if (okm) cell_velocity(S, cidx(S, xm[0], xm[1], xm[2]), um, NULL);
        else for (int b = 0; b < 3; ++b) um[b] = u0[b];
        const double h = (okp && okm) ? 2.0 : 1.0;
        for (int b = 0; b < 3; ++b) g[a][b] = (up[b] - um[b]) / h;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Sfd[a][b] = 0.5 * (g[a][b] + g[b][a]);
}

static void band_of_cell(const or_state* S, size_t o, int x, int y, int z, cell_band* B)
{
    const or_params* P = &S->P;
    memset(B, 0, sizeof *B);
    const double d0 = S->d0 ? S->d0[o] : 1.0;
    B->d = d0;
    B->sigma = 1.0;
    if (S->flags[o] & FL_B) {
        const or_rotor* R = &S->rot[S->tag[o]].r;
        B->d = d0 * S->d[o];
        solid_velocity(R, x, y, z, B->uB);
        B->sigma = P->sigma_band;
        if (P->wall_model && (S->flags[o] & FL_W)) {
            for (int k = 0; k < 3; ++k) B->uB[k] += S->wm_du[3 * o + k];
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) B->Sfd[p][q] = S->wm_S[9 * o + 3 * p + q];
            B->sigma = 0.0;
        } else if (P->sigma_band < 1.0) {
            fd_strain(S, x, y, z, B->Sfd);
        }
    }
}

static void collide_all(or_state* S)
{
    const or_params* P = &S->P;
    const or_lattice* L = &S->L;
    int a = P->flow_axis;
    int dims[3] = {P->nx, P->ny, P->nz};
    int cur = (int)(S->step & 1), prev = cur ^ 1;
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                int xi[3] = {x, y, z};
                int b = (a + 1) % 3, c = (a + 2) % 3;
                size_t pl = (size_t)xi[c] * dims[b] + xi[b];
                double fin[OR_MAXQ], fout[OR_MAXQ];
                if (P->open_boundaries && xi[a] == 0) {
                    double u[3];
                    inflow_velocity(S, x, y, z, S->step, u);
                    equilibrium(L, 1.0, u, fout);
                } else if (P->open_boundaries && xi[a] == dims[a] - 1) {
                    equilibrium(L, 1.0, S->uplane[prev] + 3 * pl, fout);
                } else {
                    for (int i = 0; i < L->q; ++i) fin[i] = S->f[(size_t)i * S->N + o];
                    cell_band B;
                    band_of_cell(S, o, x, y, z, &B);
                    double u[3];
                    collide(L, fin, &B, P->tau_mo, P->c_smag, fout, u);
                    if (P->open_boundaries && xi[a] == dims[a] - 2)
                        for (int k = 0; k < 3; ++k) S->uplane[cur][3 * pl + k] = u[k];
                }
                for (int i = 0; i < L->q; ++i) S->fpost[(size_t)i * S->N + o] = fout[i];
            }
}

/* Momentum exchange on post-collision populations over B = {d < 1}, per tag. */
static void boundary_force(or_state* S)
{
    const or_lattice* L = &S->L;
    const or_params* P = &S->P;
    for (int k = 0; k < S->nrot; ++k)
        for (int a = 0; a < 3; ++a) S->F[k][a] = S->M[k][a] = 0.0;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                if (!(S->flags[o] & FL_B)) continue;
                int tg = S->tag[o];
                const or_rotor* R = &S->rot[tg].r;
                double us[3];
                solid_velocity(R, x, y, z, us);
                double Fc[3] = {0, 0, 0};
                int xi[3] = {x, y, z};
                for (int i = 1; i < L->q; ++i) {
                    int nb[3];
                    if (!neighbour(S, xi, L->c[i], +1, nb)) continue;
                    size_t on = cidx(S, nb[0], nb[1], nb[2]);
                    int ib = L->opp[i];
                    for (int a = 0; a < 3; ++a) {
                        if (P->force_form == 0)
                            Fc[a] += (L->c[ib][a] - us[a]) * S->fpost[(size_t)ib * S->N + on]
                                   - (L->c[i][a] - us[a]) * S->fpost[(size_t)i * S->N + o];
                        else
                            Fc[a] += (L->c[i][a] - us[a]) * S->fpost[(size_t)i * S->N + on]
                                   + (L->c[i][a] + us[a]) * S->fpost[(size_t)i * S->N + o];
                    }
                }
                double r[3] = {x - R->center[0], y - R->center[1], z - R->center[2]};
                for (int a = 0; a < 3; ++a) S->F[tg][a] += Fc[a];
                S->M[tg][0] += r[1] * Fc[2] - r[2] * Fc[1];
                S->M[tg][1] += r[2] * Fc[0] - r[0] * Fc[2];
                S->M[tg][2] += r[0] * Fc[1] - r[1] * Fc[0];
            }
}

/* Pull streaming f_i(x, t+1) = f*_i(x - c_i); populations entering through an
   open face are not defined by the scheme (the boundary cell overwrites them
   with an equilibrium) and are filled with the cell's own post-collision value. */
static void stream_all(or_state* S)
{
    const or_lattice* L = &S->L;
    const or_params* P = &S->P;
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                int xi[3] = {x, y, z};
                for (int i = 0; i < L->q; ++i) {
                    int nb[3];
                    size_t src = o;
                    if (neighbour(S, xi, L->c[i], -1, nb)) src = cidx(S, nb[0], nb[1], nb[2]);
                    S->f[(size_t)i * S->N + o] = S->fpost[(size_t)i * S->N + src];
                }
            }
}

/* ------------------------------------------------------------------ */
/* exported API (ctypes)                                               */
/* ------------------------------------------------------------------ */

void or_destroy(or_state* S);

or_state* or_create(const or_params* P, const or_rotor* rotors, int nrot)
{
    if (!P || P->nx < 2 || P->ny < 2 || P->nz < 2 || nrot < 0 || nrot > OR_MAXROT) return NULL;
    if (P->flow_axis < 0 || P->flow_axis > 2) return NULL;
    or_state* S = (or_state*)calloc(1, sizeof(or_state));
    if (!S) return NULL;
    S->P = *P;
    if (lattice_init(&S->L, P->q)) { free(S); return NULL; }
    if (P->n_modes > 0) {
        S->modes = (double*)malloc(sizeof(double) * 9 * P->n_modes);
        memcpy(S->modes, P->modes, sizeof(double) * 9 * P->n_modes);
    }
    S->P.modes = S->modes;
    S->nrot = nrot;
    for (int k = 0; k < nrot; ++k) {
        S->rot[k].r = rotors[k];
        if (rotors[k].n_blades < 0 || rotors[k].n_blades > 8 || rotors[k].axis < 0 || rotors[k].axis > 2) {
            or_destroy(S);
            return NULL;
        }
        size_t ng = (size_t)rotors[k].gx * rotors[k].gy * rotors[k].gz;
        S->rot[k].sdf = (float*)malloc(sizeof(float) * (ng ? ng : 1));
        if (ng) memcpy(S->rot[k].sdf, rotors[k].sdf, sizeof(float) * ng);
        S->rot[k].r.sdf = S->rot[k].sdf;
    }
    size_t N = (size_t)P->nx * P->ny * P->nz;
    S->N = N;
    int q = P->q;
    S->f = (double*)malloc(sizeof(double) * q * N);
    S->fpost = (double*)malloc(sizeof(double) * q * N);
    S->phi = (float*)malloc(sizeof(float) * N);
    S->d = (double*)malloc(sizeof(double) * N);
    S->tag = (signed char*)malloc(N);
    S->which = (signed char*)malloc(N);
    S->flags = (unsigned char*)calloc(N, 1);
    S->nrm = (double*)calloc(3 * N, sizeof(double));
    S->y1 = (double*)calloc(3 * N, sizeof(double));
    S->wm_du = (double*)calloc(3 * N, sizeof(double));
    S->wm_S = (double*)calloc(9 * N, sizeof(double));
    S->wm_ut = (double*)calloc(N, sizeof(double));
    S->wm_active = (unsigned char*)calloc(N, 1);
    int dims[3] = {P->nx, P->ny, P->nz};
    int a = P->flow_axis;
    size_t npl = (size_t)dims[(a + 1) % 3] * dims[(a + 2) % 3];
    S->uplane[0] = (double*)malloc(sizeof(double) * 3 * npl);
    S->uplane[1] = (double*)malloc(sizeof(double) * 3 * npl);
    if (!S->f || !S->fpost || !S->phi || !S->d || !S->tag || !S->which || !S->flags || !S->nrm || !S->y1 ||
        !S->wm_du || !S->wm_S || !S->wm_ut || !S->wm_active || !S->uplane[0] || !S->uplane[1]) {
        or_destroy(S);
        return NULL;
    }
    /* initial state: f = f^eq(1, U a) everywhere, outlet plane velocity U a */
    double u0[3] = {0, 0, 0};
    u0[a] = P->u_in;
    double feq[OR_MAXQ];
    equilibrium(&S->L, 1.0, u0, feq);
    for (int i = 0; i < q; ++i)
        for (size_t x = 0; x < N; ++x) S->f[(size_t)i * N + x] = feq[i];
    for (size_t p = 0; p < npl; ++p)
        for (int k = 0; k < 3; ++k) S->uplane[0][3 * p + k] = S->uplane[1][3 * p + k] = u0[k];
    return S;
}

void or_destroy(or_state* S)
{
    if (!S) return;
    for (int k = 0; k < S->nrot; ++k) free(S->rot[k].sdf);
    free(S->modes); free(S->f); free(S->fpost); free(S->phi); free(S->d); free(S->tag); free(S->which); free(S->flags);
    free(S->nrm); free(S->y1); free(S->wm_du); free(S->wm_S); free(S->wm_ut); free(S->wm_active);
    free(S->uplane[0]); free(S->uplane[1]);
    free(S->d0);
    free(S);
}

/* Evolve structure (listing "HHRRLBM-FSI") for torque-driven rotors: rigid
   rotation about the rotor axis, I dOmega/dt = Q_aero - Q_gen(Omega), with the
   aerodynamic torque Q_aero = M . a of this step's momentum exchange and the
   generator torque Q_gen = q_gen0 + k_gen Omega |Omega|; explicit Euler with
   dt = 1: theta += Omega, then Omega += (Q_aero - Q_gen(Omega)) / I. */
static void evolve_structure(or_state* S)
{
    for (int k = 0; k < S->nrot; ++k) {
        rotor_store* rs = &S->rot[k];
        if (!rs->driven) continue;
        const double om = rs->r.omega;
        const double q_aero = S->M[k][rs->r.axis];
        const double q_gen = rs->q_gen0 + rs->k_gen * om * fabs(om);
        rs->theta += om;
        rs->r.omega = om + (q_aero - q_gen) / rs->inertia;
    }
}

/* One time step, in the order of the listing "HHRRLBM-FSI": porosity update
   (kinematics theta = theta0 + Omega t), wall model, collide, boundary force,
   stream, time averages; then t += 1 (evolve structure). */
void or_step(or_state* S, int n)
{
    for (int s = 0; s < n; ++s) {
        update_porosity(S);
        wall_model(S);
        collide_all(S);
        boundary_force(S);
        stream_all(S);
        for (int k = 0; k < S->nrot; ++k)
            for (int a = 0; a < 3; ++a) { S->Fsum[k][a] += S->F[k][a]; S->Msum[k][a] += S->M[k][a]; }
        evolve_structure(S);
        S->navg += 1;
        S->step += 1;
    }
}

long or_time(const or_state* S) { return S->step; }

void or_get_populations(const or_state* S, double* out)
{
    memcpy(out, S->f, sizeof(double) * S->L.q * S->N);
}

void or_set_populations(or_state* S, const double* in)
{
    memcpy(S->f, in, sizeof(double) * S->L.q * S->N);
}

/* f = f^eq(rho, u) per cell; rho[N], u[3][N] */
void or_init_equilibrium(or_state* S, const double* rho, const double* u)
{
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < (long)S->N; ++x) {
        double uu[3] = {u[x], u[S->N + x], u[2 * S->N + x]};
        double feq[OR_MAXQ];
        equilibrium(&S->L, rho[x], uu, feq);
        for (int i = 0; i < S->L.q; ++i) S->f[(size_t)i * S->N + x] = feq[i];
    }
}

/* density rho[N] and velocity u[3][N] of the current populations */
void or_fields(const or_state* S, double* rho, double* u)
{
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < (long)S->N; ++x) {
        double uu[3], r;
        cell_velocity(S, (size_t)x, uu, &r);
        rho[x] = r;
        for (int k = 0; k < 3; ++k) u[(size_t)k * S->N + x] = uu[k];
    }
}

/* per-rotor force and torque of the last step, and their running means */
void or_forces(const or_state* S, double* F, double* M, double* Favg, double* Mavg)
{
    for (int k = 0; k < S->nrot; ++k)
        for (int a = 0; a < 3; ++a) {
            if (F) F[3 * k + a] = S->F[k][a];
            if (M) M[3 * k + a] = S->M[k][a];
            if (Favg) Favg[3 * k + a] = S->navg ? S->Fsum[k][a] / S->navg : 0.0;
            if (Mavg) Mavg[3 * k + a] = S->navg ? S->Msum[k][a] / S->navg : 0.0;
        }
}

void or_reset_average(or_state* S)
{
    memset(S->Fsum, 0, sizeof S->Fsum);
    memset(S->Msum, 0, sizeof S->Msum);
    S->navg = 0;
}

/* total mass sum_x sum_i f_i, with Neumaier's compensated summation so that
   the rounding of the 19N-term sum stays below the invariants it checks */
double or_mass(const or_state* S)
{
    double s = 0.0, comp = 0.0;
    for (size_t k = 0; k < (size_t)S->L.q * S->N; ++k) {
        double v = S->f[k], t = s + v;
        comp += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    return s + comp;
}

/* geometry of the last porosity update: phi (binary32), d, flags, tag */
void or_geometry(const or_state* S, float* phi, double* d, unsigned char* flags, signed char* tag)
{
    if (phi) memcpy(phi, S->phi, sizeof(float) * S->N);
    if (d) memcpy(d, S->d, sizeof(double) * S->N);
    if (flags) memcpy(flags, S->flags, S->N);
    if (tag) memcpy(tag, S->tag, S->N);
}

/* wall-model state of the last evaluation: du[N][3], S[N][9], u_tau[N], active[N], y1[N][3] */
void or_wall_state(const or_state* S, double* du, double* Sm, double* ut, unsigned char* active, double* y1)
{
    if (du) memcpy(du, S->wm_du, sizeof(double) * 3 * S->N);
    if (Sm) memcpy(Sm, S->wm_S, sizeof(double) * 9 * S->N);
    if (ut) memcpy(ut, S->wm_ut, sizeof(double) * S->N);
    if (active) memcpy(active, S->wm_active, S->N);
    if (y1) memcpy(y1, S->y1, sizeof(double) * 3 * S->N);
}

void or_newton_stats(const or_state* S, long* iters, long* evals)
{
    *iters = S->wm_newton_iters;
    *evals = S->wm_evals;
}

/* inflow velocity of the inlet plane at time t: out[n_c][n_b][3] (b = axis+1, c = axis+2) */
void or_inflow_plane(const or_state* S, long t, double* out)
{
    int a = S->P.flow_axis, b = (a + 1) % 3, c = (a + 2) % 3;
    int dims[3] = {S->P.nx, S->P.ny, S->P.nz};
    for (int ic = 0; ic < dims[c]; ++ic)
        for (int ib = 0; ib < dims[b]; ++ib) {
            int xi[3];
            xi[a] = 0; xi[b] = ib; xi[c] = ic;
            inflow_velocity(S, xi[0], xi[1], xi[2], t, out + 3 * ((size_t)ic * dims[b] + ib));
        }
}

/* ---- single-cell entry points for unit checks ---- */

int or_lattice_table(int q, int* c, double* w, int* opp)
{
    or_lattice L;
    if (lattice_init(&L, q)) return -1;
    for (int i = 0; i < q; ++i) {
        for (int k = 0; k < 3; ++k) c[3 * i + k] = L.c[i][k];
        w[i] = L.w[i];
        if (opp) opp[i] = L.opp[i];
    }
    return 0;
}

int or_equilibrium(int q, double rho, const double* u, double* feq)
{
    or_lattice L;
    if (lattice_init(&L, q)) return -1;
    equilibrium(&L, rho, u, feq);
    return 0;
}

int or_regularized_neq(int q, const double* a2, const double* u, double* f1)
{
    or_lattice L;
    if (lattice_init(&L, q)) return -1;
    double A[3][3];
    for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) A[p][r] = a2[3 * p + r];
    regularized_neq(&L, A, u, f1);
    return 0;
}

double or_smagorinsky_tau(double tau_mo, double c_smag, double rho, const double* Pneq)
{
    double A[3][3];
    for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) A[p][r] = Pneq[3 * p + r];
    return smagorinsky_tau(tau_mo, c_smag, rho, A);
}

/* n cells: f[n][q] in, band data d[n], uB[n][3], sigma[n], Sfd[n][9]; fout[n][q], tau[n] */
int or_collide_cells(int q, int n, const double* f, const double* d, const double* uB,
                     const double* sigma, const double* Sfd, double tau_mo, double c_smag,
                     double* fout, double* tau)
{
    or_lattice L;
    if (lattice_init(&L, q)) return -1;
    for (int c = 0; c < n; ++c) {
        cell_band B;
        B.d = d ? d[c] : 1.0;
        for (int k = 0; k < 3; ++k) B.uB[k] = uB ? uB[3 * c + k] : 0.0;
        B.sigma = sigma ? sigma[c] : 1.0;
        for (int p = 0; p < 3; ++p)
            for (int r = 0; r < 3; ++r) B.Sfd[p][r] = Sfd ? Sfd[9 * c + 3 * p + r] : 0.0;
        double t = collide(&L, f + (size_t)q * c, &B, tau_mo, c_smag, fout + (size_t)q * c, NULL);
        if (tau) tau[c] = t;
    }
    return 0;
}

double or_spalding_yplus(double up, double E, double kappa) { return spalding_yplus(up, E, kappa); }

double or_spalding_uplus(double yp, double E, double kappa, double tol, int maxit)
{
    return spalding_uplus(yp, E, kappa, tol, maxit);
}

double or_wall_newton(double u, double y, double nu, double guess, double E, double kappa,
                      double tol, int maxit, int* iters)
{
    return wf_newton(u, y, nu, guess, E, kappa, tol, maxit, iters);
}

double or_porosity(double phi, double eps, int linear) { return porosity_of_phi(phi, eps, linear); }

/* binary32 signed distance of n cells (xyz[n][3]) to a rotor at time t */
void or_rotor_phi(const or_rotor* R, long t, int n, const int* xyz, float* phi, int* which)
{
    blade_frames B;
    blade_frames_at(R, t, &B);
    for (int c = 0; c < n; ++c)
        phi[c] = rotor_phi_f32(R, &B, xyz[3 * c], xyz[3 * c + 1], xyz[3 * c + 2], which ? which + c : NULL);
}

void or_rotor_normal(const or_rotor* R, long t, int which, int x, int y, int z, double* n)
{
    blade_frames B;
    blade_frames_at(R, t, &B);
    rotor_normal(R, &B, which, x, y, z, n);
}

size_t or_sizeof_params(void) { return sizeof(or_params); }
size_t or_sizeof_rotor(void) { return sizeof(or_rotor); }

/* ================================================================== */
/* Discrete adjoint of the time step (FP64).                          */
/*                                                                    */
/* J = (1/n_avg) sum over the last n_avg steps of                     */
/*     sum_k [ wT_k F_k(t).a_k + wQ_k M_k(t).a_k ]                    */
/* differentiated with respect to each rotor's pitch and the static    */
/* porosity multiplier d0 (d_eff = d0 d, d0 = 1 by default), with the  */
/* cell sets (force cells, wall cells) frozen at their forward values. */
/* Every local Jacobian is taken by complex-step differentiation       */
/* (f(x + i h) = f(x) + i h f'(x) + O(h^2), h = 1e-30): derivatives to */
/* rounding, with no hand-derived formula; the two wall-model Newton   */
/* solves are differentiated through the iterations they take (complex */
/* step through the iterates, stopping rule and guard included).  The  */
/* finite-difference strain of the sigma < 1 band is transposed by     */
/* hand (it is linear in the neighbours' velocities), with            */
/* du/df_i = (c_i - u) / rho.                                          */
/* ================================================================== */

typedef double complex cplx;
static const double CSTEP = 1e-30;

static void equilibrium_c(const or_lattice* L, cplx rho, const cplx u[3], cplx* feq)
{
    cplx A2[3][3], A3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            A2[a][b] = rho * u[a] * u[b];
            for (int g = 0; g < 3; ++g) A3[a][b][g] = rho * u[a] * u[b] * u[g];
        }
    for (int i = 0; i < L->q; ++i) {
        cplx cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        cplx c2 = 0, c3 = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                c2 += L->H2[i][a][b] * A2[a][b];
                for (int g = 0; g < 3; ++g) c3 += L->H3[i][a][b][g] * A3[a][b][g];
            }
        feq[i] = L->w[i] * (rho + rho * cu / CS2 + c2 / (2.0 * CS2 * CS2) + c3 / (6.0 * CS2 * CS2 * CS2));
    }
}

/* complex twin of collide(): same formulas, complex band parameters */
typedef struct { cplx d, uB[3], sigma, Sfd[3][3]; } cell_band_c;

static void collide_c(const or_lattice* L, const cplx* f, const cell_band_c* B, double tau_mo, double c_smag,
                      cplx* fout)
{
    cplx rho = 0, j[3] = {0, 0, 0}, Pi[3][3] = {{0}};
    for (int i = 0; i < L->q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += L->c[i][a] * f[i];
            for (int b = 0; b < 3; ++b) Pi[a][b] += L->c[i][a] * L->c[i][b] * f[i];
        }
    }
    cplx u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    cplx Pneq[3][3], Q = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Pneq[a][b] = Pi[a][b] - rho * CS2 * delta(a, b) - rho * u[a] * u[b];
            Q += Pneq[a][b] * Pneq[a][b];
        }
    cplx tau = 0.5 * (tau_mo + csqrt(tau_mo * tau_mo + 18.0 * sqrt(2.0) * c_smag * c_smag * csqrt(Q) / rho));
    cplx uh[3];
    for (int a = 0; a < 3; ++a) uh[a] = B->d * u[a] + (1.0 - B->d) * B->uB[a];
    cplx feq[OR_MAXQ];
    equilibrium_c(L, rho, uh, feq);
    cplx a3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int g = 0; g < 3; ++g) a3[a][b][g] = uh[a] * Pneq[b][g] + uh[b] * Pneq[a][g] + uh[g] * Pneq[a][b];
    for (int i = 0; i < L->q; ++i) {
        cplx h2 = 0, h3 = 0, hs = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                h2 += L->H2[i][a][b] * Pneq[a][b];
                hs += L->H2[i][a][b] * B->Sfd[a][b];
                for (int g = 0; g < 3; ++g) h3 += L->H3[i][a][b][g] * a3[a][b][g];
            }
        cplx f1 = L->w[i] * (h2 / (2.0 * CS2 * CS2) + h3 / (6.0 * CS2 * CS2 * CS2));
        cplx f1fd = L->w[i] * rho * tau / CS2 * hs;
        fout[i] = feq[i] + (1.0 - 1.0 / tau) * (B->sigma * f1 - (1.0 - B->sigma) * f1fd);
    }
}

/* Vector-Jacobian product of one collision: given the adjoint lam_star of
   the post-collision populations, the adjoint of the pre-collision
   populations and of the band parameters d, u^B, S (S as a full 3x3). */
static void collide_vjp(const or_lattice* L, const double* f, const cell_band* B, double tau_mo, double c_smag,
                        const double* lam_star, double* lam_f, double* g_d, double g_uB[3], double g_S[3][3])
{
    cplx fc[OR_MAXQ] = {0}, out[OR_MAXQ];
    cell_band_c Bc;
    Bc.d = B->d;
    Bc.sigma = B->sigma;
    for (int a = 0; a < 3; ++a) {
        Bc.uB[a] = B->uB[a];
        for (int b = 0; b < 3; ++b) Bc.Sfd[a][b] = B->Sfd[a][b];
    }
    for (int i = 0; i < L->q; ++i) fc[i] = f[i];
    for (int jdir = 0; jdir < L->q; ++jdir) {
        fc[jdir] += I * CSTEP;
        collide_c(L, fc, &Bc, tau_mo, c_smag, out);
        fc[jdir] = f[jdir];
        double s = 0.0;
        for (int i = 0; i < L->q; ++i) s += lam_star[i] * cimag(out[i]) / CSTEP;
        lam_f[jdir] = s;
    }
    if (g_d) {
        Bc.d += I * CSTEP;
        collide_c(L, fc, &Bc, tau_mo, c_smag, out);
        Bc.d = B->d;
        double s = 0.0;
        for (int i = 0; i < L->q; ++i) s += lam_star[i] * cimag(out[i]) / CSTEP;
        *g_d = s;
    }
    if (g_uB)
        for (int a = 0; a < 3; ++a) {
            Bc.uB[a] += I * CSTEP;
            collide_c(L, fc, &Bc, tau_mo, c_smag, out);
            Bc.uB[a] = B->uB[a];
            double s = 0.0;
            for (int i = 0; i < L->q; ++i) s += lam_star[i] * cimag(out[i]) / CSTEP;
            g_uB[a] = s;
        }
    if (g_S)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                Bc.Sfd[a][b] += I * CSTEP;
                collide_c(L, fc, &Bc, tau_mo, c_smag, out);
                Bc.Sfd[a][b] = B->Sfd[a][b];
                double s = 0.0;
                for (int i = 0; i < L->q; ++i) s += lam_star[i] * cimag(out[i]) / CSTEP;
                g_S[a][b] = s;
            }
}

/* n cells: as or_collide_cells, plus the adjoint lam_star[n][q] ->
   lam_f[n][q], g_d[n], g_uB[n][3], g_S[n][9] (any output may be NULL) */
int or_collide_vjp_cells(int q, int n, const double* f, const double* d, const double* uB, const double* sigma,
                         const double* Sfd, double tau_mo, double c_smag, const double* lam_star, double* lam_f,
                         double* g_d, double* g_uB, double* g_S)
{
    or_lattice L;
    if (lattice_init(&L, q)) return -1;
    #pragma omp parallel for schedule(static)
    for (int c = 0; c < n; ++c) {
        cell_band B;
        B.d = d ? d[c] : 1.0;
        for (int k = 0; k < 3; ++k) B.uB[k] = uB ? uB[3 * c + k] : 0.0;
        B.sigma = sigma ? sigma[c] : 1.0;
        for (int p = 0; p < 3; ++p)
            for (int r = 0; r < 3; ++r) B.Sfd[p][r] = Sfd ? Sfd[9 * c + 3 * p + r] : 0.0;
        double gd, gu[3], gS[3][3];
        collide_vjp(&L, f + (size_t)q * c, &B, tau_mo, c_smag, lam_star + (size_t)q * c, lam_f + (size_t)q * c,
                    &gd, gu, gS);
        if (g_d) g_d[c] = gd;
        for (int k = 0; k < 3; ++k)
            if (g_uB) g_uB[3 * c + k] = gu[k];
        for (int p = 0; p < 3; ++p)
            for (int r = 0; r < 3; ++r)
                if (g_S) g_S[9 * c + 3 * p + r] = gS[p][r];
    }
    return 0;
}

/* ---- setters used by gradient checks ---- */

/* Static porosity multiplier d0 [N] (copied; NULL restores d0 = 1). */
int or_set_d0(or_state* S, const double* d0)
{
    if (!d0) { free(S->d0); S->d0 = NULL; return 0; }
    if (!S->d0) S->d0 = (double*)malloc(sizeof(double) * S->N);
    if (!S->d0) return -1;
    memcpy(S->d0, d0, sizeof(double) * S->N);
    return 0;
}

int or_set_pitch(or_state* S, int k, double pitch)
{
    if (k < 0 || k >= S->nrot) return -1;
    S->rot[k].r.pitch = pitch;
    return 0;
}

/* on = 1: from now on the cell sets (force set, wall set, tag, component)
   follow the pitch each rotor has at this call, while porosity, normal and
   wall distance follow the current pitch (Sec. 3.1 quantities with the set
   memberships held fixed); on = 0: both follow the current pitch. */
void or_freeze_sets(or_state* S, int on)
{
    S->frozen = on ? 1 : 0;
    for (int k = 0; k < S->nrot; ++k) S->decision_pitch[k] = S->rot[k].r.pitch;
}

/* ---- complex twins of the geometry (pitch enters through cp, sp) ---- */

static cplx blade_sample_c(const or_rotor* R, cplx p0, cplx p1, cplx p2)
{
    double h = R->spacing;
    cplx g[3] = {(p0 - R->origin[0]) / h, (p1 - R->origin[1]) / h, (p2 - R->origin[2]) / h};
    double fl[3] = {floor(creal(g[0])), floor(creal(g[1])), floor(creal(g[2]))};
    if (!(fl[0] >= 0.0 && fl[0] <= R->gx - 2 && fl[1] >= 0.0 && fl[1] <= R->gy - 2 && fl[2] >= 0.0 &&
          fl[2] <= R->gz - 2))
        return INFINITY;
    int i0 = (int)fl[0], j0 = (int)fl[1], k0 = (int)fl[2];
    cplx t[3] = {g[0] - fl[0], g[1] - fl[1], g[2] - fl[2]};
    cplx v = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                cplx wgt = (cx ? t[0] : 1.0 - t[0]) * (cy ? t[1] : 1.0 - t[1]) * (cz ? t[2] : 1.0 - t[2]);
                size_t o = ((size_t)(k0 + cz) * R->gy + (size_t)(j0 + cy)) * R->gx + (size_t)(i0 + cx);
                v += wgt * (double)R->sdf[o];
            }
    return v;
}

/* phi of one component in FP64 with pitch frames (cp, sp) */
static cplx component_phi_c(const or_rotor* R, const blade_frames* B, int which, int ix, int iy, int iz,
                            cplx cp, cplx sp)
{
    int a = R->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    double rl[3] = {ix - R->center[0], iy - R->center[1], iz - R->center[2]};
    double rb = rl[b], rc = rl[c], ra = rl[a];
    if (which >= R->n_blades) return sqrt(rb * rb + rc * rc + ra * ra) - R->hub_radius;
    double ck = B->ckd[which], sk = B->skd[which];
    double pR = ck * rb + sk * rc, pT = ck * rc - sk * rb;
    cplx qT = cp * pT - sp * ra, qA = cp * ra + sp * pT;
    return blade_sample_c(R, pR, qT, qA);
}

static cplx porosity_c(cplx phi, double eps, int linear)
{
    double pr = creal(phi);
    if (pr <= -0.5 * eps) return 0.0;
    if (pr >= 0.5 * eps) return 1.0;
    cplx t = phi / eps + 0.5;
    return linear ? t : t * t * (3.0 - 2.0 * t);
}

/* complex twin of rotor_normal */
static void rotor_normal_c(const or_rotor* R, const blade_frames* B, int which, int ix, int iy, int iz, cplx cp,
                           cplx sp, cplx n_out[3])
{
    int a = R->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    double rl[3] = {ix - R->center[0], iy - R->center[1], iz - R->center[2]};
    cplx v[3];
    if (which >= R->n_blades) {
        v[0] = rl[0]; v[1] = rl[1]; v[2] = rl[2];
    } else {
        double rb = rl[b], rc = rl[c], ra = rl[a];
        double ck = B->ckd[which], sk = B->skd[which];
        double pR = ck * rb + sk * rc, pT = ck * rc - sk * rb;
        cplx qT = cp * pT - sp * ra, qA = cp * ra + sp * pT;
        double h = R->spacing;
        cplx g[3] = {(pR - R->origin[0]) / h, (qT - R->origin[1]) / h, (qA - R->origin[2]) / h};
        int i0 = (int)floor(creal(g[0])), j0 = (int)floor(creal(g[1])), k0 = (int)floor(creal(g[2]));
        if (i0 < 0) i0 = 0;
        if (i0 > R->gx - 2) i0 = R->gx - 2;
        if (j0 < 0) j0 = 0;
        if (j0 > R->gy - 2) j0 = R->gy - 2;
        if (k0 < 0) k0 = 0;
        if (k0 > R->gz - 2) k0 = R->gz - 2;
        cplx t[3] = {g[0] - i0, g[1] - j0, g[2] - k0};
        cplx gb[3] = {0, 0, 0};
        int dims[3] = {R->gx, R->gy, R->gz};
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    int node[3] = {i0 + cx, j0 + cy, k0 + cz};
                    cplx wgt = (cx ? t[0] : 1.0 - t[0]) * (cy ? t[1] : 1.0 - t[1]) * (cz ? t[2] : 1.0 - t[2]);
                    for (int d = 0; d < 3; ++d) {
                        int lo[3] = {node[0], node[1], node[2]}, hi[3] = {node[0], node[1], node[2]};
                        lo[d] = node[d] > 0 ? node[d] - 1 : node[d];
                        hi[d] = node[d] < dims[d] - 1 ? node[d] + 1 : node[d];
                        size_t olo = ((size_t)lo[2] * R->gy + lo[1]) * R->gx + lo[0];
                        size_t ohi = ((size_t)hi[2] * R->gy + hi[1]) * R->gx + hi[0];
                        double der = ((double)R->sdf[ohi] - (double)R->sdf[olo]) / ((hi[d] - lo[d]) * h);
                        gb[d] += wgt * der;
                    }
                }
        cplx vT = cp * gb[1] + sp * gb[2];
        cplx vA = -sp * gb[1] + cp * gb[2];
        cplx vR = gb[0];
        cplx lab[3];
        lab[b] = ck * vR - sk * vT;
        lab[c] = sk * vR + ck * vT;
        lab[a] = vA;
        v[0] = lab[0]; v[1] = lab[1]; v[2] = lab[2];
    }
    cplx nrm = csqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (creal(nrm) > 0.0) { n_out[0] = v[0] / nrm; n_out[1] = v[1] / nrm; n_out[2] = v[2] / nrm; }
    else { n_out[0] = n_out[1] = n_out[2] = 0.0; }
}

/* ---- complex twin of one wall-model cell ---- */

static cplx spalding_yplus_c(cplx up, double E, double kappa)
{
    cplx k = kappa * up;
    return up + (cexp(k) - 1.0 - k - 0.5 * k * k - k * k * k / 6.0) / E;
}

/* complex twins of the two Newton solves: the same iterations as
   wf_newton / spalding_uplus, every branch taken on the real part, so that
   the imaginary part carries the derivative of the iterate actually
   returned (a capped, unconverged solve included) */
static cplx wf_newton_c(cplx u, cplx y, double nu, cplx guess, double E, double kappa, double tol, int maxit)
{
    cplx ut = guess;
    cplx fv = spalding_yplus_c(u / ut, E, kappa) - y * ut / nu;
    int it = 0;
    while (it < maxit) {
        /* the step of wf_step: f/f' with both scaled by exp(-kappa u+) */
        cplx up = u / ut;
        cplx k = kappa * up;
        cplx sc = cexp(-k);
        cplx P2 = 1.0 + k + 0.5 * k * k, P3 = P2 + k * k * k / 6.0;
        cplx fs = (up - y * ut / nu) * sc + (1.0 - P3 * sc) / E;
        cplx fps = -(sc + kappa / E * (1.0 - P2 * sc)) * up / ut - y / nu * sc;
        cplx un = ut - fs / fps;
        if (!(creal(un) > 0.0)) un = 0.5 * ut;
        cplx fn = spalding_yplus_c(u / un, E, kappa) - y * un / nu;
        ut = un;
        ++it;
        if (fabs(creal(fn) - creal(fv)) < tol) break;
        fv = fn;
    }
    return ut;
}

static cplx spalding_uplus_c(cplx yp, double E, double kappa, double tol, int maxit)
{
    cplx lg = clog(1.0 + E * yp) / kappa;
    cplx up = creal(yp) < creal(lg) ? yp : lg;
    cplx g = spalding_yplus_c(up, E, kappa) - yp;
    for (int it = 0; it < maxit; ++it) {
        cplx k = kappa * up;
        cplx dyp = 1.0 + kappa / E * (cexp(k) - 1.0 - k - 0.5 * k * k);
        cplx un = up - g / dyp;
        if (!(creal(un) > 0.0)) un = 0.5 * up;
        cplx gn = spalding_yplus_c(un, E, kappa) - yp;
        up = un;
        if (fabs(creal(gn) - creal(g)) < tol) break;
        g = gn;
    }
    return up;
}

/* Outputs du[3], Sm[9] and u_tau of wall cell o at (x, y, z) as functions of
   the eight trilinear corner velocities uc[8][3], the geometry (n, y1) and
   the Newton start value (the previous step's u_tau when warm, else the
   estimate of Eq. (guess)).  Returns 0 for a cell the forward left inactive. */
static int wall_cell_c(const or_state* S, size_t o, int x, int y, int z, const cplx uc[8][3], const cplx n[3],
                       cplx y1, int warm, cplx guess_prev, cplx du[3], cplx Sm[9], cplx* utau_out)
{
    const or_params* P = &S->P;
    double nu = (P->tau_mo - 0.5) * CS2;
    int dims[3] = {P->nx, P->ny, P->nz};
    for (int k = 0; k < 3; ++k) du[k] = 0.0;
    for (int k = 0; k < 9; ++k) Sm[k] = 0.0;
    *utau_out = 0.0;
    if (!S->wm_active[o]) return 0;
    int xi[3] = {x, y, z};
    cplx t[3];
    for (int k = 0; k < 3; ++k) {
        cplx xs = xi[k] + P->wm_ysample * n[k];
        double fl = floor(creal(xs));
        int i0 = (int)fl;
        t[k] = xs - fl;
        if (P->open_boundaries && k == P->flow_axis) {
            if (i0 < 0) t[k] = 0.0;
            if (i0 > dims[k] - 2) t[k] = 1.0;
        }
    }
    cplx us_[3] = {0, 0, 0};
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                cplx wgt = (cx ? t[0] : 1.0 - t[0]) * (cy ? t[1] : 1.0 - t[1]) * (cz ? t[2] : 1.0 - t[2]);
                int m = (cz * 2 + cy) * 2 + cx;
                for (int k = 0; k < 3; ++k) us_[k] += wgt * uc[m][k];
            }
    double usol[3];
    solid_velocity(&S->rot[S->tag[o]].r, x, y, z, usol);
    cplx ur[3] = {us_[0] - usol[0], us_[1] - usol[1], us_[2] - usol[2]};
    cplx un = ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2];
    cplx ut[3] = {ur[0] - un * n[0], ur[1] - un * n[1], ur[2] - un * n[2]};
    cplx utm = csqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    cplx th[3] = {ut[0] / utm, ut[1] / utm, ut[2] / utm};
    cplx ysamp = y1 + P->wm_ysample;
    cplx guess = warm ? guess_prev : csqrt(nu * utm / P->wm_ysample);
    cplx utau = wf_newton_c(utm, ysamp, nu, guess, P->wm_E, P->wm_kappa, P->wm_tol, P->wm_maxit);
    cplx y1p = y1 * utau / nu;
    cplx up = spalding_uplus_c(y1p, P->wm_E, P->wm_kappa, P->wm_tol, P->wm_maxit);
    cplx uwall = utau * up;
    for (int k = 0; k < 3; ++k) du[k] = uwall * th[k];
    cplx g = (utm - uwall) / P->wm_ysample;
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) Sm[3 * p + q] = 0.5 * g * (th[p] * n[q] + n[p] * th[q]);
    *utau_out = utau;
    return 1;
}

/* corner cells of the wall-model sample of cell o (same clamping and
   wrapping as wall_model); returns the real trilinear setup in idx[8] */
static void wall_corners(const or_state* S, size_t o, int x, int y, int z, size_t idx[8])
{
    const or_params* P = &S->P;
    int dims[3] = {P->nx, P->ny, P->nz};
    const double* n = S->nrm + 3 * o;
    double xs[3] = {x + P->wm_ysample * n[0], y + P->wm_ysample * n[1], z + P->wm_ysample * n[2]};
    int i0[3];
    for (int k = 0; k < 3; ++k) {
        i0[k] = (int)floor(xs[k]);
        if (P->open_boundaries && k == P->flow_axis) {
            if (i0[k] < 0) i0[k] = 0;
            if (i0[k] > dims[k] - 2) i0[k] = dims[k] - 2;
        }
    }
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                int p[3] = {i0[0] + cx, i0[1] + cy, i0[2] + cz};
                for (int k = 0; k < 3; ++k)
                    if (!(P->open_boundaries && k == P->flow_axis)) p[k] = wrap(p[k], dims[k]);
                idx[(cz * 2 + cy) * 2 + cx] = cidx(S, p[0], p[1], p[2]);
            }
}

/* ---- the reverse sweep ---- */

typedef struct {
    double* f;          /* [T][q][N] pre-collision populations at the start of each step */
    double* wm_ut;      /* [T][N] */
    unsigned char* wm_active; /* [T][N] */
    double* uplane;     /* [T][2][3 npl] */
} or_tape;

/* J = (1/n_avg) sum_{t = T - n_avg}^{T-1} sum_k [ wT_k F_k(t).a_k + wQ_k M_k(t).a_k ]
   over the next T steps from the current state, and its gradient with
   respect to every rotor's pitch (dJdp[nrot]) and the static porosity
   multiplier (dJdd0[N]), cell sets frozen at their forward values (the
   reading for the non-smooth points of the step).  On return the state has
   advanced T steps, exactly as or_step(S, T).  The trajectory is kept in
   host memory: T (q + 1) N doubles. */
int or_adjoint(or_state* S, int T, int n_avg, const double* wT, const double* wQ, double* J_out, double* dJdp,
               double* dJdd0)
{
    const or_params* P = &S->P;
    const or_lattice* L = &S->L;
    const int q = L->q;
    const size_t N = S->N;
    int dims[3] = {P->nx, P->ny, P->nz};
    const int ax = P->flow_axis, bx = (ax + 1) % 3, cxx = (ax + 2) % 3;
    const size_t npl = (size_t)dims[bx] * dims[cxx];
    if (T < 1 || n_avg < 1 || n_avg > T) return -1;
    for (int k = 0; k < S->nrot; ++k)
        if (S->rot[k].driven) return -3;   /* gradients cover prescribed rotation only */
    or_tape tp;
    tp.f = (double*)malloc(sizeof(double) * (size_t)T * q * N);
    tp.wm_ut = (double*)malloc(sizeof(double) * (size_t)T * N);
    tp.wm_active = (unsigned char*)malloc((size_t)T * N);
    tp.uplane = (double*)malloc(sizeof(double) * (size_t)T * 6 * npl);
    double* lam = (double*)calloc((size_t)q * N, sizeof(double));
    double* lam_star = (double*)malloc(sizeof(double) * (size_t)q * N);
    double* lam_new = (double*)malloc(sizeof(double) * (size_t)q * N);
    double* g_up_cur = (double*)calloc(3 * npl, sizeof(double));   /* dJ/d uplane written in this step */
    double* g_up_prev = (double*)calloc(3 * npl, sizeof(double));  /* dJ/d uplane read in this step */
    double* g_uB = (double*)malloc(sizeof(double) * 3 * N);
    double* g_S = (double*)malloc(sizeof(double) * 9 * N);
    double* gp_cell = (double*)malloc(sizeof(double) * N);
    double* wm_ubar = (double*)malloc(sizeof(double) * 24 * N);
    double* wm_pbar = (double*)malloc(sizeof(double) * N);
    double* g_ut_cur = (double*)calloc(N, sizeof(double));   /* dJ/d u_tau of this step (next step's start) */
    double* g_ut_prev = (double*)calloc(N, sizeof(double));  /* dJ/d u_tau of the previous step */
    if (!tp.f || !tp.wm_ut || !tp.wm_active || !tp.uplane || !lam || !lam_star || !lam_new || !g_up_cur ||
        !g_up_prev || !g_uB || !g_S || !gp_cell || !wm_ubar || !wm_pbar || !g_ut_cur || !g_ut_prev) {
        free(tp.f); free(tp.wm_ut); free(tp.wm_active); free(tp.uplane); free(lam); free(lam_star);
        free(lam_new); free(g_up_cur); free(g_up_prev); free(g_uB); free(g_S); free(gp_cell); free(wm_ubar);
        free(wm_pbar); free(g_ut_cur); free(g_ut_prev);
        return -2;
    }
    const long t0 = S->step;
    /* forward, recording the state each step starts from */
    double J = 0.0;
    for (int s = 0; s < T; ++s) {
        memcpy(tp.f + (size_t)s * q * N, S->f, sizeof(double) * q * N);
        memcpy(tp.wm_ut + (size_t)s * N, S->wm_ut, sizeof(double) * N);
        memcpy(tp.wm_active + (size_t)s * N, S->wm_active, N);
        memcpy(tp.uplane + (size_t)s * 6 * npl, S->uplane[0], sizeof(double) * 3 * npl);
        memcpy(tp.uplane + (size_t)s * 6 * npl + 3 * npl, S->uplane[1], sizeof(double) * 3 * npl);
        or_step(S, 1);
        if (s >= T - n_avg)
            for (int k = 0; k < S->nrot; ++k) {
                int a = S->rot[k].r.axis;
                J += (wT[k] * S->F[k][a] + wQ[k] * S->M[k][a]) / n_avg;
            }
    }
    /* keep the final forward state to put back at the end */
    double* f_end = (double*)malloc(sizeof(double) * q * N);
    double* ut_end = (double*)malloc(sizeof(double) * N);
    unsigned char* act_end = (unsigned char*)malloc(N);
    double* up_end = (double*)malloc(sizeof(double) * 6 * npl);
    memcpy(f_end, S->f, sizeof(double) * q * N);
    memcpy(ut_end, S->wm_ut, sizeof(double) * N);
    memcpy(act_end, S->wm_active, N);
    memcpy(up_end, S->uplane[0], sizeof(double) * 3 * npl);
    memcpy(up_end + 3 * npl, S->uplane[1], sizeof(double) * 3 * npl);
    double Fk[OR_MAXROT][3], Mk[OR_MAXROT][3];
    memcpy(Fk, S->F, sizeof Fk);
    memcpy(Mk, S->M, sizeof Mk);
    long it_end = S->wm_newton_iters, ev_end = S->wm_evals, step_end = S->step;

    for (int k = 0; k < S->nrot; ++k) dJdp[k] = 0.0;
    for (size_t x = 0; x < N; ++x) dJdd0[x] = 0.0;

    for (int s = T - 1; s >= 0; --s) {
        /* recompute the forward quantities of step s */
        memcpy(S->f, tp.f + (size_t)s * q * N, sizeof(double) * q * N);
        memcpy(S->wm_ut, tp.wm_ut + (size_t)s * N, sizeof(double) * N);
        memcpy(S->wm_active, tp.wm_active + (size_t)s * N, N);
        memcpy(S->uplane[0], tp.uplane + (size_t)s * 6 * npl, sizeof(double) * 3 * npl);
        memcpy(S->uplane[1], tp.uplane + (size_t)s * 6 * npl + 3 * npl, sizeof(double) * 3 * npl);
        S->step = t0 + s;
        update_porosity(S);
        wall_model(S);

        /* adjoint of streaming: transpose of stream_all */
        for (size_t m = 0; m < (size_t)q * N; ++m) lam_star[m] = 0.0;
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x) {
                    size_t o = cidx(S, x, y, z);
                    int xi[3] = {x, y, z};
                    for (int i = 0; i < q; ++i) {
                        int nb[3];
                        size_t src = o;
                        if (neighbour(S, xi, L->c[i], -1, nb)) src = cidx(S, nb[0], nb[1], nb[2]);
                        lam_star[(size_t)i * N + src] += lam[(size_t)i * N + o];
                    }
                }
        /* adjoint of the force: transpose of boundary_force, weighted */
        if (s >= T - n_avg)
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        size_t o = cidx(S, x, y, z);
                        if (!(S->flags[o] & FL_B)) continue;
                        const or_rotor* R = &S->rot[S->tag[o]].r;
                        int k = S->tag[o], a = R->axis;
                        double us[3];
                        solid_velocity(R, x, y, z, us);
                        double r[3] = {x - R->center[0], y - R->center[1], z - R->center[2]};
                        /* J per step = wT F_a + wQ (r x F)_a = F . v,  v = wT e_a + wQ (e_a x r) */
                        double ea[3] = {0, 0, 0};
                        ea[a] = 1.0;
                        double v[3] = {wT[k] * ea[0] + wQ[k] * (ea[1] * r[2] - ea[2] * r[1]),
                                       wT[k] * ea[1] + wQ[k] * (ea[2] * r[0] - ea[0] * r[2]),
                                       wT[k] * ea[2] + wQ[k] * (ea[0] * r[1] - ea[1] * r[0])};
                        for (int m = 0; m < 3; ++m) v[m] /= n_avg;
                        int xi[3] = {x, y, z};
                        for (int i = 1; i < q; ++i) {
                            int nb[3];
                            if (!neighbour(S, xi, L->c[i], +1, nb)) continue;
                            size_t on = cidx(S, nb[0], nb[1], nb[2]);
                            int ib = L->opp[i];
                            double cib = 0.0, ci = 0.0, cip = 0.0;
                            for (int m = 0; m < 3; ++m) {
                                cib += (L->c[ib][m] - us[m]) * v[m];
                                ci += (L->c[i][m] - us[m]) * v[m];
                                cip += (L->c[i][m] + us[m]) * v[m];
                            }
                            if (P->force_form == 0) {
                                lam_star[(size_t)ib * N + on] += cib;
                                lam_star[(size_t)i * N + o] -= ci;
                            } else {
                                lam_star[(size_t)i * N + on] += ci;
                                lam_star[(size_t)i * N + o] += cip;
                            }
                        }
                    }

        /* adjoint of the collision, cell by cell */
        for (size_t m = 0; m < 3 * npl; ++m) g_up_prev[m] = 0.0;
        #pragma omp parallel for schedule(static)
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x) {
                    size_t o = cidx(S, x, y, z);
                    int xi[3] = {x, y, z};
                    size_t pl = (size_t)xi[cxx] * dims[bx] + xi[bx];
                    double ls[OR_MAXQ], lf[OR_MAXQ];
                    for (int i = 0; i < q; ++i) ls[i] = lam_star[(size_t)i * N + o];
                    gp_cell[o] = 0.0;
                    for (int k = 0; k < 3; ++k) g_uB[3 * o + k] = 0.0;
                    for (int k = 0; k < 9; ++k) g_S[9 * o + k] = 0.0;
                    for (int i = 0; i < q; ++i) lf[i] = 0.0;
                    if (P->open_boundaries && xi[ax] == 0) {
                        /* inlet: f* = f^eq(1, u_in(t)) does not depend on the state */
                    } else if (P->open_boundaries && xi[ax] == dims[ax] - 1) {
                        /* outlet: f* = f^eq(1, u_plane), u_plane from the previous step */
                        int prev = (int)((S->step & 1) ^ 1);
                        const double* u0 = S->uplane[prev] + 3 * pl;
                        for (int k = 0; k < 3; ++k) {
                            cplx uc[3] = {u0[0], u0[1], u0[2]}, fe[OR_MAXQ];
                            uc[k] += I * CSTEP;
                            equilibrium_c(L, 1.0, uc, fe);
                            double sacc = 0.0;
                            for (int i = 0; i < q; ++i) sacc += ls[i] * cimag(fe[i]) / CSTEP;
                            g_up_prev[3 * pl + k] = sacc;
                        }
                    } else {
                        double fin[OR_MAXQ];
                        for (int i = 0; i < q; ++i) fin[i] = S->f[(size_t)i * N + o];
                        cell_band B;
                        band_of_cell(S, o, x, y, z, &B);
                        double gd, gu[3], gS[3][3];
                        collide_vjp(L, fin, &B, P->tau_mo, P->c_smag, ls, lf, &gd, gu, gS);
                        const double d0 = S->d0 ? S->d0[o] : 1.0;
                        if (S->flags[o] & FL_B) {
                            /* d = d0 d_rotor(pitch); u^B = u_s + du_WM */
                            dJdd0[o] += gd * S->d[o];
                            const or_rotor* R = &S->rot[S->tag[o]].r;
                            blade_frames BF;
                            blade_frames_at(R, S->step, &BF);
                            cplx pc = R->pitch + I * CSTEP;
                            cplx val = component_phi_c(R, &BF, S->which[o], x, y, z, ccos(pc), csin(pc));
                            double ddp = cimag(porosity_c(val, P->eps_h, P->transition)) / CSTEP;
                            gp_cell[o] = gd * d0 * ddp;
                            for (int k = 0; k < 3; ++k) g_uB[3 * o + k] = gu[k];
                            for (int p = 0; p < 3; ++p)
                                for (int r = 0; r < 3; ++r) g_S[9 * o + 3 * p + r] = gS[p][r];
                        } else {
                            dJdd0[o] += gd;
                        }
                        if (P->open_boundaries && xi[ax] == dims[ax] - 2) {
                            /* u of this cell became the outlet's u_plane for the next step */
                            double rho = 0.0, jm[3] = {0, 0, 0};
                            for (int i = 0; i < q; ++i) {
                                rho += fin[i];
                                for (int k = 0; k < 3; ++k) jm[k] += L->c[i][k] * fin[i];
                            }
                            const double* gu_pl = g_up_cur + 3 * pl;
                            for (int i = 0; i < q; ++i)
                                for (int k = 0; k < 3; ++k)
                                    lf[i] += gu_pl[k] * (L->c[i][k] - jm[k] / rho) / rho;
                        }
                    }
                    for (int i = 0; i < q; ++i) lam_new[(size_t)i * N + o] = lf[i];
                }

        /* adjoint of the finite-difference strain (sigma < 1): S^FD of a force
           cell off the wall set is built by fd_strain from the pre-collision
           velocities of its axis neighbours, g_ab = (u_b(x + e_a) - u_b(x - e_a)) / h_a
           and S = (g + g^T) / 2; its transpose hands dJ/dg_ab = (gS_ab + gS_ba) / 2
           to those velocities (to the cell itself where a one-sided difference
           replaced a neighbour across an open face), and du/df_i = (c_i - u) / rho
           to their populations */
        if (P->sigma_band < 1.0)
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        size_t o = cidx(S, x, y, z);
                        if (!(S->flags[o] & FL_B) || (P->wall_model && (S->flags[o] & FL_W))) continue;
                        double G[3][3];
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) G[a][b] = 0.5 * (g_S[9 * o + 3 * a + b] + g_S[9 * o + 3 * b + a]);
                        const int xi[3] = {x, y, z};
                        for (int a = 0; a < 3; ++a) {
                            int e[3] = {0, 0, 0};
                            e[a] = 1;
                            int xp[3], xm[3];
                            const int okp = neighbour(S, xi, e, +1, xp), okm = neighbour(S, xi, e, -1, xm);
                            const double h = (okp && okm) ? 2.0 : 1.0;
                            const size_t cp = okp ? cidx(S, xp[0], xp[1], xp[2]) : o;
                            const size_t cm = okm ? cidx(S, xm[0], xm[1], xm[2]) : o;
                            for (int side = 0; side < 2; ++side) {
                                const size_t cn = side == 0 ? cp : cm;
                                const double sg = side == 0 ? 1.0 / h : -1.0 / h;
                                double u[3], rho;
                                cell_velocity(S, cn, u, &rho);
                                for (int i = 0; i < q; ++i) {
                                    double acc = 0.0;
                                    for (int b = 0; b < 3; ++b) acc += sg * G[a][b] * (L->c[i][b] - u[b]);
                                    lam_new[(size_t)i * N + cn] += acc / rho;
                                }
                            }
                        }
                    }

        /* adjoint of the wall model: corner velocities and pitch */
        if (P->wall_model) {
            #pragma omp parallel for schedule(dynamic, 64)
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        size_t o = cidx(S, x, y, z);
                        for (int m = 0; m < 24; ++m) wm_ubar[24 * o + m] = 0.0;
                        wm_pbar[o] = 0.0;
                        g_ut_prev[o] = 0.0;
                        if (!((S->flags[o] & FL_W) && S->wm_active[o])) continue;
                        size_t idx[8];
                        wall_corners(S, o, x, y, z, idx);
                        double ucr[8][3];
                        for (int m = 0; m < 8; ++m) cell_velocity(S, idx[m], ucr[m], NULL);
                        const or_rotor* R = &S->rot[S->tag[o]].r;
                        blade_frames BF;
                        blade_frames_at(R, S->step, &BF);
                        const double* nr = S->nrm + 3 * o;
                        const double* y1v = S->y1 + 3 * o;
                        double y1r = sqrt(y1v[0] * y1v[0] + y1v[1] * y1v[1] + y1v[2] * y1v[2]);
                        double gout[13];
                        for (int k = 0; k < 3; ++k) gout[k] = g_uB[3 * o + k];
                        for (int k = 0; k < 9; ++k) gout[3 + k] = g_S[9 * o + k];
                        gout[12] = g_ut_cur[o];     /* u_tau is the next step's Newton start */
                        const int warm = tp.wm_active[(size_t)s * N + o];
                        const double guess_prev = tp.wm_ut[(size_t)s * N + o];
                        /* 24 corner-velocity directions, the pitch, the Newton start */
                        for (int dir = 0; dir < 26; ++dir) {
                            if (dir == 25 && !warm) break;
                            cplx uc[8][3], n[3], y1 = y1r, du[3], Sm[9], ut_out, gs = guess_prev;
                            for (int m = 0; m < 8; ++m)
                                for (int k = 0; k < 3; ++k) uc[m][k] = ucr[m][k];
                            for (int k = 0; k < 3; ++k) n[k] = nr[k];
                            if (dir < 24) {
                                uc[dir / 3][dir % 3] += I * CSTEP;
                            } else if (dir == 25) {
                                gs += I * CSTEP;
                            } else {
                                cplx pc = R->pitch + I * CSTEP, cp = ccos(pc), sp = csin(pc);
                                cplx nc[3];
                                rotor_normal_c(R, &BF, S->which[o], x, y, z, cp, sp, nc);
                                for (int k = 0; k < 3; ++k) n[k] = nr[k] + I * cimag(nc[k]);
                                cplx val = component_phi_c(R, &BF, S->which[o], x, y, z, cp, sp);
                                /* y1 = max(phi, 1/2): the forward's branch, on its binary32 phi */
                                float vf = component_phi_f32(R, &BF, S->which[o], x, y, z);
                                if ((double)vf > 0.5) y1 = y1r + I * cimag(val);
                            }
                            wall_cell_c(S, o, x, y, z, (const cplx(*)[3])uc, n, y1, warm, gs, du, Sm, &ut_out);
                            double acc = 0.0;
                            for (int k = 0; k < 3; ++k) acc += gout[k] * cimag(du[k]) / CSTEP;
                            for (int k = 0; k < 9; ++k) acc += gout[3 + k] * cimag(Sm[k]) / CSTEP;
                            acc += gout[12] * cimag(ut_out) / CSTEP;
                            if (dir < 24) wm_ubar[24 * o + dir] = acc;
                            else if (dir == 24) wm_pbar[o] = acc;
                            else g_ut_prev[o] = acc;
                        }
                    }
            /* scatter into the corner cells' populations: du/df_i = (c_i - u) / rho */
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        size_t o = cidx(S, x, y, z);
                        if (!((S->flags[o] & FL_W) && S->wm_active[o])) continue;
                        size_t idx[8];
                        wall_corners(S, o, x, y, z, idx);
                        for (int m = 0; m < 8; ++m) {
                            double u[3], rho;
                            cell_velocity(S, idx[m], u, &rho);
                            for (int i = 0; i < q; ++i) {
                                double acc = 0.0;
                                for (int k = 0; k < 3; ++k) acc += wm_ubar[24 * o + 3 * m + k] * (L->c[i][k] - u[k]);
                                lam_new[(size_t)i * N + idx[m]] += acc / rho;
                            }
                        }
                        dJdp[S->tag[o]] += wm_pbar[o];
                    }
        }
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x) {
                    size_t o = cidx(S, x, y, z);
                    if (S->flags[o] & FL_B) dJdp[S->tag[o]] += gp_cell[o];
                }
        double* tswap = lam; lam = lam_new; lam_new = tswap;
        tswap = g_up_cur; g_up_cur = g_up_prev; g_up_prev = tswap;
        tswap = g_ut_cur; g_ut_cur = g_ut_prev; g_ut_prev = tswap;
        if (!P->wall_model)
            for (size_t m = 0; m < N; ++m) g_ut_cur[m] = 0.0;
    }

    /* put back the final forward state */
    memcpy(S->f, f_end, sizeof(double) * q * N);
    memcpy(S->wm_ut, ut_end, sizeof(double) * N);
    memcpy(S->wm_active, act_end, N);
    memcpy(S->uplane[0], up_end, sizeof(double) * 3 * npl);
    memcpy(S->uplane[1], up_end + 3 * npl, sizeof(double) * 3 * npl);
    memcpy(S->F, Fk, sizeof Fk);
    memcpy(S->M, Mk, sizeof Mk);
    S->wm_newton_iters = it_end;
    S->wm_evals = ev_end;
    /* geometry arrays as or_step leaves them: those of the last step taken */
    S->step = step_end - 1;
    update_porosity(S);
    S->step = step_end;
    *J_out = J;
    free(f_end); free(ut_end); free(act_end); free(up_end);
    free(tp.f); free(tp.wm_ut); free(tp.wm_active); free(tp.uplane); free(lam); free(lam_star); free(lam_new);
    free(g_up_cur); free(g_up_prev); free(g_uB); free(g_S); free(gp_cell); free(wm_ubar); free(wm_pbar);
    free(g_ut_cur); free(g_ut_prev);
    return 0;
}

/* d(d_rotor)/d(pitch) of every force-set cell for the geometry of the last
   porosity update (complex step, component and sets frozen), 0 elsewhere. */
void or_porosity_tangent(const or_state* S, double* dd)
{
    const or_params* P = &S->P;
    long t = S->step > 0 ? S->step - 1 : 0;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                dd[o] = 0.0;
                if (!(S->flags[o] & FL_B)) continue;
                const or_rotor* R = &S->rot[S->tag[o]].r;
                blade_frames BF;
                blade_frames_at(R, t, &BF);
                cplx pc = R->pitch + I * CSTEP;
                cplx val = component_phi_c(R, &BF, S->which[o], x, y, z, ccos(pc), csin(pc));
                dd[o] = cimag(porosity_c(val, P->eps_h, P->transition)) / CSTEP;
            }
}

/* Tangents d(du_WM)/d(pitch) [N][3] and d(S_WM)/d(pitch) [N][9] of the wall
   model at the current step (porosity update and wall model are run first,
   as at the start of or_step, without advancing the state). */
void or_wall_tangent(or_state* S, double* ddu, double* dSm)
{
    const or_params* P = &S->P;
    double* guess = (double*)malloc(sizeof(double) * S->N);
    unsigned char* warm = (unsigned char*)malloc(S->N);
    memcpy(guess, S->wm_ut, sizeof(double) * S->N);
    memcpy(warm, S->wm_active, S->N);
    update_porosity(S);
    wall_model(S);
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                size_t o = cidx(S, x, y, z);
                for (int k = 0; k < 3; ++k) ddu[3 * o + k] = 0.0;
                for (int k = 0; k < 9; ++k) dSm[9 * o + k] = 0.0;
                if (!(P->wall_model && (S->flags[o] & FL_W) && S->wm_active[o])) continue;
                size_t idx[8];
                wall_corners(S, o, x, y, z, idx);
                cplx uc[8][3];
                for (int m = 0; m < 8; ++m) {
                    double u[3];
                    cell_velocity(S, idx[m], u, NULL);
                    for (int k = 0; k < 3; ++k) uc[m][k] = u[k];
                }
                const or_rotor* R = &S->rot[S->tag[o]].r;
                blade_frames BF;
                blade_frames_at(R, S->step, &BF);
                const double* y1v = S->y1 + 3 * o;
                double y1r = sqrt(y1v[0] * y1v[0] + y1v[1] * y1v[1] + y1v[2] * y1v[2]);
                cplx pc = R->pitch + I * CSTEP, cp = ccos(pc), sp = csin(pc);
                cplx nc[3], n[3], y1 = y1r, du[3], Sm[9];
                rotor_normal_c(R, &BF, S->which[o], x, y, z, cp, sp, nc);
                for (int k = 0; k < 3; ++k) n[k] = S->nrm[3 * o + k] + I * cimag(nc[k]);
                cplx val = component_phi_c(R, &BF, S->which[o], x, y, z, cp, sp);
                float vf = component_phi_f32(R, &BF, S->which[o], x, y, z);
                if ((double)vf > 0.5) y1 = y1r + I * cimag(val);
                cplx ut_out;
                wall_cell_c(S, o, x, y, z, (const cplx(*)[3])uc, n, y1, warm[o], guess[o], du, Sm, &ut_out);
                for (int k = 0; k < 3; ++k) ddu[3 * o + k] = cimag(du[k]) / CSTEP;
                for (int k = 0; k < 9; ++k) dSm[9 * o + k] = cimag(Sm[k]) / CSTEP;
            }
    free(guess);
    free(warm);
}

/* d n / d(pitch) of component `which` of rotor R at cell (x, y, z), time t */
void or_rotor_normal_tangent(const or_rotor* R, long t, int which, int x, int y, int z, double* dn)
{
    blade_frames BF;
    blade_frames_at(R, t, &BF);
    cplx pc = R->pitch + I * CSTEP, nc[3];
    rotor_normal_c(R, &BF, which, x, y, z, ccos(pc), csin(pc), nc);
    for (int k = 0; k < 3; ++k) dn[k] = cimag(nc[k]) / CSTEP;
}


/* Torque-driven rotation of rotor k from the current step on: moment of
   inertia about the axis (> 0), generator torque q_gen0 + k_gen Omega |Omega|.
   The rotor starts from its current angle and angular velocity. */
int or_set_drive(or_state* S, int k, double inertia, double k_gen, double q_gen0)
{
    if (k < 0 || k >= S->nrot || !(inertia > 0.0)) return -1;
    rotor_store* rs = &S->rot[k];
    rs->theta = rotor_angle(rs, S->step);
    rs->driven = 1;
    rs->inertia = inertia;
    rs->k_gen = k_gen;
    rs->q_gen0 = q_gen0;
    return 0;
}

/* angle and angular velocity of rotor k at the current step */
int or_drive_state(const or_state* S, int k, double* theta, double* omega)
{
    if (k < 0 || k >= S->nrot) return -1;
    *theta = rotor_angle(&S->rot[k], S->step);
    *omega = S->rot[k].r.omega;
    return 0;
}


/* finite-difference strain of every cell of the current state, [N][3][3] */
void or_fd_strain(const or_state* S, double* out)
{
    const or_params* P = &S->P;
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                double Sm[3][3];
                fd_strain(S, x, y, z, Sm);
                double* o = out + 9 * cidx(S, x, y, z);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) o[3 * a + b] = Sm[a][b];
            }
}
