/*
 * FP64 CPU oracle for the phase-field thermocapillary lattice Boltzmann method
 * (Wang, He & Wang, "Phase-field-based lattice Boltzmann model for simulating
 * thermocapillary flows", arXiv 2306.11320).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain definition that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no source, header,
 * table or helper with the CUDA library.
 *
 * Structure of one time step (every pass is a plain loop over all nodes, two
 * full population buffers, no tiling and no fusion):
 *   pass 1  zeroth moments phi = sum f_i (Sec. 3.1), T = sum h_i (Eq. 31)
 *   pass 2  per-node macroscopic state: isotropic stencils, property closures
 *           (Eq. 45), chemical potential, interfacial force (Eq. 11), velocity
 *           and pressure (Sec. 3.1), d(phi u)/dt (Eq. 44), local grad T (Eq. 40)
 *   pass 3  BGK collisions of the three LBEs (Eq. 14, Sec. 3.1 NS LBE, Eq. 28)
 *   pass 4  pull streaming with the heat-capacitance weighted update of Eq. 28
 *           and the boundary rules of Sec. 4
 *
 * Readings of places where the paper is silent or garbled (the CUDA path takes
 * the same readings):
 *   R1  D2Q9 weights 4/9, 1/9 (x4), 1/36 (x4) (the printed 4/9 for i=1..4 is a typo).
 *   R2  Isotropic central stencils: grad X = sum_i w_i c_i X(x+c_i) / cs2,
 *       lap X = sum_i 2 w_i (X(x+c_i) - X(x)) / cs2.  grad rho = d(rho)/d(phi) grad phi
 *       (derivative of Eq. 8), grad sigma = sigma'(T) grad T (stencil grad T).
 *   R3  Ghost values outside the fluid: phi mirrored across halfway walls (zero
 *       normal gradient, neutral wetting), T = 2 T_wall - T_fluid (linear to the
 *       wall value at the halfway point); inlet T = 2 T_in - T, outlet zero gradient.
 *   R4  Local grad T for the thermal source: grad T = -sum_i c_i (h_i - w_i T) / (tau_h cs2)
 *       (from Eq. 40; the inline formula after Eq. 42 drops c_i and the sign).
 *   R5  rho c_p in Eq. 28 is taken at the destination node at time t.
 *   R6  Property interpolation (Eq. 45) uses phi clamped to [-1, 1]; phi itself is never clipped.
 *   R7  n = grad phi / |grad phi| is set to zero when |grad phi| <= 1e-10.
 *   R8  Walls: halfway bounce-back for f and g; anti-bounce-back for h with the
 *       wall temperature taken at the link's wall-crossing point.
 *   R9  Inlet (x = -1/2): velocity bounce-back g_i = g*_opp + 2 w_i rho c_i.u_in / cs2,
 *       f_i = f*_opp + 2 w_i phi_in c_i.u_in / cs2, anti-bounce-back for h with T_in;
 *       u_in(y) = 6 u_ave y (H - y) / H^2 along x.  Outlet (x = nx - 1/2), "stress free":
 *       pressure anti-bounce-back g_i = -g*_opp + 2 w_i [p_out/cs2 + rho ((c_i.u)^2/(2 cs2^2)
 *       - u.u/(2 cs2))] with the node's own u; f and h extrapolated with zero gradient in x
 *       (the h copy is the adiabatic condition).
 *   R10 (phi u) at the step before the first is phi0 u0 of the initial fields.
 */
#include <tgmath.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* Arithmetic type of the oracle: double (the reference).  A float build
 * (-DORACLE_REAL=float -fsingle-precision-constant) evaluates the same algorithm in
 * float32; tests use it only to measure the float32 rounding floor of the method. */
#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

/* D2Q9 velocity set in the paper's order (Sec. 4, Eq. 43): rest, the four axis
 * directions at angles (i-1) pi/2, the four diagonals at angles (2i-1) pi/4. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const real WQ[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const real CS2 = 1.0 / 3.0;
/* order-parameter values of the two bulk phases (Sec. 2) */
static const real PHI_L = -1.0, PHI_H = 1.0;

typedef struct {
    double rho_l, rho_h, mu_l, mu_h, lambda_l, lambda_h, cp_l, cp_h;
    double W, M_phi;
    double sigma_ref, sigma_T, sigma_TT, T_ref;
    double Gx, Gy;
    double u_ave, phi_in, T_in, p_out;
    double T_bot, T_bot_amp, T_bot_k, T_bot_slope, T_top, T_top_slope;
    double trt_lambda; /* two-relaxation-time "magic" parameter (tau+ - 1/2)(tau- - 1/2) */
    int sigma_law; /* 0 linear (Eq. 12), 1 parabolic (Eq. 63) */
    int bc_x;      /* 0 periodic, 1 velocity inlet at x=-1/2 and outflow at x=nx-1/2 */
    int bc_y;      /* 0 halfway no-slip walls at y=-1/2 and y=ny-1/2, 1 periodic */
    int normal_law; /* interface normal in R_i: 0 from the stencil grad phi (R7), 1 local from f (Sec. 3) */
    int collision;  /* g and h LBEs: 0 BGK (Sec. 3), 1 two relaxation times (TRT) */
} orc_params;

/* the parameters in the oracle's arithmetic type */
typedef struct {
    real rho_l, rho_h, mu_l, mu_h, lambda_l, lambda_h, cp_l, cp_h;
    real W, M_phi;
    real sigma_ref, sigma_T, sigma_TT, T_ref;
    real Gx, Gy;
    real u_ave, phi_in, T_in, p_out;
    real T_bot, T_bot_amp, T_bot_k, T_bot_slope, T_top, T_top_slope;
    real trt_lambda;
    int sigma_law, bc_x, bc_y, normal_law, collision;
} rparams;

typedef struct {
    orc_params P;
    rparams R;
    int nx, ny;
    long long t;
    real *f, *g, *h;          /* [Q][ny][nx] pre-collision populations at time t */
    real *fs, *gs, *hs;       /* post-collision scratch */
    real *f2, *g2, *h2;       /* next-time buffers */
    real *phiu_prev;          /* [2][ny][nx]: (phi u) at the previous step */
    /* macroscopic fields of the current time level */
    real *phi, *T, *ux, *uy, *p, *rho, *rcp, *tau_g, *tau_h, *Fhat;
    real *dphiux, *dphiuy, *nx_, *ny_, *Fx, *Fy, *gradrx, *gradry;
} orc_sim;

/* ---------------------------------------------------------------- lattice */

void orc_lattice(int *ex, int *ey, double *w, int *opp)
{
    for (int i = 0; i < Q; ++i) {
        ex[i] = EX[i];
        ey[i] = EY[i];
        w[i] = WQ[i];
        /* opposite direction: the one with c_j = -c_i */
        for (int j = 0; j < Q; ++j)
            if (EX[j] == -EX[i] && EY[j] == -EY[i]) opp[i] = j;
    }
}

static int opposite(int i)
{
    for (int j = 0; j < Q; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i]) return j;
    return -1;
}

/* ------------------------------------------------------ per-node operators */

/* Property interpolation, Eq. 45: linear in phi between the two bulk values. */
real orc_interp(real phi, real xi_l, real xi_h)
{
    real pc = phi < PHI_L ? PHI_L : (phi > PHI_H ? PHI_H : phi); /* R6 */
    return (pc - PHI_H) / (PHI_L - PHI_H) * xi_l + (pc - PHI_L) / (PHI_H - PHI_L) * xi_h;
}

/* Allen-Cahn equilibrium, Sec. 3.1: f_i^eq = w_i phi (1 + c_i.u / cs2). */
void orc_feq(real phi, real ux, real uy, real *out)
{
    for (int i = 0; i < Q; ++i) {
        real cu = EX[i] * ux + EY[i] * uy;
        out[i] = WQ[i] * phi * (1.0 + cu / CS2);
    }
}

/* Allen-Cahn source, Sec. 3.1:
 * R_i = w_i c_i.[ d_t(phi u) + cs2 n (1 - phi^2) / (sqrt2 W) ] / cs2. */
void orc_Ri(real phi, real dphiux, real dphiuy, real nx, real ny, real W,
            real *out)
{
    real theta = (1.0 - phi * phi) / (sqrt(2.0) * W);
    real ax = dphiux + CS2 * nx * theta;
    real ay = dphiuy + CS2 * ny * theta;
    for (int i = 0; i < Q; ++i) out[i] = WQ[i] * (EX[i] * ax + EY[i] * ay) / CS2;
}

/* s_i(u) of the NS equilibrium, Sec. 3.1. */
static real s_i(int i, real ux, real uy)
{
    real cu = EX[i] * ux + EY[i] * uy;
    real uu = ux * ux + uy * uy;
    return WQ[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Pressure-based NS equilibrium, Sec. 3.1:
 * g_0^eq = p/cs2 (w_0 - 1) + rho s_0(u),  g_i^eq = p/cs2 w_i + rho s_i(u). */
void orc_geq(real p, real rho, real ux, real uy, real *out)
{
    for (int i = 0; i < Q; ++i) {
        real wp = (i == 0) ? (WQ[0] - 1.0) : WQ[i];
        out[i] = p / CS2 * wp + rho * s_i(i, ux, uy);
    }
}

/* NS forcing, Sec. 3.1:
 * G_i = w_i [ u.grad rho + c_i.(Fs + G)/cs2 + u grad rho : (c_i c_i - cs2 I)/cs2 ]. */
void orc_Gi(real ux, real uy, real grx, real gry, real Fx, real Fy, real *out)
{
    real ug = ux * grx + uy * gry;
    for (int i = 0; i < Q; ++i) {
        real cF = EX[i] * Fx + EY[i] * Fy;
        real cu = EX[i] * ux + EY[i] * uy;
        real cg = EX[i] * grx + EY[i] * gry;
        real dyad = cu * cg - CS2 * ug; /* u grad rho : (c c - cs2 I) */
        out[i] = WQ[i] * (ug + cF / CS2 + dyad / CS2);
    }
}

/* Thermal equilibrium, Eq. 31 (labelled weq_31): h_i^eq = w_i T. */
void orc_heq(real T, real *out)
{
    for (int i = 0; i < Q; ++i) out[i] = WQ[i] * T;
}

/* Thermal source, Eq. 30: Fhat_i = w_i Fhat. */
void orc_Fhat_i(real Fhat, real *out)
{
    for (int i = 0; i < Q; ++i) out[i] = WQ[i] * Fhat;
}

/* Surface tension law: linear (Eq. 12) or parabolic (Eq. 63), and dsigma/dT. */
static void sigma_of_T(const rparams *P, real T, real *sig, real *dsig)
{
    if (P->sigma_law == 1) {
        *sig = 0.5 * P->sigma_TT * (T - P->T_ref) * (T - P->T_ref) + P->sigma_ref;
        *dsig = P->sigma_TT * (T - P->T_ref);
    } else {
        *sig = P->sigma_ref + P->sigma_T * (T - P->T_ref);
        *dsig = P->sigma_T;
    }
}

/* Interfacial force, last line of Eq. 11:
 * Fs = 3 sqrt2 W / 4 [ |grad phi|^2 grad sigma - (grad sigma . grad phi) grad phi
 *                      + sigma mu_phi grad phi / W^2 ]. */
void orc_Fs(real W, real sigma, real gsx, real gsy, real mu_phi, real gpx,
            real gpy, real *Fx, real *Fy)
{
    real k = 3.0 * sqrt(2.0) * W / 4.0;
    real g2 = gpx * gpx + gpy * gpy;
    real sp = gsx * gpx + gsy * gpy;
    *Fx = k * (g2 * gsx - sp * gpx + sigma * mu_phi * gpx / (W * W));
    *Fy = k * (g2 * gsy - sp * gpy + sigma * mu_phi * gpy / (W * W));
}

/* Chemical potential (Sec. 2, after Eq. 11):
 * mu_phi = (phi - phi_l)(phi - phi_h)(phi - (phi_l + phi_h)/2) - W^2 lap phi. */
real orc_mu_phi(real phi, real lap, real W)
{
    return (phi - PHI_L) * (phi - PHI_H) * (phi - 0.5 * (PHI_L + PHI_H)) - W * W * lap;
}

/* ------------------------------------------------------------ wall values */

static real T_wall_bottom(const rparams *P, int nx, real x)
{
    const real pi = 3.14159265358979323846;
    return P->T_bot + P->T_bot_amp * cos(2.0 * pi * P->T_bot_k * x / nx) + P->T_bot_slope * x;
}

static real T_wall_top(const rparams *P, real x)
{
    return P->T_top + P->T_top_slope * x;
}

/* Poiseuille inlet profile along x (Sec. 4.3, Eq. 62 with u along the channel):
 * y is measured from the bottom wall, H = ny. */
static real u_inlet(const rparams *P, int ny, real y)
{
    real H = (real)ny;
    return 6.0 * P->u_ave * y * (H - y) / (H * H);
}

/* ------------------------------------------------------- ghost-aware reads */

static inline size_t IDX(const orc_sim *s, int x, int y) { return (size_t)y * s->nx + x; }

/* phi at a lattice point one step outside the fluid (R3). */
static real phi_at(const orc_sim *s, int x, int y)
{
    if (y < 0 || y >= s->ny) {
        if (s->R.bc_y == 1) y = (y + s->ny) % s->ny;
        else y = y < 0 ? 0 : s->ny - 1;
    }
    if (x < 0 || x >= s->nx) {
        if (s->R.bc_x == 0) x = (x + s->nx) % s->nx;
        else x = x < 0 ? 0 : s->nx - 1;
    }
    return s->phi[IDX(s, x, y)];
}

/* T at a lattice point one step outside the fluid (R3). */
static real T_at(const orc_sim *s, int x, int y)
{
    if (y < 0 || y >= s->ny) {
        if (s->R.bc_y == 1) {
            y = (y + s->ny) % s->ny;
        } else if (y < 0) {
            return 2.0 * T_wall_bottom(&s->R, s->nx, (real)x) - T_at(s, x, 0);
        } else {
            return 2.0 * T_wall_top(&s->R, (real)x) - T_at(s, x, s->ny - 1);
        }
    }
    if (x < 0 || x >= s->nx) {
        if (s->R.bc_x == 0) x = (x + s->nx) % s->nx;
        else if (x < 0) return 2.0 * s->R.T_in - s->T[IDX(s, 0, y)];
        else return s->T[IDX(s, s->nx - 1, y)];
    }
    return s->T[IDX(s, x, y)];
}

/* ------------------------------------------------------------ life cycle */

static void real_params(const orc_params *P, rparams *R)
{
    R->rho_l = (real)P->rho_l;
    R->rho_h = (real)P->rho_h;
    R->mu_l = (real)P->mu_l;
    R->mu_h = (real)P->mu_h;
    R->lambda_l = (real)P->lambda_l;
    R->lambda_h = (real)P->lambda_h;
    R->cp_l = (real)P->cp_l;
    R->cp_h = (real)P->cp_h;
    R->W = (real)P->W;
    R->M_phi = (real)P->M_phi;
    R->sigma_ref = (real)P->sigma_ref;
    R->sigma_T = (real)P->sigma_T;
    R->sigma_TT = (real)P->sigma_TT;
    R->T_ref = (real)P->T_ref;
    R->Gx = (real)P->Gx;
    R->Gy = (real)P->Gy;
    R->u_ave = (real)P->u_ave;
    R->phi_in = (real)P->phi_in;
    R->T_in = (real)P->T_in;
    R->p_out = (real)P->p_out;
    R->T_bot = (real)P->T_bot;
    R->T_bot_amp = (real)P->T_bot_amp;
    R->T_bot_k = (real)P->T_bot_k;
    R->T_bot_slope = (real)P->T_bot_slope;
    R->T_top = (real)P->T_top;
    R->T_top_slope = (real)P->T_top_slope;
    R->sigma_law = P->sigma_law;
    R->bc_x = P->bc_x;
    R->bc_y = P->bc_y;
    R->normal_law = P->normal_law;
    R->collision = P->collision;
    R->trt_lambda = (real)P->trt_lambda;
}

static real *alloc0(size_t n) { return (real *)calloc(n, sizeof(real)); }

int orc_create(int nx, int ny, const orc_params *P, orc_sim **out)
{
    if (nx < 3 || ny < 3 || !P || !out) return -1;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return -2;
    s->P = *P;
    real_params(P, &s->R);
    s->nx = nx;
    s->ny = ny;
    size_t N = (size_t)nx * ny;
    s->f = alloc0(Q * N); s->g = alloc0(Q * N); s->h = alloc0(Q * N);
    s->fs = alloc0(Q * N); s->gs = alloc0(Q * N); s->hs = alloc0(Q * N);
    s->f2 = alloc0(Q * N); s->g2 = alloc0(Q * N); s->h2 = alloc0(Q * N);
    s->phiu_prev = alloc0(2 * N);
    s->phi = alloc0(N); s->T = alloc0(N); s->ux = alloc0(N); s->uy = alloc0(N);
    s->p = alloc0(N); s->rho = alloc0(N); s->rcp = alloc0(N); s->tau_g = alloc0(N);
    s->tau_h = alloc0(N); s->Fhat = alloc0(N); s->dphiux = alloc0(N); s->dphiuy = alloc0(N);
    s->nx_ = alloc0(N); s->ny_ = alloc0(N); s->Fx = alloc0(N); s->Fy = alloc0(N);
    s->gradrx = alloc0(N); s->gradry = alloc0(N);
    if (!s->gradry) return -2;
    *out = s;
    return 0;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    real *bufs[] = {s->f, s->g, s->h, s->fs, s->gs, s->hs, s->f2, s->g2, s->h2,
                      s->phiu_prev, s->phi, s->T, s->ux, s->uy, s->p, s->rho, s->rcp,
                      s->tau_g, s->tau_h, s->Fhat, s->dphiux, s->dphiuy, s->nx_, s->ny_,
                      s->Fx, s->Fy, s->gradrx, s->gradry};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    free(s);
}

/* Initial populations from macroscopic fields (the paper gives none; R10):
 * f = f^eq(phi0, u0), g = g^eq(p0, rho(phi0), u0), h = h^eq(T0), (phi u)_prev = phi0 u0. */
int orc_init(orc_sim *s, const double *phi, const double *ux, const double *uy,
             const double *p, const double *T)
{
    size_t N = (size_t)s->nx * s->ny;
    real e[Q];
    for (size_t n = 0; n < N; ++n) {
        real rho = orc_interp((real)phi[n], s->R.rho_l, s->R.rho_h);
        orc_feq((real)phi[n], (real)ux[n], (real)uy[n], e);
        for (int i = 0; i < Q; ++i) s->f[i * N + n] = e[i];
        orc_geq((real)p[n], rho, (real)ux[n], (real)uy[n], e);
        for (int i = 0; i < Q; ++i) s->g[i * N + n] = e[i];
        orc_heq((real)T[n], e);
        for (int i = 0; i < Q; ++i) s->h[i * N + n] = e[i];
        s->phiu_prev[n] = (real)phi[n] * (real)ux[n];
        s->phiu_prev[N + n] = (real)phi[n] * (real)uy[n];
    }
    s->t = 0;
    return 0;
}

static void to_real(real *dst, const double *src, size_t n)
{
    for (size_t k = 0; k < n; ++k) dst[k] = (real)src[k];
}

static void to_double(double *dst, const real *src, size_t n)
{
    for (size_t k = 0; k < n; ++k) dst[k] = (double)src[k];
}

int orc_set_state(orc_sim *s, const double *f, const double *g, const double *h,
                  const double *phiu_prev)
{
    size_t N = (size_t)s->nx * s->ny;
    to_real(s->f, f, Q * N);
    to_real(s->g, g, Q * N);
    to_real(s->h, h, Q * N);
    to_real(s->phiu_prev, phiu_prev, 2 * N);
    return 0;
}

int orc_get_state(const orc_sim *s, double *f, double *g, double *h, double *phiu_prev)
{
    size_t N = (size_t)s->nx * s->ny;
    if (f) to_double(f, s->f, Q * N);
    if (g) to_double(g, s->g, Q * N);
    if (h) to_double(h, s->h, Q * N);
    if (phiu_prev) to_double(phiu_prev, s->phiu_prev, 2 * N);
    return 0;
}

/* -------------------------------------------------- pass 1 and 2: moments */

static void macroscopic(orc_sim *s)
{
    const rparams *P = &s->R;
    const int nx = s->nx, ny = s->ny;
    const size_t N = (size_t)nx * ny;
    const real tau_phi = P->M_phi / CS2 + 0.5; /* M_phi = cs2 (tau_phi - 1/2), Sec. 3.1 */
    (void)tau_phi;

    /* pass 1: zeroth moments */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = IDX(s, x, y);
            real sf = 0.0, sh = 0.0;
            for (int i = 0; i < Q; ++i) {
                sf += s->f[i * N + n];
                sh += s->h[i * N + n];
            }
            s->phi[n] = sf;
            s->T[n] = sh;
        }

    /* pass 2: stencils, closures, forces, velocity, pressure */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = IDX(s, x, y);
            real phi = s->phi[n], T = s->T[n];

            /* isotropic stencils (R2) */
            real gpx = 0, gpy = 0, lap = 0, gtx = 0, gty = 0;
            for (int i = 1; i < Q; ++i) {
                real pn = phi_at(s, x + EX[i], y + EY[i]);
                real tn = T_at(s, x + EX[i], y + EY[i]);
                gpx += WQ[i] * EX[i] * pn;
                gpy += WQ[i] * EY[i] * pn;
                lap += 2.0 * WQ[i] * (pn - phi);
                gtx += WQ[i] * EX[i] * tn;
                gty += WQ[i] * EY[i] * tn;
            }
            gpx /= CS2; gpy /= CS2; lap /= CS2; gtx /= CS2; gty /= CS2;

            /* closures: Eq. 45 for rho, mu, lambda and rho c_p */
            real rho = orc_interp(phi, P->rho_l, P->rho_h);
            real mu = orc_interp(phi, P->mu_l, P->mu_h);
            real lam = orc_interp(phi, P->lambda_l, P->lambda_h);
            real rcp = orc_interp(phi, P->rho_l * P->cp_l, P->rho_h * P->cp_h);
            real tau_g = mu / (rho * CS2) + 0.5;     /* mu = rho cs2 (tau_g - 1/2) */
            real tau_h = lam / CS2 + 0.5;            /* lambda = (tau_h - 1/2) cs2 */

            /* chemical potential and interfacial force with Marangoni stress */
            real sig, dsig;
            sigma_of_T(P, T, &sig, &dsig);
            real mu_phi = orc_mu_phi(phi, lap, P->W);
            real Fsx, Fsy;
            orc_Fs(P->W, sig, dsig * gtx, dsig * gty, mu_phi, gpx, gpy, &Fsx, &Fsy);
            real Fx = Fsx + P->Gx, Fy = Fsy + P->Gy;

            /* velocity: rho u = sum c_i g_i + dt/2 (Fs + G) */
            real mx = 0, my = 0, s_ne0 = 0;
            for (int i = 0; i < Q; ++i) {
                real gi = s->g[i * N + n];
                mx += EX[i] * gi;
                my += EY[i] * gi;
                if (i != 0) s_ne0 += gi;
            }
            real ux = (mx + 0.5 * Fx) / rho;
            real uy = (my + 0.5 * Fy) / rho;

            /* grad rho from Eq. 8 */
            real drdphi = (P->rho_l - P->rho_h) / (PHI_L - PHI_H);
            real grx = drdphi * gpx, gry = drdphi * gpy;

            /* pressure: p = cs2/(1 - w0) [ sum_{i!=0} g_i + dt/2 u.grad rho + rho s_0(u) ] */
            real p = CS2 / (1.0 - WQ[0]) * (s_ne0 + 0.5 * (ux * grx + uy * gry) +
                                              rho * s_i(0, ux, uy));

            /* d_t(phi u), first-order Euler (Eq. 44) */
            real dpx = phi * ux - s->phiu_prev[n];
            real dpy = phi * uy - s->phiu_prev[N + n];

            /* unit normal (R7) */
            real gn = sqrt(gpx * gpx + gpy * gpy);
            real nnx = 0.0, nny = 0.0;
            if (gn > 1e-10) {
                nnx = gpx / gn;
                nny = gpy / gn;
            }
            if (P->normal_law == 1) {
                /* local recovery (Sec. 3): J = sum_i c_i (f_i - f_i^eq) + d_t(phi u) / 2
                 * equals -cs2 tau_phi grad phi + M_phi Theta(phi) n with n the unit normal
                 * (Theta = (1 - phi^2)/(sqrt2 W) for phi in [-1, 1]), and M_phi Theta <
                 * cs2 tau_phi |grad phi| on the profile, so n = -J / |J| */
                real feq[Q];
                orc_feq(phi, ux, uy, feq);
                real jx = 0.5 * dpx, jy = 0.5 * dpy;
                for (int i = 0; i < Q; ++i) {
                    real ne = s->f[i * N + n] - feq[i];
                    jx += EX[i] * ne;
                    jy += EY[i] * ne;
                }
                real jn = sqrt(jx * jx + jy * jy);
                real tau_phi = P->M_phi / CS2 + 0.5;
                nnx = nny = 0.0;
                if (jn > 1e-10 * CS2 * tau_phi) {
                    nnx = -jx / jn;
                    nny = -jy / jn;
                }
            }

            /* local temperature gradient from the non-equilibrium part of h (Eq. 40, R4) */
            real qx = 0, qy = 0;
            for (int i = 0; i < Q; ++i) {
                real neq = s->h[i * N + n] - WQ[i] * T;
                qx += EX[i] * neq;
                qy += EY[i] * neq;
            }
            real gTx = -qx / (tau_h * CS2);
            real gTy = -qy / (tau_h * CS2);
            real Fhat = -rcp * (ux * gTx + uy * gTy); /* Eq. 27 source */

            s->ux[n] = ux; s->uy[n] = uy; s->p[n] = p; s->rho[n] = rho; s->rcp[n] = rcp;
            s->tau_g[n] = tau_g; s->tau_h[n] = tau_h; s->Fhat[n] = Fhat;
            s->dphiux[n] = dpx; s->dphiuy[n] = dpy; s->nx_[n] = nnx; s->ny_[n] = nny;
            s->Fx[n] = Fx; s->Fy[n] = Fy; s->gradrx[n] = grx; s->gradry[n] = gry;
        }
}

/* ------------------------------------------------------- pass 3: collide */

/* Two-relaxation-time collision of population i (the extension the paper points to
 * for stability, Sec. 3): with X_i^{+/-} = (X_i +/- X_opp(i)) / 2 for the populations q,
 * their equilibria e and the source S,
 *   q*_i = q_i - (q_i^+ - e_i^+) / tau_p - (q_i^- - e_i^-) / tau_m + c^+ S_i^+ + c^- S_i^-,
 * c^{+/-} = 1 - 1/(2 tau_{+/-}) when the source carries the half-step factor (NS LBE),
 * 1 otherwise (thermal LBE).  tau_p = tau_m is the BGK collision. */
static real trt_one(const real *q, size_t N, size_t n, int i, const real *e, const real *src,
                    real tau_p, real tau_m, int half_step_source)
{
    int o = 0;
    for (int j = 0; j < Q; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i]) o = j;
    real qp = 0.5 * (q[i * N + n] + q[o * N + n]), qm = 0.5 * (q[i * N + n] - q[o * N + n]);
    real ep = 0.5 * (e[i] + e[o]), em = 0.5 * (e[i] - e[o]);
    real sp = 0.5 * (src[i] + src[o]), sm = 0.5 * (src[i] - src[o]);
    real cp = half_step_source ? 1.0 - 0.5 / tau_p : 1.0;
    real cm = half_step_source ? 1.0 - 0.5 / tau_m : 1.0;
    return q[i * N + n] - (qp - ep) / tau_p - (qm - em) / tau_m + cp * sp + cm * sm;
}

static void collide(orc_sim *s)
{
    const rparams *P = &s->R;
    const int nx = s->nx, ny = s->ny;
    const size_t N = (size_t)nx * ny;
    const real tau_phi = P->M_phi / CS2 + 0.5;

#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = IDX(s, x, y);
            real eq[Q], src[Q];

            /* Allen-Cahn LBE, Eq. 14 */
            orc_feq(s->phi[n], s->ux[n], s->uy[n], eq);
            orc_Ri(s->phi[n], s->dphiux[n], s->dphiuy[n], s->nx_[n], s->ny_[n], P->W, src);
            for (int i = 0; i < Q; ++i) {
                real fi = s->f[i * N + n];
                s->fs[i * N + n] = fi - (fi - eq[i]) / tau_phi + (1.0 - 0.5 / tau_phi) * src[i];
            }

            /* Navier-Stokes LBE, Sec. 3.1 */
            real tg = s->tau_g[n];
            orc_geq(s->p[n], s->rho[n], s->ux[n], s->uy[n], eq);
            orc_Gi(s->ux[n], s->uy[n], s->gradrx[n], s->gradry[n], s->Fx[n], s->Fy[n], src);
            if (P->collision == 1) {
                /* TRT: the viscosity stays on the even part (tau+ = tau_g) */
                real tm = 0.5 + P->trt_lambda / (tg - 0.5);
                for (int i = 0; i < Q; ++i)
                    s->gs[i * N + n] = trt_one(s->g, N, n, i, eq, src, tg, tm, 1);
            } else {
                for (int i = 0; i < Q; ++i) {
                    real gi = s->g[i * N + n];
                    s->gs[i * N + n] = gi - (gi - eq[i]) / tg + (1.0 - 0.5 / tg) * src[i];
                }
            }

            /* thermal LBE, Eq. 28: collision part (the rho c_p weighting is applied
             * in the streaming pass) */
            real th = s->tau_h[n];
            orc_heq(s->T[n], eq);
            orc_Fhat_i(s->Fhat[n], src);
            if (P->collision == 1) {
                /* TRT: the conductivity stays on the odd part (tau- = tau_h) */
                real tp = 0.5 + P->trt_lambda / (th - 0.5);
                for (int i = 0; i < Q; ++i)
                    s->hs[i * N + n] = trt_one(s->h, N, n, i, eq, src, tp, th, 0);
            } else {
                for (int i = 0; i < Q; ++i) {
                    real hi = s->h[i * N + n];
                    s->hs[i * N + n] = hi - (hi - eq[i]) / th + src[i];
                }
            }
        }
}

/* -------------------------------------------------------- pass 4: stream */

/* Eq. 28 solved for the new population at the destination y:
 * h_i(y, t+1) = h_i(y, t) + [ hstar_i(y - c_i) - h_i(y, t) ] / (rho c_p)(y). */
static void stream(orc_sim *s)
{
    const rparams *P = &s->R;
    const int nx = s->nx, ny = s->ny;
    const size_t N = (size_t)nx * ny;

#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = IDX(s, x, y);
            real rcp = s->rcp[n];
            for (int i = 0; i < Q; ++i) {
                int sx = x - EX[i], sy = y - EY[i];
                int o = opposite(i);
                real hold = s->h[i * N + n];
                real fnew, gnew, hin;
                int out_y = (sy < 0 || sy >= ny) && P->bc_y == 0;
                if (P->bc_y == 1) sy = (sy + ny) % ny;
                int out_x = (sx < 0 || sx >= nx) && P->bc_x == 1;
                if (P->bc_x == 0) sx = (sx + nx) % nx;

                if (out_y) {
                    /* halfway bounce-back (R8); anti-bounce-back for h with the wall
                     * temperature at the wall-crossing point of the link */
                    real xc = x - 0.5 * EX[i];
                    real Tw = (y - EY[i] < 0) ? T_wall_bottom(P, nx, xc) : T_wall_top(P, xc);
                    fnew = s->fs[o * N + n];
                    gnew = s->gs[o * N + n];
                    hin = -s->hs[o * N + n] + 2.0 * WQ[i] * Tw;
                } else if (out_x && sx < 0) {
                    /* velocity inlet (R9) */
                    real ycr = y + 0.5 - 0.5 * EY[i];
                    real uin = u_inlet(P, ny, ycr);
                    real cu = EX[i] * uin;
                    fnew = s->fs[o * N + n] + 2.0 * WQ[i] * P->phi_in * cu / CS2;
                    gnew = s->gs[o * N + n] + 2.0 * WQ[i] * s->rho[n] * cu / CS2;
                    hin = -s->hs[o * N + n] + 2.0 * WQ[i] * P->T_in;
                } else if (out_x) {
                    /* outflow (R9): pressure anti-bounce-back for g with p = p_out and the
                     * node's own velocity; zero-gradient post-collision f and h */
                    size_t m = IDX(s, nx - 1, sy);
                    real ux = s->ux[n], uy = s->uy[n];
                    real cu = EX[i] * ux + EY[i] * uy;
                    real sym = P->p_out / CS2 + s->rho[n] * (cu * cu / (2.0 * CS2 * CS2) -
                                                               (ux * ux + uy * uy) / (2.0 * CS2));
                    fnew = s->fs[i * N + m];
                    gnew = -s->gs[o * N + n] + 2.0 * WQ[i] * sym;
                    hin = s->hs[i * N + m];
                } else {
                    size_t m = IDX(s, sx, sy);
                    fnew = s->fs[i * N + m];
                    gnew = s->gs[i * N + m];
                    hin = s->hs[i * N + m];
                }
                s->f2[i * N + n] = fnew;
                s->g2[i * N + n] = gnew;
                s->h2[i * N + n] = hold + (hin - hold) / rcp;
            }
        }
}

static void swap_ptr(real **a, real **b)
{
    real *t = *a;
    *a = *b;
    *b = t;
}

int orc_step(orc_sim *s, long long nsteps)
{
    const size_t N = (size_t)s->nx * s->ny;
    for (long long k = 0; k < nsteps; ++k) {
        macroscopic(s);
        collide(s);
        stream(s);
        /* (phi u) of this step becomes the previous value for the next one */
        for (size_t n = 0; n < N; ++n) {
            s->phiu_prev[n] = s->phi[n] * s->ux[n];
            s->phiu_prev[N + n] = s->phi[n] * s->uy[n];
        }
        swap_ptr(&s->f, &s->f2);
        swap_ptr(&s->g, &s->g2);
        swap_ptr(&s->h, &s->h2);
        s->t += 1;
    }
    return 0;
}

long long orc_time(const orc_sim *s) { return s->t; }

/* Macroscopic fields of the current state (the same computation the next step
 * starts with).  Any output pointer may be NULL. */
int orc_get_fields(orc_sim *s, double *phi, double *ux, double *uy, double *p, double *T)
{
    macroscopic(s);
    size_t N = (size_t)s->nx * s->ny;
    if (phi) to_double(phi, s->phi, N);
    if (ux) to_double(ux, s->ux, N);
    if (uy) to_double(uy, s->uy, N);
    if (p) to_double(p, s->p, N);
    if (T) to_double(T, s->T, N);
    return 0;
}

/* Extra per-node quantities of the current state for invariant checks:
 * out[k*N + n] for k = 0 rho, 1 rho c_p, 2 Fhat, 3 Fx, 4 Fy, 5 tau_g, 6 tau_h,
 * 7 n_x, 8 n_y (interface normal), 9, 10 grad rho. */
int orc_get_aux(orc_sim *s, double *out)
{
    macroscopic(s);
    size_t N = (size_t)s->nx * s->ny;
    to_double(out + 0 * N, s->rho, N);
    to_double(out + 1 * N, s->rcp, N);
    to_double(out + 2 * N, s->Fhat, N);
    to_double(out + 3 * N, s->Fx, N);
    to_double(out + 4 * N, s->Fy, N);
    to_double(out + 5 * N, s->tau_g, N);
    to_double(out + 6 * N, s->tau_h, N);
    to_double(out + 7 * N, s->nx_, N);
    to_double(out + 8 * N, s->ny_, N);
    to_double(out + 9 * N, s->gradrx, N);
    to_double(out + 10 * N, s->gradry, N);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
