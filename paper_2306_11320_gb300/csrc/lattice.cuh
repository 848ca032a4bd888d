// D2Q9 lattice and per-node physics of the phase-field thermocapillary LBM
// (arXiv 2306.11320), float32 device code shared by every kernel of the library.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tpf {

// D2Q9 in the order of Eq. 43: rest, axis directions at angles (i-1) pi/2,
// diagonals at angles (2i-1) pi/4.  Weights 4/9, 1/9, 1/36 (the 4/9 printed for the
// axis directions is a typo: the weights must sum to one), cs2 = 1/3.
__host__ __device__ constexpr int cx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__host__ __device__ constexpr int cy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
__host__ __device__ constexpr float wq(int i) { return i == 0 ? 4.f / 9.f : (i < 5 ? 1.f / 9.f : 1.f / 36.f); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
// pressure weight of the NS equilibrium at rest: g_i^eq(u = 0) = wg(i) p / cs2
__host__ __device__ constexpr float wg(int i) { return i == 0 ? 4.f / 9.f - 1.f : wq(i); }
constexpr float kCs2 = 1.f / 3.f;
constexpr float kInvCs2 = 3.f;

// Everything a kernel needs, precomputed on the host from tpflbm_params.
struct DevParams {
    int nx, ny, bc_x, bc_y, sigma_law, storage, normal_law, collision;
    long long plane;  // elements per population plane (>= nx*ny, padded)
    // Eq. 45 as a + b * clamp(phi): value = (xi_l + xi_h)/2 + (xi_h - xi_l)/2 * phi
    float rho_a, rho_b, mu_a, mu_b, lam_a, lam_b, rcp_a, rcp_b;
    float drho_dphi;  // (rho_h - rho_l)/2, derivative of Eq. 8
    float W2, inv_W2, theta_k;  // W^2, 1/W^2, 1/(sqrt2 W)
    float jthr2;      // local normal: |J|^2 below which n = 0 ((1e-10 cs2 tau_phi)^2)
    float trt_lambda; // TRT magic parameter (collision == 1)
    float kFs;                  // 3 sqrt2 W / 4 (Eq. 11)
    float inv_tau_phi, src_phi; // 1/tau_phi, 1 - 1/(2 tau_phi)
    float sigma_ref, sigma_T, sigma_TT, T_ref;
    float Gx, Gy;
    float u_ave, phi_in, T_in, p_out;
    float T_bot, T_bot_amp, T_bot_k, T_bot_slope, T_top, T_top_slope;
    // float16 codec: stored = s_k (q - r); decoded = stored / s_k + r, r per node
    float s_f, s_g, s_h, is_f, is_g, is_h;
};

__device__ __forceinline__ float clamp1(float phi) { return fminf(1.f, fmaxf(-1.f, phi)); }

__device__ __forceinline__ float T_wall_bottom(const DevParams& P, float x)
{
    return P.T_bot + P.T_bot_amp * cospif(2.f * P.T_bot_k * x / (float)P.nx) + P.T_bot_slope * x;
}
__device__ __forceinline__ float T_wall_top(const DevParams& P, float x) { return P.T_top + P.T_top_slope * x; }
// Poiseuille inlet of Sec. 4.3 along x, y measured from the bottom wall.
__device__ __forceinline__ float u_inlet(const DevParams& P, float y)
{
    const float H = (float)P.ny;
    return 6.f * P.u_ave * y * (H - y) / (H * H);
}

// ---------------------------------------------------------------- storage

struct StoreF32 {
    using elem = float;
    // global memory (read-only path)
    template <class I>
    static __device__ __forceinline__ float ld(const float* __restrict__ p, I k, float, float) { return __ldg(p + k); }
    // shared memory (staged copies)
    template <class I>
    static __device__ __forceinline__ float lds(const float* p, I k, float, float) { return p[k]; }
    template <class I>
    static __device__ __forceinline__ void st(float* __restrict__ p, I k, float v, float, float) { p[k] = v; }
};
struct StoreF16 {
    using elem = __half;
    template <class I>
    static __device__ __forceinline__ float ld(const __half* __restrict__ p, I k, float inv_s, float ref)
    {
        return fmaf(__half2float(p[k]), inv_s, ref);
    }
    template <class I>
    static __device__ __forceinline__ float lds(const __half* p, I k, float inv_s, float ref)
    {
        return fmaf(__half2float(p[k]), inv_s, ref);
    }
    template <class I>
    static __device__ __forceinline__ void st(__half* __restrict__ p, I k, float v, float s, float ref)
    {
        p[k] = __float2half_rn((v - ref) * s);
    }
};

// -------------------------------------------------------------- node physics

struct Macro {
    float phi, T, ux, uy, p, rho, rcp, inv_tau_g, src_g, inv_tau_h;
    float Fx, Fy, grx, gry, dpux, dpuy, nx, ny, Fhat;
};

// D2Q9 sums written out term by term.  A loop over i with coefficients c_ix, c_iy
// would multiply by zero for the directions without that component, which IEEE
// arithmetic does not let the compiler drop.
//   first moment: (sum_i c_ix q_i, sum_i c_iy q_i)
__device__ __forceinline__ void dq9_moment1(const float* q, float& mx, float& my)
{
    const float a = q[5] - q[7], b = q[8] - q[6];  // c_5 = (1,1) vs c_7, c_8 = (1,-1) vs c_6
    mx = (q[1] - q[3]) + (a + b);
    my = (q[2] - q[4]) + (a - b);
}
//   isotropic gradient: sum_i w_i c_i X_i / cs2 = (X_1 - X_3)/3 + (X_5 - X_7 + X_8 - X_6)/12, ...
__device__ __forceinline__ void dq9_grad(const float* X, float& gx, float& gy)
{
    const float a = X[5] - X[7], b = X[8] - X[6];
    gx = fmaf(1.f / 3.f, X[1] - X[3], (1.f / 12.f) * (a + b));
    gy = fmaf(1.f / 3.f, X[2] - X[4], (1.f / 12.f) * (a - b));
}

// Per-node macroscopic state of one time level.  phin[i] and Tn[i] are phi and T at
// x + c_i (ghost values outside the fluid already applied), phin[0] = phi(x).
__device__ __forceinline__ Macro node_macro(const DevParams& P, const float* f, const float* g,
                                            const float* h, const float* phin, const float* Tn,
                                            float pux_prev, float puy_prev)
{
    Macro m;
    const float phi = phin[0], T = Tn[0];
    m.phi = phi;
    m.T = T;
    // isotropic stencils: grad X = sum w_i c_i X_i / cs2, lap X = sum 2 w_i (X_i - X_0) / cs2
    float gpx, gpy, gtx, gty;
    dq9_grad(phin, gpx, gpy);
    dq9_grad(Tn, gtx, gty);
    const float lap_axis = ((phin[1] - phi) + (phin[3] - phi)) + ((phin[2] - phi) + (phin[4] - phi));
    const float lap_diag = ((phin[5] - phi) + (phin[7] - phi)) + ((phin[6] - phi) + (phin[8] - phi));
    const float lap = fmaf(2.f / 3.f, lap_axis, (1.f / 6.f) * lap_diag);

    // closures, Eq. 45
    const float pc = clamp1(phi);
    const float rho = fmaf(P.rho_b, pc, P.rho_a);
    const float mu = fmaf(P.mu_b, pc, P.mu_a);
    const float lam = fmaf(P.lam_b, pc, P.lam_a);
    const float rcp = fmaf(P.rcp_b, pc, P.rcp_a);
    // correctly rounded reciprocals instead of divisions
    const float inv_rho = __frcp_rn(rho);
    const float tau_g = mu * kInvCs2 * inv_rho + 0.5f;
    const float tau_h = lam * kInvCs2 + 0.5f;
    m.rho = rho;
    m.rcp = rcp;
    m.inv_tau_g = __frcp_rn(tau_g);
    m.src_g = 1.f - 0.5f * m.inv_tau_g;
    m.inv_tau_h = __frcp_rn(tau_h);

    // surface tension law and its T derivative
    float sig, dsig;
    if (P.sigma_law == 1) {
        const float dT = T - P.T_ref;
        sig = 0.5f * P.sigma_TT * dT * dT + P.sigma_ref;
        dsig = P.sigma_TT * dT;
    } else {
        sig = P.sigma_ref + P.sigma_T * (T - P.T_ref);
        dsig = P.sigma_T;
    }
    // chemical potential with phi_l = -1, phi_h = 1
    const float mu_phi = (phi + 1.f) * (phi - 1.f) * phi - P.W2 * lap;
    // interfacial force, last line of Eq. 11
    const float gsx = dsig * gtx, gsy = dsig * gty;
    const float g2 = gpx * gpx + gpy * gpy;
    const float sp = gsx * gpx + gsy * gpy;
    const float cm = sig * mu_phi * P.inv_W2;
    const float Fx = P.kFs * (g2 * gsx - sp * gpx + cm * gpx) + P.Gx;
    const float Fy = P.kFs * (g2 * gsy - sp * gpy + cm * gpy) + P.Gy;
    m.Fx = Fx;
    m.Fy = Fy;

    // velocity and pressure moments of the NS populations
    float mx, my;
    dq9_moment1(g, mx, my);
    const float sne0 = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
    const float ux = (mx + 0.5f * Fx) * inv_rho;
    const float uy = (my + 0.5f * Fy) * inv_rho;
    const float grx = P.drho_dphi * gpx, gry = P.drho_dphi * gpy;
    const float uu = ux * ux + uy * uy;
    const float s0 = wq(0) * (-0.5f * kInvCs2 * uu);
    m.p = kCs2 / (1.f - wq(0)) * (sne0 + 0.5f * (ux * grx + uy * gry) + rho * s0);
    m.ux = ux;
    m.uy = uy;
    m.grx = grx;
    m.gry = gry;

    // d_t(phi u), first-order Euler (Eq. 44)
    m.dpux = phi * ux - pux_prev;
    m.dpuy = phi * uy - puy_prev;

    // unit normal; zero where |grad phi| <= 1e-10
    float nvx = gpx, nvy = gpy, nthr = 1e-20f;
    if (P.normal_law == 1) {
        // local recovery (Sec. 3): J = sum_i c_i (f_i - f_i^eq) + d_t(phi u)/2 =
        // -cs2 tau_phi grad phi + M_phi Theta n, so n = -J/|J|; sum_i c_i f_i^eq = phi u
        float jx, jy;
        dq9_moment1(f, jx, jy);
        nvx = -(jx + 0.5f * m.dpux - phi * ux);
        nvy = -(jy + 0.5f * m.dpuy - phi * uy);
        nthr = P.jthr2;
    }
    const float gn2 = nvx * nvx + nvy * nvy;
    if (gn2 > nthr) {
        const float r = rsqrtf(gn2);
        m.nx = nvx * r;
        m.ny = nvy * r;
    } else {
        m.nx = 0.f;
        m.ny = 0.f;
    }

    // local grad T from the non-equilibrium part of h (Eq. 40), thermal source of Eq. 27
    float qx, qy;
    dq9_moment1(h, qx, qy);
    const float k = -m.inv_tau_h * kInvCs2;
    m.Fhat = -rcp * (ux * qx + uy * qy) * k;
    return m;
}

// Equilibria of the three LBEs (Sec. 3.1 f^eq and g^eq, Eq. 31 h^eq).  The rest
// populations are formed as the remainder of the moving ones (sum f^eq = phi,
// sum g^eq = 0, sum h^eq = T), which is the printed form because the weights sum
// to one; in float32 the rounded weights sum to 1 + 7.5e-9, and the printed form
// would then create phi and T at that rate every step.
__device__ __forceinline__ void node_equilibria_(float phi, float rho, float ux, float uy, float p, float T,
                                                 float* feq, float* geq, float* heq)
{
    const float uu = ux * ux + uy * uy;
    const float pcs = p * kInvCs2;
    float sf = 0.f, sg = 0.f, sh = 0.f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy;
        feq[i] = wq(i) * phi * (1.f + cu * kInvCs2);
        const float si = wq(i) * (cu * kInvCs2 + 0.5f * cu * cu * kInvCs2 * kInvCs2 - 0.5f * uu * kInvCs2);
        geq[i] = pcs * wq(i) + rho * si;
        heq[i] = wq(i) * T;
        sf += feq[i];
        sg += geq[i];
        sh += heq[i];
    }
    feq[0] = phi - sf;
    geq[0] = -sg;
    heq[0] = T - sh;
}

// Two-relaxation-time collisions of g and h (the stability extension of Sec. 3): with
// X^{+/-} = (X_i +/- X_opp(i)) / 2, the even part relaxes at om_p, the odd part at om_m,
// (tau_p - 1/2)(tau_m - 1/2) = Lambda; the viscosity stays on the even part of g
// (tau_p = tau_g), the conductivity on the odd part of h (tau_m = tau_h).
__device__ __forceinline__ void node_collide_trt_gh(const DevParams& P, const Macro& m, float* g, float* h)
{
    const float ux = m.ux, uy = m.uy;
    const float FxC = m.Fx * kInvCs2, FyC = m.Fy * kInvCs2;
    const float Fh = m.Fhat;
    float feq[9], geq[9], heq[9], Gs[9];
    node_equilibria_(m.phi, m.rho, ux, uy, m.p, m.T, feq, geq, heq);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy;
        const float cg = cx(i) * m.grx + cy(i) * m.gry;
        Gs[i] = wq(i) * (cx(i) * FxC + cy(i) * FyC + cu * cg * kInvCs2);
    }
    const float og_p = m.inv_tau_g;
    const float og_m = __frcp_rn(0.5f + P.trt_lambda * __frcp_rn(__frcp_rn(og_p) - 0.5f));
    const float oh_m = m.inv_tau_h;
    const float oh_p = __frcp_rn(0.5f + P.trt_lambda * __frcp_rn(__frcp_rn(oh_m) - 0.5f));
    const float cg_p = 1.f - 0.5f * og_p, cg_m = 1.f - 0.5f * og_m;
    g[0] = g[0] + (geq[0] - g[0]) * og_p + cg_p * Gs[0];
    h[0] = h[0] + (heq[0] - h[0]) * oh_p + wq(0) * Fh;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int o = opp(i);
        if (o < i) continue;  // each pair once
        const float gp = 0.5f * (g[i] + g[o]), gm = 0.5f * (g[i] - g[o]);
        const float ep = 0.5f * (geq[i] + geq[o]), em = 0.5f * (geq[i] - geq[o]);
        const float sp = 0.5f * (Gs[i] + Gs[o]), sm = 0.5f * (Gs[i] - Gs[o]);
        const float dp = (ep - gp) * og_p + cg_p * sp, dm = (em - gm) * og_m + cg_m * sm;
        g[i] = g[i] + dp + dm;
        g[o] = g[o] + dp - dm;
        const float hp = 0.5f * (h[i] + h[o]), hm = 0.5f * (h[i] - h[o]);
        const float hep = 0.5f * (heq[i] + heq[o]), hem = 0.5f * (heq[i] - heq[o]);
        const float hdp = (hep - hp) * oh_p + wq(i) * Fh, hdm = (hem - hm) * oh_m;
        h[i] = h[i] + hdp + hdm;
        h[o] = h[o] + hdp - hdm;
    }
}

// Collisions of the three LBEs at one node (Eq. 14, Sec. 3.1 NS LBE, Eq. 28 collision
// part); overwrites f, g, h with the post-collision populations.  BGK q_i* = q_i +
// om (q_i^eq - q_i) + c S_i is evaluated as (1 - om) q_i + w_i t_i, where t_i collects
// the relaxed equilibrium and the source of direction i:
//   f: t_i = om phi + c_i . (3 om phi u + (1 - om/2) a),  R_i = w_i c_i . a,
//      a = 3 d_t(phi u) + n (1 - phi^2) / (sqrt2 W)
//   g: t_i = om (3 p - 3/2 rho u.u) + c_i . 3 (om rho u + (1 - om/2) F)
//            + (c_i.u) (9/2 om rho (c_i.u) + 3 (1 - om/2) (c_i . grad rho))
//      (G_i = w_i [3 c_i . F + 3 (c_i.u)(c_i . grad rho)], its u.grad rho terms cancel)
//   h: t_i = om T + Fhat
// Opposite directions share c_i.u c_i.u and (c_i.u)(c_i.grad rho).  The rest
// populations of f and h are the remainders that keep sum_i f_i* = phi and
// sum_i h_i* = T + Fhat exactly in exact arithmetic (the float32 weights sum to
// 1 + 7.5e-9, which would otherwise create phi and T every step); g_0 enters no
// moment, its equilibrium is the printed one.
__device__ __forceinline__ void node_collide(const DevParams& P, const Macro& m, float* f, float* g, float* h)
{
    constexpr float w1 = 1.f / 9.f, w5 = 1.f / 36.f;
    const float ux = m.ux, uy = m.uy;
    // Allen-Cahn
    {
        const float om = P.inv_tau_phi, k = 1.f - om;
        const float theta = (1.f - m.phi * m.phi) * P.theta_k;
        const float ax = fmaf(3.f, m.dpux, m.nx * theta), ay = fmaf(3.f, m.dpuy, m.ny * theta);
        const float A = om * m.phi, c3 = 3.f * A;
        const float Bx = fmaf(c3, ux, P.src_phi * ax), By = fmaf(c3, uy, P.src_phi * ay);
        const float a1 = w1 * A, bx1 = w1 * Bx, by1 = w1 * By;
        const float a5 = w5 * A, bp5 = w5 * (Bx + By), bm5 = w5 * (Bx - By);
        f[1] = fmaf(k, f[1], a1 + bx1);
        f[3] = fmaf(k, f[3], a1 - bx1);
        f[2] = fmaf(k, f[2], a1 + by1);
        f[4] = fmaf(k, f[4], a1 - by1);
        f[5] = fmaf(k, f[5], a5 + bp5);
        f[7] = fmaf(k, f[7], a5 - bp5);
        f[8] = fmaf(k, f[8], a5 + bm5);
        f[6] = fmaf(k, f[6], a5 - bm5);
        f[0] = m.phi - (((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
    }
    if (P.collision == 1) {
        node_collide_trt_gh(P, m, g, h);
        return;
    }
    // Navier-Stokes
    {
        const float om = m.inv_tau_g, k = 1.f - om, sg = m.src_g;
        const float orho = om * m.rho;
        const float P0 = om * fmaf(-1.5f * m.rho, ux * ux + uy * uy, 3.f * m.p);
        const float Vx = 3.f * fmaf(orho, ux, sg * m.Fx), Vy = 3.f * fmaf(orho, uy, sg * m.Fy);
        const float K1 = 4.5f * orho, K2 = 3.f * sg;
        // pair (i, o): t_i = P0 + Q + c_i.V, t_o = P0 + Q - c_i.V, Q = cu (K1 cu + K2 cg)
        auto pair = [&](int i, int o, float w, float cu, float cg, float cv) {
            const float base = fmaf(cu, fmaf(K1, cu, K2 * cg), P0);
            g[i] = fmaf(k, g[i], w * (base + cv));
            g[o] = fmaf(k, g[o], w * (base - cv));
        };
        pair(1, 3, w1, ux, m.grx, Vx);
        pair(2, 4, w1, uy, m.gry, Vy);
        pair(5, 7, w5, ux + uy, m.grx + m.gry, Vx + Vy);
        pair(8, 6, w5, ux - uy, m.grx - m.gry, Vx - Vy);
        // g_0^eq = (w_0 - 1) p / cs2 + rho w_0 (-u.u / (2 cs2)), G_0 = 0
        g[0] = fmaf(k, g[0], om * (-(5.f / 3.f) * m.p - (2.f / 3.f) * m.rho * (ux * ux + uy * uy)));
    }
    // thermal, source w_i Fhat
    {
        const float om = m.inv_tau_h, k = 1.f - om;
        const float t = fmaf(om, m.T, m.Fhat);
        const float t1 = w1 * t, t5 = w5 * t;
        h[1] = fmaf(k, h[1], t1);
        h[2] = fmaf(k, h[2], t1);
        h[3] = fmaf(k, h[3], t1);
        h[4] = fmaf(k, h[4], t1);
        h[5] = fmaf(k, h[5], t5);
        h[6] = fmaf(k, h[6], t5);
        h[7] = fmaf(k, h[7], t5);
        h[8] = fmaf(k, h[8], t5);
        h[0] = (m.T + m.Fhat) - (((h[1] + h[2]) + (h[3] + h[4])) + ((h[5] + h[6]) + (h[7] + h[8])));
    }
}

// Equilibrium populations of a node from macroscopic values (initial state).
__device__ __forceinline__ void node_equilibria(const DevParams& P, float phi, float ux, float uy, float p,
                                                float T, float* f, float* g, float* h)
{
    const float rho = fmaf(P.rho_b, clamp1(phi), P.rho_a);
    node_equilibria_(phi, rho, ux, uy, p, T, f, g, h);
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// phi and T at lattice point (gx, gy), at most one step outside the fluid.
// get(x, y, phi, T) returns the values of an interior node.  Ghost rules: phi is
// mirrored across walls, inlet and outflow (zero normal gradient); T = 2 T_wall - T
// across walls, 2 T_in - T across the inlet, zero gradient across the outflow.
template <class Get>
__device__ __forceinline__ void phiT_at(const DevParams& P, int gx, int gy, Get get, float& phi, float& T)
{
    int x = gx, y = gy;
    if (P.bc_x == 0) x = wrap(x, P.nx);
    if (P.bc_y == 1) y = wrap(y, P.ny);
    const bool ox = x < 0 || x >= P.nx;
    const bool oy = y < 0 || y >= P.ny;
    const int mx = ox ? (x < 0 ? 0 : P.nx - 1) : x;
    const int my = oy ? (y < 0 ? 0 : P.ny - 1) : y;
    float ph, tm;
    get(mx, my, ph, tm);
    phi = ph;
    float tx = tm;
    if (ox && x < 0) tx = 2.f * P.T_in - tm;
    if (oy) T = 2.f * (y < 0 ? T_wall_bottom(P, (float)gx) : T_wall_top(P, (float)gx)) - tx;
    else T = tx;
}

}  // namespace tpf
