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
    float gpx = 0.f, gpy = 0.f, lap = 0.f, gtx = 0.f, gty = 0.f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        gpx += wq(i) * cx(i) * phin[i];
        gpy += wq(i) * cy(i) * phin[i];
        lap += wq(i) * (phin[i] - phi);
        gtx += wq(i) * cx(i) * Tn[i];
        gty += wq(i) * cy(i) * Tn[i];
    }
    gpx *= kInvCs2; gpy *= kInvCs2; lap *= 2.f * kInvCs2; gtx *= kInvCs2; gty *= kInvCs2;

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
    float mx = 0.f, my = 0.f, sne0 = 0.f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        mx += cx(i) * g[i];
        my += cy(i) * g[i];
        sne0 += g[i];
    }
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
        float jx = 0.5f * m.dpux - phi * ux, jy = 0.5f * m.dpuy - phi * uy;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (cx(i) != 0) jx += (float)cx(i) * f[i];
            if (cy(i) != 0) jy += (float)cy(i) * f[i];
        }
        nvx = -jx;
        nvy = -jy;
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
    float qx = 0.f, qy = 0.f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        qx += cx(i) * h[i];
        qy += cy(i) * h[i];
    }
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

// BGK collisions of the three LBEs at one node (Eq. 14, Sec. 3.1 NS LBE, Eq. 28
// collision part).  Overwrites f, g, h with the post-collision populations.
__device__ __forceinline__ void node_collide(const DevParams& P, const Macro& m, float* f, float* g, float* h)
{
    const float ux = m.ux, uy = m.uy;
    const float theta = (1.f - m.phi * m.phi) * P.theta_k;
    const float ax = (m.dpux + kCs2 * m.nx * theta) * kInvCs2;
    const float ay = (m.dpuy + kCs2 * m.ny * theta) * kInvCs2;
    const float FxC = m.Fx * kInvCs2, FyC = m.Fy * kInvCs2;
    const float Fh = m.Fhat;
    float feq[9], geq[9], heq[9];
    node_equilibria_(m.phi, m.rho, ux, uy, m.p, m.T, feq, geq, heq);
    float Gs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy;
        // Allen-Cahn with source R_i
        const float Ri = wq(i) * (cx(i) * ax + cy(i) * ay);
        f[i] = f[i] + (feq[i] - f[i]) * P.inv_tau_phi + P.src_phi * Ri;
        // Navier-Stokes forcing; its u.grad rho terms cancel:
        // G_i = w_i [ c_i.(Fs + G)/cs2 + (c_i.u)(c_i.grad rho)/cs2 ]
        const float cg = cx(i) * m.grx + cy(i) * m.gry;
        Gs[i] = wq(i) * (cx(i) * FxC + cy(i) * FyC + cu * cg * kInvCs2);
    }
    if (P.collision == 1) {
        // two relaxation times (the stability extension of Sec. 3) for g and h: with
        // X^{+/-} = (X_i +/- X_opp(i)) / 2, the even part relaxes at om_p, the odd part at
        // om_m, (tau_p - 1/2)(tau_m - 1/2) = Lambda; the viscosity stays on the even part
        // of g (tau_p = tau_g), the conductivity on the odd part of h (tau_m = tau_h)
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
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            g[i] = g[i] + (geq[i] - g[i]) * m.inv_tau_g + m.src_g * Gs[i];
            // thermal with source w_i Fhat
            h[i] = h[i] + (heq[i] - h[i]) * m.inv_tau_h + wq(i) * Fh;
        }
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
