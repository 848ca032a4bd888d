// Kernels and C-ABI of the tpflbm library (declarations and conventions in
// include/tpflbm.h).  One fused kernel advances the three coupled D2Q9 LBEs of
// arXiv 2306.11320 by one time step; the others initialise, read back and reduce.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/tpflbm.h"
#include "lattice.cuh"

using namespace tpf;

namespace {

// ------------------------------------------------------------- step kernel
//
// Push scheme on pre-collision state.  A CTA owns a BX x BY tile of nodes (one
// node per thread) and stages, for the tile plus a one-node ring, phi = sum f_i,
// T = sum h_i (ghost rules applied) and the pre-collision h_i in shared memory.
// Each thread then computes its node's macroscopic state (stencils from shared
// memory), collides the three LBEs, and writes every post-collision population to
// the node it streams to in buffer B.  The thermal update of Eq. 28 needs the
// destination's own h_i(y, t) and rho c_p(y), both found in shared memory because
// every destination lies in the tile or its ring.  Populations leaving through a
// wall, the inlet or the outflow plane are reflected into the node itself with the
// corresponding rule.  Every (direction, node) slot of B is written exactly once.

template <int BX, int BY, class S>
__global__ void __launch_bounds__(BX * BY)
k_step(const DevParams P, const typename S::elem* __restrict__ A, typename S::elem* __restrict__ B,
       float* __restrict__ phiu)
{
    constexpr int SX = BX + 2, SY = BY + 2, SN = SX * SY;
    __shared__ float s_phi[SN];
    __shared__ float s_T[SN];
    __shared__ float s_h[9][SN];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * BX + tx;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < P.nx && y < P.ny;
    const long long pl = P.plane;
    const long long n = (long long)y * P.nx + x;

    float f[9], g[9], h[9];
    if (active) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = S::ld(A, i * pl + n, P.is_f, 0.f);
            g[i] = S::ld(A, (9 + i) * pl + n, P.is_g, 0.f);
            h[i] = S::ld(A, (18 + i) * pl + n, P.is_h, wq(i) * P.X_h);
        }
        float sf = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            sf += f[i];
            sh += h[i];
        }
        const int k = (ty + 1) * SX + tx + 1;
        s_phi[k] = sf;
        s_T[k] = sh;
#pragma unroll
        for (int i = 0; i < 9; ++i) s_h[i][k] = h[i];
    }

    // phi, T and h of an interior node read straight from A
    auto get = [&](int gx, int gy, float& ph, float& tt) {
        const long long m = (long long)gy * P.nx + gx;
        float sf = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            sf += S::ld(A, i * pl + m, P.is_f, 0.f);
            sh += S::ld(A, (18 + i) * pl + m, P.is_h, wq(i) * P.X_h);
        }
        ph = sf;
        tt = sh;
    };

    // ring (and the unused part of ragged tiles)
    for (int k = tid; k < SN; k += BX * BY) {
        const int lx = k % SX, ly = k / SX;
        const bool own = lx >= 1 && lx <= BX && ly >= 1 && ly <= BY &&
                         (x0 + lx - 1) < P.nx && (y0 + ly - 1) < P.ny;
        if (own) continue;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        int wx = gx, wy = gy;
        if (P.bc_x == 0) wx = wrap(wx, P.nx);
        if (P.bc_y == 1) wy = wrap(wy, P.ny);
        const bool far = gx < -1 || gx > P.nx || gy < -1 || gy > P.ny;
        if (far) {
            s_phi[k] = 0.f;
            s_T[k] = 0.f;
            continue;
        }
        if (wx >= 0 && wx < P.nx && wy >= 0 && wy < P.ny) {
            const long long m = (long long)wy * P.nx + wx;
            float sf = 0.f, sh = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                sf += S::ld(A, i * pl + m, P.is_f, 0.f);
                const float hv = S::ld(A, (18 + i) * pl + m, P.is_h, wq(i) * P.X_h);
                sh += hv;
                s_h[i][k] = hv;
            }
            s_phi[k] = sf;
            s_T[k] = sh;
        } else {
            float ph, tt;
            phiT_at(P, gx, gy, get, ph, tt);
            s_phi[k] = ph;
            s_T[k] = tt;
        }
    }
    __syncthreads();
    if (!active) return;

    const int lx = tx + 1, ly = ty + 1;
    float phin[9], Tn[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int k = (ly + cy(i)) * SX + lx + cx(i);
        phin[i] = s_phi[k];
        Tn[i] = s_T[k];
    }
    const float pux = phiu[n], puy = phiu[pl + n];
    const Macro m = node_macro(P, f, g, h, phin, Tn, pux, puy);
    phiu[n] = m.phi * m.ux;
    phiu[pl + n] = m.phi * m.uy;

    node_collide(P, m, f, g, h);

    // streaming with the boundary rules
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int o = opp(i);
        int dx = x + cx(i), dy = y + cy(i);
        if (P.bc_x == 0) dx = wrap(dx, P.nx);
        if (P.bc_y == 1) dy = wrap(dy, P.ny);
        const bool out_y = dy < 0 || dy >= P.ny;
        const bool out_x = dx < 0 || dx >= P.nx;
        if (out_y) {
            // halfway bounce-back of f and g; anti-bounce-back of h with the wall
            // temperature at the link's crossing point
            const float xc = (float)x + 0.5f * cx(i);
            const float Tw = (cy(i) < 0) ? T_wall_bottom(P, xc) : T_wall_top(P, xc);
            S::st(B, o * pl + n, f[i], P.s_f, 0.f);
            S::st(B, (9 + o) * pl + n, g[i], P.s_g, 0.f);
            const float hold = s_h[o][ly * SX + lx];
            const float hin = -h[i] + 2.f * wq(o) * Tw;
            S::st(B, (18 + o) * pl + n, hold + (hin - hold) / m.rcp, P.s_h, wq(o) * P.X_h);
        } else if (out_x && dx < 0) {
            // velocity inlet: bounce-back carrying the inlet momentum and phi_in
            const float ycr = (float)y + 0.5f + 0.5f * cy(i);
            const float cu = cx(o) * u_inlet(P, ycr);
            S::st(B, o * pl + n, f[i] + 2.f * wq(o) * P.phi_in * cu * kInvCs2, P.s_f, 0.f);
            S::st(B, (9 + o) * pl + n, g[i] + 2.f * wq(o) * m.rho * cu * kInvCs2, P.s_g, 0.f);
            const float hold = s_h[o][ly * SX + lx];
            const float hin = -h[i] + 2.f * wq(o) * P.T_in;
            S::st(B, (18 + o) * pl + n, hold + (hin - hold) / m.rcp, P.s_h, wq(o) * P.X_h);
        } else if (out_x) {
            // outflow: pressure anti-bounce-back of g (f and h arrive by the copy below)
            const float cu = cx(o) * m.ux + cy(o) * m.uy;
            const float sym = P.p_out * kInvCs2 +
                              m.rho * (0.5f * cu * cu * kInvCs2 * kInvCs2 - 0.5f * (m.ux * m.ux + m.uy * m.uy) * kInvCs2);
            S::st(B, (9 + o) * pl + n, -g[i] + 2.f * wq(o) * sym, P.s_g, 0.f);
        } else {
            const long long d = (long long)dy * P.nx + dx;
            S::st(B, i * pl + d, f[i], P.s_f, 0.f);
            S::st(B, (9 + i) * pl + d, g[i], P.s_g, 0.f);
            const int kd = (ly + cy(i)) * SX + lx + cx(i);
            const float rcp_d = fmaf(P.rcp_b, clamp1(s_phi[kd]), P.rcp_a);
            const float hold = s_h[i][kd];
            S::st(B, (18 + i) * pl + d, hold + (h[i] - hold) / rcp_d, P.s_h, wq(i) * P.X_h);
        }
        // zero-gradient outflow of f and h: the ghost column beyond x = nx-1 carries
        // the post-collision populations of the last column
        if (P.bc_x == 1 && x == P.nx - 1 && cx(i) < 0) {
            const int ey = y + cy(i);
            if (ey >= 0 && ey < P.ny) {
                const long long d = (long long)ey * P.nx + x;
                S::st(B, i * pl + d, f[i], P.s_f, 0.f);
                const int kd = (ly + cy(i)) * SX + lx;
                const float rcp_d = fmaf(P.rcp_b, clamp1(s_phi[kd]), P.rcp_a);
                const float hold = s_h[i][kd];
                S::st(B, (18 + i) * pl + d, hold + (h[i] - hold) / rcp_d, P.s_h, wq(i) * P.X_h);
            }
        }
    }
}

// ------------------------------------------------------- auxiliary kernels

// Macroscopic state of node (x, y) read straight from global memory.
template <class S>
__device__ Macro macro_at(const DevParams& P, const typename S::elem* __restrict__ A,
                          const float* __restrict__ phiu, int x, int y)
{
    const long long pl = P.plane;
    const long long n = (long long)y * P.nx + x;
    float f[9], g[9], h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f[i] = S::ld(A, i * pl + n, P.is_f, 0.f);
        g[i] = S::ld(A, (9 + i) * pl + n, P.is_g, 0.f);
        h[i] = S::ld(A, (18 + i) * pl + n, P.is_h, wq(i) * P.X_h);
    }
    auto get = [&](int gx, int gy, float& ph, float& tt) {
        const long long m = (long long)gy * P.nx + gx;
        float sf = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            sf += S::ld(A, i * pl + m, P.is_f, 0.f);
            sh += S::ld(A, (18 + i) * pl + m, P.is_h, wq(i) * P.X_h);
        }
        ph = sf;
        tt = sh;
    };
    float phin[9], Tn[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) phiT_at(P, x + cx(i), y + cy(i), get, phin[i], Tn[i]);
    return node_macro(P, f, g, h, phin, Tn, phiu[n], phiu[pl + n]);
}

template <class S>
__global__ void k_fields(const DevParams P, const typename S::elem* __restrict__ A,
                         const float* __restrict__ phiu, float* __restrict__ out)
{
    const long long N = (long long)P.nx * P.ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
        const Macro m = macro_at<S>(P, A, phiu, x, y);
        out[n] = m.phi;
        out[P.plane + n] = m.ux;
        out[2 * P.plane + n] = m.uy;
        out[3 * P.plane + n] = m.p;
        out[4 * P.plane + n] = m.T;
    }
}

template <class S>
__global__ void k_init(const DevParams P, const float* __restrict__ in, typename S::elem* __restrict__ A,
                       float* __restrict__ phiu)
{
    const long long N = (long long)P.nx * P.ny;
    const long long pl = P.plane;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const float phi = in[n], ux = in[pl + n], uy = in[2 * pl + n], p = in[3 * pl + n], T = in[4 * pl + n];
        float f[9], g[9], h[9];
        node_equilibria(P, phi, ux, uy, p, T, f, g, h);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S::st(A, i * pl + n, f[i], P.s_f, 0.f);
            S::st(A, (9 + i) * pl + n, g[i], P.s_g, 0.f);
            S::st(A, (18 + i) * pl + n, h[i], P.s_h, wq(i) * P.X_h);
        }
        phiu[n] = phi * ux;
        phiu[pl + n] = phi * uy;
    }
}

// Convert one population plane between float32 staging and the storage format.
template <class S>
__global__ void k_plane_encode(const DevParams P, const float* __restrict__ in, typename S::elem* __restrict__ out,
                               float s, float ref)
{
    const long long N = (long long)P.nx * P.ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x)
        S::st(out, n, in[n], s, ref);
}
template <class S>
__global__ void k_plane_decode(const DevParams P, const typename S::elem* __restrict__ in, float* __restrict__ out,
                               float is, float ref)
{
    const long long N = (long long)P.nx * P.ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x)
        out[n] = S::ld(in, n, is, ref);
}

// FP64 reductions (see tpflbm_diagnostics).  Each block writes 8 partial sums;
// k_reduce_final adds the partials of all blocks in a fixed order.
constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;

template <class S>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_partial(const DevParams P, const typename S::elem* __restrict__ A, const float* __restrict__ phiu,
                 double* __restrict__ partial)
{
    const long long N = (long long)P.nx * P.ny;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
        const Macro m = macro_at<S>(P, A, phiu, x, y);
        acc[0] += m.phi;
        acc[1] += (double)m.rcp * m.T;
        acc[2] += m.T;
        if (m.phi < 0.f) {
            acc[3] += (double)m.phi * m.uy;
            acc[4] += m.phi;
            acc[5] += (double)m.phi * m.ux;
            acc[6] += (double)m.phi * x;
        }
        if (!isfinite(m.phi) || !isfinite(m.ux) || !isfinite(m.uy) || !isfinite(m.T)) acc[7] += 1.0;
    }
    __shared__ double red[8][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += red[threadIdx.x][w];
        partial[blockIdx.x * 8 + threadIdx.x] = v;
    }
}

__global__ void k_reduce_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out)
{
    if (threadIdx.x < 8) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partial[b * 8 + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

}  // namespace

// ===================================================================== host

struct tpflbm {
    int nx = 0, ny = 0;
    tpflbm_params hp{};
    DevParams dp{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool owns = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* popA = nullptr;
    void* popB = nullptr;
    float* phiu = nullptr;
    float* fields = nullptr;  // 5 planes of float staging
    double* red = nullptr;    // kRedMaxBlocks * 8 partials + 8 results
    long long t = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

constexpr int kBX = 32, kBY = 8;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

long long plane_of(int nx, int ny) { return (((long long)nx * ny + 63) / 64) * 64; }

struct Layout {
    size_t popA, popB, phiu, fields, red, total;
};

Layout layout_of(int nx, int ny, int storage)
{
    const long long pl = plane_of(nx, ny);
    const size_t e = storage == TPF_STORAGE_FP16 ? 2 : 4;
    Layout L{};
    size_t off = 0;
    L.popA = off; off = align256(off + 27 * (size_t)pl * e);
    L.popB = off; off = align256(off + 27 * (size_t)pl * e);
    L.phiu = off; off = align256(off + 2 * (size_t)pl * 4);
    L.fields = off; off = align256(off + 5 * (size_t)pl * 4);
    L.red = off; off = align256(off + (kRedMaxBlocks * 8 + 8) * sizeof(double));
    L.total = off;
    return L;
}

int fail(tpflbm_t h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(tpflbm_t h, cudaError_t e, const char* what)
{
    return fail(h, TPF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TPF_CUDA(h, call)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);   \
    } while (0)

float pow2_scale(double requested, double fallback)
{
    double s = requested > 0 ? requested : fallback;
    return (float)std::exp2(std::round(std::log2(s)));
}

int validate(int nx, int ny, const tpflbm_params* p, std::string& why)
{
    if (!p) { why = "params is NULL"; return TPF_ERR_INVALID_ARG; }
    if (nx < 3 || ny < 3) { why = "nx and ny must be >= 3"; return TPF_ERR_INVALID_ARG; }
    if ((long long)nx * ny > (1LL << 31)) { why = "lattice too large"; return TPF_ERR_INVALID_ARG; }
    if (p->storage != TPF_STORAGE_FP32 && p->storage != TPF_STORAGE_FP16) { why = "unknown storage"; return TPF_ERR_INVALID_ARG; }
    if (p->bc_x < 0 || p->bc_x > 1 || p->bc_y < 0 || p->bc_y > 1) { why = "bc_x/bc_y must be 0 or 1"; return TPF_ERR_INVALID_ARG; }
    if (p->sigma_law < 0 || p->sigma_law > 1) { why = "sigma_law must be 0 or 1"; return TPF_ERR_INVALID_ARG; }
    if (!(p->rho_l > 0 && p->rho_h > 0)) { why = "densities must be positive"; return TPF_ERR_INVALID_ARG; }
    if (!(p->mu_l > 0 && p->mu_h > 0 && p->lambda_l > 0 && p->lambda_h > 0)) { why = "mu and lambda must be positive (tau > 1/2)"; return TPF_ERR_INVALID_ARG; }
    if (!(p->cp_l > 0 && p->cp_h > 0)) { why = "heat capacities must be positive"; return TPF_ERR_INVALID_ARG; }
    if (!(p->M_phi > 0) || !(p->W > 0)) { why = "M_phi and W must be positive"; return TPF_ERR_INVALID_ARG; }
    if (p->bc_x == 1 && p->bc_y == 1) { why = "an inlet/outflow channel needs walls (bc_y = 0)"; return TPF_ERR_INVALID_ARG; }
    return TPF_OK;
}

DevParams make_dev_params(int nx, int ny, const tpflbm_params& p)
{
    DevParams d{};
    d.nx = nx; d.ny = ny; d.bc_x = p.bc_x; d.bc_y = p.bc_y; d.sigma_law = p.sigma_law; d.storage = p.storage;
    d.plane = plane_of(nx, ny);
    auto ab = [](double l, double h, float& a, float& b) { a = (float)(0.5 * (l + h)); b = (float)(0.5 * (h - l)); };
    ab(p.rho_l, p.rho_h, d.rho_a, d.rho_b);
    ab(p.mu_l, p.mu_h, d.mu_a, d.mu_b);
    ab(p.lambda_l, p.lambda_h, d.lam_a, d.lam_b);
    ab(p.rho_l * p.cp_l, p.rho_h * p.cp_h, d.rcp_a, d.rcp_b);
    d.drho_dphi = (float)(0.5 * (p.rho_h - p.rho_l));
    d.W2 = (float)(p.W * p.W);
    d.inv_W2 = (float)(1.0 / (p.W * p.W));
    d.theta_k = (float)(1.0 / (std::sqrt(2.0) * p.W));
    d.kFs = (float)(3.0 * std::sqrt(2.0) * p.W / 4.0);
    const double tau_phi = p.M_phi * 3.0 + 0.5;
    d.inv_tau_phi = (float)(1.0 / tau_phi);
    d.src_phi = (float)(1.0 - 0.5 / tau_phi);
    d.sigma_ref = (float)p.sigma_ref; d.sigma_T = (float)p.sigma_T; d.sigma_TT = (float)p.sigma_TT; d.T_ref = (float)p.T_ref;
    d.Gx = (float)p.Gx; d.Gy = (float)p.Gy;
    d.u_ave = (float)p.u_ave; d.phi_in = (float)p.phi_in; d.T_in = (float)p.T_in; d.p_out = (float)p.p_out;
    d.T_bot = (float)p.T_bot; d.T_bot_amp = (float)p.T_bot_amp; d.T_bot_k = (float)p.T_bot_k;
    d.T_bot_slope = (float)p.T_bot_slope; d.T_top = (float)p.T_top; d.T_top_slope = (float)p.T_top_slope;
    if (p.storage == TPF_STORAGE_FP16) {
        d.s_f = pow2_scale(p.fp16_scale_f, 1.0);
        d.s_g = pow2_scale(p.fp16_scale_g, 1024.0);
        d.s_h = pow2_scale(p.fp16_scale_h, 1.0);
        d.X_h = (float)p.fp16_ref_T;
    } else {
        d.s_f = d.s_g = d.s_h = 1.f;
        d.X_h = 0.f;
    }
    d.is_f = 1.f / d.s_f; d.is_g = 1.f / d.s_g; d.is_h = 1.f / d.s_h;
    return d;
}

int grid_1d(long long N)
{
    long long b = (N + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

int finish_create(tpflbm_t h, int nx, int ny, const tpflbm_params* p, void* ws, size_t bytes, bool owns)
{
    h->nx = nx; h->ny = ny; h->hp = *p;
    h->dp = make_dev_params(nx, ny, *p);
    cudaGetDevice(&h->device);
    const Layout L = layout_of(nx, ny, p->storage);
    h->ws = ws; h->ws_bytes = bytes; h->owns = owns;
    char* b = (char*)ws;
    h->popA = b + L.popA;
    h->popB = b + L.popB;
    h->phiu = (float*)(b + L.phiu);
    h->fields = (float*)(b + L.fields);
    h->red = (double*)(b + L.red);
    return TPF_OK;
}

template <class S>
void launch_step(tpflbm_t h)
{
    const DevParams& P = h->dp;
    dim3 blk(kBX, kBY), grd((P.nx + kBX - 1) / kBX, (P.ny + kBY - 1) / kBY);
    k_step<kBX, kBY, S><<<grd, blk, 0, h->stream>>>(P, (const typename S::elem*)h->popA,
                                                  (typename S::elem*)h->popB, h->phiu);
    std::swap(h->popA, h->popB);
}

// copy a [ny][nx] float field (host or device) into staging plane k
int stage_in(tpflbm_t h, const float* src, int k, float fill)
{
    const long long N = (long long)h->nx * h->ny;
    float* dst = h->fields + k * h->dp.plane;
    if (!src) {
        if (fill == 0.f) {
            TPF_CUDA(h, cudaMemsetAsync(dst, 0, N * sizeof(float), h->stream));
        } else {
            // fill with a constant through a tiny host buffer round
            float* tmp = new (std::nothrow) float[N];
            if (!tmp) return fail(h, TPF_ERR_OOM, "host allocation failed");
            for (long long i = 0; i < N; ++i) tmp[i] = fill;
            cudaError_t e = cudaMemcpyAsync(dst, tmp, N * sizeof(float), cudaMemcpyHostToDevice, h->stream);
            cudaError_t e2 = cudaStreamSynchronize(h->stream);
            delete[] tmp;
            if (e != cudaSuccess) return cuda_fail(h, e, "stage fill");
            if (e2 != cudaSuccess) return cuda_fail(h, e2, "stage fill sync");
        }
        return TPF_OK;
    }
    TPF_CUDA(h, cudaMemcpyAsync(dst, src, N * sizeof(float), cudaMemcpyDefault, h->stream));
    return TPF_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

size_t tpflbm_workspace_bytes(int nx, int ny, const tpflbm_params* p)
{
    std::string why;
    if (validate(nx, ny, p, why) != TPF_OK) return 0;
    return layout_of(nx, ny, p->storage).total;
}

int tpflbm_create(int nx, int ny, const tpflbm_params* p, tpflbm_t* out)
{
    if (!out) return fail(nullptr, TPF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    int rc = validate(nx, ny, p, why);
    if (rc != TPF_OK) return fail(nullptr, rc, why);
    const size_t bytes = layout_of(nx, ny, p->storage).total;
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? TPF_ERR_OOM : TPF_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    tpflbm_t h = new (std::nothrow) tpflbm;
    if (!h) {
        cudaFree(ws);
        return fail(nullptr, TPF_ERR_OOM, "host allocation failed");
    }
    finish_create(h, nx, ny, p, ws, bytes, true);
    *out = h;
    return TPF_OK;
}

int tpflbm_create_in(int nx, int ny, const tpflbm_params* p, void* workspace, size_t bytes, tpflbm_t* out)
{
    if (!out) return fail(nullptr, TPF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    int rc = validate(nx, ny, p, why);
    if (rc != TPF_OK) return fail(nullptr, rc, why);
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(nullptr, TPF_ERR_INVALID_ARG, "workspace must be 256-byte aligned device memory");
    if (bytes < layout_of(nx, ny, p->storage).total) return fail(nullptr, TPF_ERR_INVALID_ARG, "workspace too small");
    tpflbm_t h = new (std::nothrow) tpflbm;
    if (!h) return fail(nullptr, TPF_ERR_OOM, "host allocation failed");
    finish_create(h, nx, ny, p, workspace, bytes, false);
    *out = h;
    return TPF_OK;
}

int tpflbm_set_stream(tpflbm_t h, void* stream)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return TPF_OK;
}

int tpflbm_init(tpflbm_t h, const float* phi, const float* ux, const float* uy, const float* p, const float* T)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    const float* src[5] = {phi, ux, uy, p, T};
    for (int k = 0; k < 5; ++k) {
        int rc = stage_in(h, src[k], k, k == 0 ? 1.f : 0.f);
        if (rc) return rc;
    }
    const long long N = (long long)h->nx * h->ny;
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_init<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->fields, (__half*)h->popA, h->phiu);
    else
        k_init<StoreF32><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->fields, (float*)h->popA, h->phiu);
    TPF_CUDA(h, cudaGetLastError());
    // init reads the caller's buffers asynchronously: finish before returning
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->t = 0;
    return TPF_OK;
}

int tpflbm_step(tpflbm_t h, long long nsteps)
{
    if (!h || nsteps < 0) return TPF_ERR_INVALID_ARG;
    for (long long s = 0; s < nsteps; ++s) {
        if (h->dp.storage == TPF_STORAGE_FP16) launch_step<StoreF16>(h);
        else launch_step<StoreF32>(h);
    }
    TPF_CUDA(h, cudaGetLastError());
    h->t += nsteps;
    return TPF_OK;
}

int tpflbm_get_fields(tpflbm_t h, float* phi, float* ux, float* uy, float* p, float* T)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    const long long N = (long long)h->nx * h->ny;
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_fields<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const __half*)h->popA, h->phiu, h->fields);
    else
        k_fields<StoreF32><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const float*)h->popA, h->phiu, h->fields);
    TPF_CUDA(h, cudaGetLastError());
    float* dst[5] = {phi, ux, uy, p, T};
    for (int k = 0; k < 5; ++k)
        if (dst[k])
            TPF_CUDA(h, cudaMemcpyAsync(dst[k], h->fields + k * h->dp.plane, N * sizeof(float), cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    return TPF_OK;
}

int tpflbm_get_state(tpflbm_t h, float* f, float* g, float* hh, float* phiu)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    const long long N = (long long)h->nx * h->ny;
    const long long pl = h->dp.plane;
    float* dsts[3] = {f, g, hh};
    const float iss[3] = {h->dp.is_f, h->dp.is_g, h->dp.is_h};
    for (int k = 0; k < 3; ++k) {
        if (!dsts[k]) continue;
        for (int i = 0; i < 9; ++i) {
            const int q = 9 * k + i;
            float* dst = dsts[k] + (long long)i * N;
            if (h->dp.storage == TPF_STORAGE_FP32) {
                TPF_CUDA(h, cudaMemcpyAsync(dst, (float*)h->popA + q * pl, N * 4, cudaMemcpyDefault, h->stream));
            } else {
                const float ref = k == 2 ? wq(i) * h->dp.X_h : 0.f;
                k_plane_decode<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const __half*)h->popA + q * pl,
                                                                          h->fields, iss[k], ref);
                TPF_CUDA(h, cudaGetLastError());
                TPF_CUDA(h, cudaMemcpyAsync(dst, h->fields, N * 4, cudaMemcpyDefault, h->stream));
                TPF_CUDA(h, cudaStreamSynchronize(h->stream));
            }
        }
    }
    if (phiu) {
        TPF_CUDA(h, cudaMemcpyAsync(phiu, h->phiu, N * 4, cudaMemcpyDefault, h->stream));
        TPF_CUDA(h, cudaMemcpyAsync(phiu + N, h->phiu + pl, N * 4, cudaMemcpyDefault, h->stream));
    }
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    return TPF_OK;
}

int tpflbm_set_state(tpflbm_t h, const float* f, const float* g, const float* hh, const float* phiu)
{
    if (!h || !f || !g || !hh || !phiu) return fail(h, TPF_ERR_INVALID_ARG, "set_state needs f, g, h and phiu");
    const long long N = (long long)h->nx * h->ny;
    const long long pl = h->dp.plane;
    const float* srcs[3] = {f, g, hh};
    const float ss[3] = {h->dp.s_f, h->dp.s_g, h->dp.s_h};
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i < 9; ++i) {
            const int q = 9 * k + i;
            const float* src = srcs[k] + (long long)i * N;
            if (h->dp.storage == TPF_STORAGE_FP32) {
                TPF_CUDA(h, cudaMemcpyAsync((float*)h->popA + q * pl, src, N * 4, cudaMemcpyDefault, h->stream));
            } else {
                const float ref = k == 2 ? wq(i) * h->dp.X_h : 0.f;
                TPF_CUDA(h, cudaMemcpyAsync(h->fields, src, N * 4, cudaMemcpyDefault, h->stream));
                k_plane_encode<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->fields, (__half*)h->popA + q * pl,
                                                                          ss[k], ref);
                TPF_CUDA(h, cudaGetLastError());
            }
        }
    }
    TPF_CUDA(h, cudaMemcpyAsync(h->phiu, phiu, N * 4, cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaMemcpyAsync(h->phiu + pl, phiu + N, N * 4, cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    return TPF_OK;
}

int tpflbm_diagnostics(tpflbm_t h, double out[8])
{
    if (!h || !out) return TPF_ERR_INVALID_ARG;
    const long long N = (long long)h->nx * h->ny;
    long long b = (N + kRedThreads - 1) / kRedThreads;
    const int nb = (int)(b < kRedMaxBlocks ? b : kRedMaxBlocks);
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_reduce_partial<StoreF16><<<nb, kRedThreads, 0, h->stream>>>(h->dp, (const __half*)h->popA, h->phiu, h->red);
    else
        k_reduce_partial<StoreF32><<<nb, kRedThreads, 0, h->stream>>>(h->dp, (const float*)h->popA, h->phiu, h->red);
    TPF_CUDA(h, cudaGetLastError());
    double* res = h->red + kRedMaxBlocks * 8;
    k_reduce_final<<<1, 32, 0, h->stream>>>(h->red, nb, res);
    TPF_CUDA(h, cudaGetLastError());
    TPF_CUDA(h, cudaMemcpyAsync(out, res, 8 * sizeof(double), cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (out[7] > 0) return fail(h, TPF_ERR_NONFINITE, "non-finite values in the state");
    return TPF_OK;
}

long long tpflbm_time(tpflbm_t h) { return h ? h->t : -1; }

void tpflbm_destroy(tpflbm_t h)
{
    if (!h) return;
    if (h->owns && h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
    }
    delete h;
}

const char* tpflbm_last_error(tpflbm_t h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
