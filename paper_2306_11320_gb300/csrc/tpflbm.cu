// C-ABI of the tpflbm library (declarations and conventions in include/tpflbm.h)
// and the auxiliary kernels: initialisation, field read-back, state I/O and FP64
// reductions.  The step kernels live in step.cuh.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tpflbm.h"
#include "handle.h"
#include "lattice.cuh"
#include "step.cuh"

using namespace tpf;

namespace {

constexpr int kBX = kStepBX, kBY = kStepBY;  // step tile (handle.h)
constexpr long long kGraphSteps = 64;  // steps per replayed CUDA graph (even)

// ------------------------------------------------------- auxiliary kernels

// Macroscopic state of node (x, y) read straight from global memory.
template <class S>
__device__ Macro macro_at(const DevParams& P, const typename S::elem* __restrict__ A,
                          const RefT* __restrict__ ref, const float* __restrict__ phiu, int x, int y)
{
    const long long pl = P.plane;
    const int n = y * P.nx + x;
    float f[9], g[9], h[9];
    load_node<S>(P, A, ref, x, y, f, g, h);
    auto get = [&](int gx, int gy, float& ph, float& tt) {
        float a[9], c[9];
        load_node<S, false>(P, A, ref, gx, gy, a, nullptr, c);
        float sf = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            sf += a[i];
            sh += c[i];
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
__global__ void k_fields(const DevParams P, const typename S::elem* __restrict__ A, const RefT* __restrict__ ref,
                         const float* __restrict__ phiu, float* __restrict__ out)
{
    const long long N = (long long)P.nx * P.ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
        const Macro m = macro_at<S>(P, A, ref, phiu, x, y);
        out[n] = m.phi;
        out[P.plane + n] = m.ux;
        out[2 * P.plane + n] = m.uy;
        out[3 * P.plane + n] = m.p;
        out[4 * P.plane + n] = m.T;
    }
}

// Equilibrium populations from the staged fields (planes 0-4: phi, ux, uy, p, T).
// FP16 records: (phi, 0), (p / cs2, 0), (T, 0) of each node (first moments zero), so
// that every population is encoded against the rest equilibrium of its writer
// (ref_source).
//
// With HALF_SRC, half of each selected forcing source is taken off the equilibria
// (bit 0 of `which`: f_i -= R_i / 2 with R_i the interface term of the Allen-Cahn
// source, d_t(phi u) = 0; bit 1: g_i -= G_i / 2 with the NS forcing at the given u).  For a scheme that adds its
// source as (1 - 1/(2 tau)) S after the collision, these are the populations whose
// moments decode to the given fields: sum_i c_i g_i + F/2 = rho u and the pressure
// moment returns p.  The interfacial force, normal and density gradient come from
// the same stencils and ghost values as in the step, evaluated on the given phi, T.
template <class S, bool HALF_SRC>
__global__ void k_init(const DevParams P, const float* __restrict__ in, typename S::elem* __restrict__ A,
                       RefT* __restrict__ ref, float* __restrict__ phiu, int which = 0)
{
    const long long N = (long long)P.nx * P.ny;
    const long long pl = P.plane;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
        const float phi = in[n], ux = in[pl + n], uy = in[2 * pl + n], p = in[3 * pl + n], T = in[4 * pl + n];
        float f[9], g[9], h[9];
        node_equilibria(P, phi, ux, uy, p, T, f, g, h);
        if constexpr (HALF_SRC) {
            auto get = [&](int gx, int gy, float& ph, float& tt) {
                ph = in[(long long)gy * P.nx + gx];
                tt = in[4 * pl + (long long)gy * P.nx + gx];
            };
            float phin[9], Tn[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) phiT_at(P, x + cx(i), y + cy(i), get, phin[i], Tn[i]);
            const Macro m = node_macro(P, f, g, h, phin, Tn, phi * ux, phi * uy);
            const float theta = (1.f - phi * phi) * P.theta_k;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const float cu = cx(i) * ux + cy(i) * uy;
                const float Ri = wq(i) * theta * (cx(i) * m.nx + cy(i) * m.ny);
                const float cg = cx(i) * m.grx + cy(i) * m.gry;
                const float Gi = wq(i) * ((cx(i) * m.Fx + cy(i) * m.Fy) * kInvCs2 + cu * cg * kInvCs2);
                if (which & 1) f[i] -= 0.5f * Ri;
                if (which & 2) g[i] -= 0.5f * Gi;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float rf = 0.f, rg = 0.f, rh = 0.f;
            if constexpr (kRef<S>) {
                const int s = ref_source(P, x, y, i, false), sg = ref_source(P, x, y, i, true);
                rf = wq(i) * in[s];
                rg = wg(i) * (in[3 * pl + sg] * kInvCs2);
                rh = wq(i) * in[4 * pl + s];
            }
            S::st(A + i * pl, n, f[i], P.s_f, rf);
            S::st(A + (9 + i) * pl, n, g[i], P.s_g, rg);
            S::st(A + (18 + i) * pl, n, h[i], P.s_h, rh);
        }
        if constexpr (kRef<S>) {
            RefVals r;
            ref[kRecF * pl + n] = ref_pack(phi, 0.f, 0.f, r);
            ref[kRecG * pl + n] = ref_pack(p * kInvCs2, 0.f, 0.f, r);
            ref[kRecH * pl + n] = ref_pack(T, 0.f, 0.f, r);
        }
        phiu[n] = phi * ux;
        phiu[pl + n] = phi * uy;
    }
}

// State I/O of one LBE (k = 0 f, 1 g, 2 h) between 9 float32 staging planes and
// storage.  For FP16, k_lbe_ref first sets the LBE's record of each node from its
// staged populations, first moments zero: the zeroth moment (phi for f, T for h), and
// for g the pressure estimate p / cs2 = sum_{i != 0} g_i / (1 - w_0) (Eq. 21 without
// its velocity terms; any value serves as long as encoder and decoder share it).
__global__ void k_lbe_ref(const DevParams P, int k, const float* __restrict__ in, RefT* __restrict__ ref)
{
    const long long N = (long long)P.nx * P.ny;
    const long long pl = P.plane;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        float r = 0.f;
#pragma unroll
        for (int i = (k == 1 ? 1 : 0); i < 9; ++i) r += in[i * pl + n];
        if (k == 1) r /= 1.f - wq(0);
        RefVals v;
        ref[k * pl + n] = ref_pack(r, 0.f, 0.f, v);
    }
}
// reference of population i of LBE k at (x, y)
__device__ __forceinline__ float lbe_ref(const DevParams& P, int k, const RefT* __restrict__ ref, int x, int y, int i)
{
    const int s = ref_source(P, x, y, i, k == 1);
    const RefVals r = ref_unpack(ref[k * P.plane + s]);
    return k == 1 ? ref_g(i, r) : ref_pop(i, r);
}
template <class S>
__global__ void k_lbe_encode(const DevParams P, int k, const float* __restrict__ in, typename S::elem* __restrict__ A,
                             const RefT* __restrict__ ref)
{
    const long long N = (long long)P.nx * P.ny;
    const long long pl = P.plane;
    const float s = k == 0 ? P.s_f : (k == 1 ? P.s_g : P.s_h);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float r = kRef<S> ? lbe_ref(P, k, ref, x, y, i) : 0.f;
            S::st(A + (9 * k + i) * pl, n, in[i * pl + n], s, r);
        }
    }
}
template <class S>
__global__ void k_lbe_decode(const DevParams P, int k, const typename S::elem* __restrict__ A,
                             const RefT* __restrict__ ref, float* __restrict__ out)
{
    const long long N = (long long)P.nx * P.ny;
    const long long pl = P.plane;
    const float is = k == 0 ? P.is_f : (k == 1 ? P.is_g : P.is_h);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float r = kRef<S> ? lbe_ref(P, k, ref, x, y, i) : 0.f;
            out[i * pl + n] = S::ld(A + (9 * k + i) * pl, n, is, r);
        }
    }
}

// FP64 reductions (see tpflbm_diagnostics).  Each block writes 8 partial sums;
// k_reduce_final adds the partials of all blocks in a fixed order.
constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;

template <class S>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_partial(const DevParams P, const typename S::elem* __restrict__ A, const RefT* __restrict__ ref,
                 const float* __restrict__ phiu, double* __restrict__ partial)
{
    const long long N = (long long)P.nx * P.ny;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
        const Macro m = macro_at<S>(P, A, ref, phiu, x, y);
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

// One warp per quantity: lane l adds blocks l, l + 32, ... in order, then a fixed
// shuffle tree; the result does not depend on timing (deterministic).
__global__ void k_reduce_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 8) return;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += partial[b * 8 + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[k] = v;
}

// Steady-state residual: FP64 sums of |u - u_snap|^2, |u|^2 and (T - T_snap)^2 per
// block, then the snapshot is overwritten with the current u, T.
template <class S>
__global__ void __launch_bounds__(kRedThreads)
k_residual_partial(const DevParams P, const typename S::elem* __restrict__ A, const RefT* __restrict__ ref,
                   const float* __restrict__ phiu, float* __restrict__ snap, double* __restrict__ partial)
{
    const long long N = (long long)P.nx * P.ny;
    const long long pl = P.plane;
    double acc[3] = {0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)(n / P.nx);
        const Macro m = macro_at<S>(P, A, ref, phiu, x, y);
        const double dux = (double)m.ux - snap[n], duy = (double)m.uy - snap[pl + n];
        const double dT = (double)m.T - snap[2 * pl + n];
        acc[0] += dux * dux + duy * duy;
        acc[1] += (double)m.ux * m.ux + (double)m.uy * m.uy;
        acc[2] += dT * dT;
        snap[n] = m.ux;
        snap[pl + n] = m.uy;
        snap[2 * pl + n] = m.T;
    }
    __shared__ double red[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += red[threadIdx.x][w];
        partial[blockIdx.x * 8 + threadIdx.x] = v;
    }
}

// Mass-preserving projection of a predicted phase field onto the equilibrium profile
// phi = tanh(d / (sqrt(2) W)) (Sec. 2).  a_n = d_n / (sqrt(2) W) is the predicted
// scaled signed distance of node n (k_project_dist*), offset by a uniform s chosen so
// that sum phi matches a target.  Per block: sum phi(s) and its derivative
// sum (1 - phi(s)^2).
constexpr double kProjClip = 1.0 - 1e-7;
// a_n = atanh(phi_hat_n) (phi_hat clipped into (-1, 1))
__global__ void k_project_dist_atanh(const float* __restrict__ phat, long long N, float* __restrict__ a)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        a[n] = (float)atanh(fmin(fmax((double)phat[n], -kProjClip), kProjClip));
}
// a_n = (y_c(x) - y) / (sqrt(2) W) with y_c(x) the lowest zero crossing of phi_hat
// in column x going up from positive to non-positive (linear interpolation between
// the two nodes); a column without one uses the node of least |phi_hat|
__global__ void k_project_dist_contour(const float* __restrict__ phat, int nx, int ny, float inv_sw, float* __restrict__ a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    float yc = -1.f, best = 3.f;
    int jbest = 0;
    for (int j = 0; j + 1 < ny; ++j) {
        const float p0 = phat[(long long)j * nx + x], p1 = phat[(long long)(j + 1) * nx + x];
        if (p0 > 0.f && p1 <= 0.f) {
            yc = (float)j + p0 / (p0 - p1);
            break;
        }
        if (fabsf(p0) < best) {
            best = fabsf(p0);
            jbest = j;
        }
    }
    if (yc < 0.f) yc = (float)jbest;
    for (int j = 0; j < ny; ++j) a[(long long)j * nx + x] = (yc - (float)j) * inv_sw;
}
__global__ void __launch_bounds__(kRedThreads)
k_project_partial(const float* __restrict__ a, long long N, double s, double* __restrict__ partial)
{
    double sa = 0.0, sb = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const double v = tanh((double)a[n] + s);
        sa += v;
        sb += 1.0 - v * v;
    }
    __shared__ double red[2][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if (lane == 0) {
        red[0][warp] = sa;
        red[1][warp] = sb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += red[threadIdx.x][w];
        partial[blockIdx.x * 8 + threadIdx.x] = v;
    }
}
__global__ void k_project_apply(const float* __restrict__ a, long long N, double s, float* __restrict__ out)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        out[n] = (float)tanh((double)a[n] + s);
}

// Bubbles of Sec. 4.3: the connected regions of phi < 0 (4-connectivity, wrapping
// along periodic axes), each with its FP64 moments.  Labels are node indices: every
// node of the set starts with its own index and repeatedly takes the smallest label
// among itself, its in-set neighbours and its label's label (pointer jumping).  Labels
// only decrease and always name a node of the same region, so the fixed point gives
// every node of a region the region's smallest node index, its root.
constexpr int kMaxBubbles = 32;
constexpr int kBubBlocks = 40;  // kBubBlocks x kMaxBubbles x 6 partials + results fit the reduction area
static_assert((kBubBlocks + 1) * kMaxBubbles * 6 <= kRedMaxBlocks * 8 + 8, "bubble sums fit the reduction area");

__global__ void k_lab_init(const float* __restrict__ phi, long long N, int* __restrict__ lab)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        lab[n] = phi[n] < 0.f ? (int)n : -1;
}

__global__ void k_lab_hook(int nx, int ny, int bc_x, int bc_y, int* lab, int* changed)
{
    const long long N = (long long)nx * ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int l = lab[n];
        if (l < 0) continue;
        const int x = (int)(n % nx), y = (int)(n / nx);
        int m = min(l, lab[l]);
        const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int qx = nb[k][0], qy = nb[k][1];
            if (bc_x == 0) qx = wrap(qx, nx);
            if (bc_y == 1) qy = wrap(qy, ny);
            if (qx < 0 || qx >= nx || qy < 0 || qy >= ny) continue;
            const int lq = lab[(long long)qy * nx + qx];
            if (lq >= 0 && lq < m) m = lq;
        }
        if (m < l) {
            atomicMin(&lab[n], m);
            atomicMin(&lab[l], m);  // the old label's node joins too (same region)
            *changed = 1;
        }
    }
}

__global__ void k_lab_roots(const int* __restrict__ lab, long long N, int* __restrict__ count, int* __restrict__ roots)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        if (lab[n] == (int)n) {
            const int k = atomicAdd(count, 1);
            if (k < kMaxBubbles) roots[k] = (int)n;
        }
}

struct RootList {
    int n;
    int r[kMaxBubbles];
};

// Per block and bubble: node count, sum phi, sum phi u_x, sum phi u_y, sum phi dx,
// sum phi dy, with (dx, dy) the node's offset from its root, taken to the nearest
// periodic image along periodic axes.
__global__ void __launch_bounds__(256)
k_bubble_partial(int nx, int ny, int bc_x, int bc_y, const float* __restrict__ phi, const float* __restrict__ ux,
                 const float* __restrict__ uy, const int* __restrict__ lab, const RootList roots,
                 double* __restrict__ partial)
{
    __shared__ double acc[kMaxBubbles][6];
    for (int k = threadIdx.x; k < kMaxBubbles * 6; k += blockDim.x) acc[k / 6][k % 6] = 0.0;
    __syncthreads();
    const long long N = (long long)nx * ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int l = lab[n];
        if (l < 0) continue;
        int b = -1;
        for (int k = 0; k < roots.n; ++k)
            if (roots.r[k] == l) b = k;
        if (b < 0) continue;
        int dx = (int)(n % nx) - l % nx, dy = (int)(n / nx) - l / nx;
        if (bc_x == 0) dx = dx > nx / 2 ? dx - nx : (dx < -nx / 2 ? dx + nx : dx);
        if (bc_y == 1) dy = dy > ny / 2 ? dy - ny : (dy < -ny / 2 ? dy + ny : dy);
        const double ph = phi[n];
        atomicAdd(&acc[b][0], 1.0);
        atomicAdd(&acc[b][1], ph);
        atomicAdd(&acc[b][2], ph * ux[n]);
        atomicAdd(&acc[b][3], ph * uy[n]);
        atomicAdd(&acc[b][4], ph * dx);
        atomicAdd(&acc[b][5], ph * dy);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < roots.n * 6; k += blockDim.x)
        partial[(blockIdx.x * kMaxBubbles + k / 6) * 6 + k % 6] = acc[k / 6][k % 6];
}

// sums of the block partials in block order (one thread per bubble and quantity)
__global__ void k_bubble_final(const double* __restrict__ partial, int nblocks, int nb, double* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb * 6) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[(b * kMaxBubbles + k / 6) * 6 + k % 6];
    out[k] = v;
}

}  // namespace

// Scratch of tpflbm_diagnostics_static: the per-block partial sums (kRedMaxBlocks x 8)
// and the 8 results, in a fixed device array so that the entry point allocates
// nothing.  Host code must not pass this name to a kernel (on the host it is only a
// stand-in); it uses the address cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) double g_diag_scratch[kRedMaxBlocks * 8 + 8];

namespace {

thread_local std::string g_create_error;

constexpr int kStagePlanes = 9;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

long long plane_of(int nx, int ny) { return (((long long)nx * ny + 63) / 64) * 64; }

struct Layout {
    size_t pop0, pop1, ref0, ref1, phiu, stage, red, err, snap, tiles, total;
};

Layout layout_of(int nx, int ny, int storage)
{
    const long long pl = plane_of(nx, ny);
    const bool f16 = storage == TPF_STORAGE_FP16;
    const size_t e = f16 ? 2 : 4;
    Layout L{};
    size_t off = 0;
    L.pop0 = off; off = align256(off + 27 * (size_t)pl * e);
    L.pop1 = off; off = align256(off + 27 * (size_t)pl * e);
    L.ref0 = off; off = align256(off + (f16 ? 3 * (size_t)pl * sizeof(RefT) : 0));
    L.ref1 = off; off = align256(off + (f16 ? 3 * (size_t)pl * sizeof(RefT) : 0));
    L.phiu = off; off = align256(off + 2 * (size_t)pl * 4);
    L.stage = off; off = align256(off + kStagePlanes * (size_t)pl * 4);
    L.red = off; off = align256(off + (kRedMaxBlocks * 8 + 8) * sizeof(double));
    L.err = off; off = align256(off + 256);
    L.snap = off; off = align256(off + 3 * (size_t)pl * 4);
    // the TMA step kernel's tile list (x0, y0 per tile)
    L.tiles = off; off = align256(off + (size_t)((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY) * sizeof(int2));
    L.total = off;
    return L;
}

int fail(tpflbm_t h, int code, const std::string& msg)
{
    if (h) h->err_msg = msg;
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
    if ((long long)nx * ny > (1LL << 30)) { why = "lattice too large (nx * ny > 2^30)"; return TPF_ERR_INVALID_ARG; }
    if (p->storage != TPF_STORAGE_FP32 && p->storage != TPF_STORAGE_FP16) { why = "unknown storage"; return TPF_ERR_INVALID_ARG; }
    if (p->bc_x < 0 || p->bc_x > 1 || p->bc_y < 0 || p->bc_y > 1) { why = "bc_x/bc_y must be 0 or 1"; return TPF_ERR_INVALID_ARG; }
    if (p->sigma_law < 0 || p->sigma_law > 1) { why = "sigma_law must be 0 or 1"; return TPF_ERR_INVALID_ARG; }
    if (p->normal_law < 0 || p->normal_law > 1) { why = "normal_law must be 0 or 1"; return TPF_ERR_INVALID_ARG; }
    if (p->collision < 0 || p->collision > 1) { why = "collision must be 0 (BGK) or 1 (TRT)"; return TPF_ERR_INVALID_ARG; }
    if (p->collision == 1 && !(p->trt_lambda > 0.0)) { why = "TRT needs trt_lambda > 0"; return TPF_ERR_INVALID_ARG; }
    if (!(p->rho_l > 0 && p->rho_h > 0)) { why = "densities must be positive"; return TPF_ERR_INVALID_ARG; }
    if (!(p->mu_l > 0 && p->mu_h > 0 && p->lambda_l > 0 && p->lambda_h > 0)) { why = "mu and lambda must be positive (tau > 1/2)"; return TPF_ERR_INVALID_ARG; }
    if (!(p->cp_l > 0 && p->cp_h > 0)) { why = "heat capacities must be positive"; return TPF_ERR_INVALID_ARG; }
    // Eq. 28 weighs the destination's old population by (1 - 1/(rho c_p)); below one
    // that weight is negative and the thermal update amplifies instead of relaxing
    if (p->rho_l * p->cp_l < 1.0 - 1e-9 || p->rho_h * p->cp_h < 1.0 - 1e-9) {
        why = "heat capacitance rho * c_p must be >= 1 in both phases (lattice units)";
        return TPF_ERR_INVALID_ARG;
    }
    if (!(p->M_phi > 0) || !(p->W > 0)) { why = "M_phi and W must be positive"; return TPF_ERR_INVALID_ARG; }
    if (p->bc_x == 1 && p->bc_y == 1) { why = "an inlet/outflow channel needs walls (bc_y = 0)"; return TPF_ERR_INVALID_ARG; }
    if (p->fp16_scale_f < 0 || p->fp16_scale_g < 0 || p->fp16_scale_h < 0) { why = "FP16 scales must be >= 0"; return TPF_ERR_INVALID_ARG; }
    return TPF_OK;
}

DevParams make_dev_params(int nx, int ny, const tpflbm_params& p)
{
    DevParams d{};
    d.nx = nx; d.ny = ny; d.bc_x = p.bc_x; d.bc_y = p.bc_y; d.sigma_law = p.sigma_law; d.storage = p.storage;
    d.normal_law = p.normal_law;
    d.collision = p.collision;
    d.trt_lambda = (float)p.trt_lambda;
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
    d.jthr2 = (float)((1e-10 / 3.0 * tau_phi) * (1e-10 / 3.0 * tau_phi));
    d.src_phi = (float)(1.0 - 0.5 / tau_phi);
    d.sigma_ref = (float)p.sigma_ref; d.sigma_T = (float)p.sigma_T; d.sigma_TT = (float)p.sigma_TT; d.T_ref = (float)p.T_ref;
    d.Gx = (float)p.Gx; d.Gy = (float)p.Gy;
    d.u_ave = (float)p.u_ave; d.phi_in = (float)p.phi_in; d.T_in = (float)p.T_in; d.p_out = (float)p.p_out;
    d.T_bot = (float)p.T_bot; d.T_bot_amp = (float)p.T_bot_amp; d.T_bot_k = (float)p.T_bot_k;
    d.T_bot_slope = (float)p.T_bot_slope; d.T_top = (float)p.T_top; d.T_top_slope = (float)p.T_top_slope;
    if (p.storage == TPF_STORAGE_FP16) {
        d.s_f = pow2_scale(p.fp16_scale_f, 1024.0);
        d.s_g = pow2_scale(p.fp16_scale_g, 1024.0);
        d.s_h = pow2_scale(p.fp16_scale_h, 64.0);
    } else {
        d.s_f = d.s_g = d.s_h = 1.f;
    }
    d.is_f = 1.f / d.s_f; d.is_g = 1.f / d.s_g; d.is_h = 1.f / d.s_h;
    return d;
}

int grid_1d(long long N)
{
    long long b = (N + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

// ----------------------------------------------------------- TMA set-up

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

bool make_map(CUtensorMap* m, CUtensorMapDataType dt, size_t esize, void* base, int nx, int ny, int nz,
              long long plane, int bw, int bh, int bd)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)plane * esize};
    cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bd};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class S>
void setup_tma(tpflbm_t h)
{
    using L = TmaLayout<kBX, kBY, S>;
    const int nx = h->nx, ny = h->ny;
    const size_t e = sizeof(typename S::elem);
    h->tma = false;
    if (((size_t)nx * e) % 16 != 0 || ((size_t)nx * 4) % 16 != 0) return;
    // TMA tiles: every whole tile along a walled or inlet/outflow axis (the copies fill
    // the box beyond the lattice with zeros and the kernel applies the boundary rules
    // there) and, with FP32 storage, along a periodic x axis at least two tiles wide (a
    // seam tile fetches the wrapped columns from the other edge itself); otherwise, along
    // a periodic axis, the tiles whose (widened) halo lies inside the lattice
    int bx_lo = 0, by_lo = 0, bx_hi = nx / kBX - 1, by_hi = ny / kBY - 1;
    if (h->hp.bc_x == 0 && (kRef<S> || nx < 2 * kBX)) {
        bx_lo = (L::XP + kBX - 1) / kBX;
        bx_hi = -1;  // last tile index with x0 + BX + XP <= nx
        for (int b = 0; (b + 1) * kBX + L::XP <= nx; ++b) bx_hi = b;
    }
    if (h->hp.bc_y == 1) {
        by_lo = (2 + kBY - 1) / kBY;
        by_hi = -1;  // last tile index with y0 + BY + 2 <= ny
        for (int b = 0; (b + 1) * kBY + 2 <= ny; ++b) by_hi = b;
    }
    if (bx_hi < bx_lo || by_hi < by_lo) return;
    h->bx0 = bx_lo; h->by0 = by_lo;
    h->ntbx = bx_hi - bx_lo + 1; h->ntby = by_hi - by_lo + 1;
    const CUtensorMapDataType dt = sizeof(typename S::elem) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const long long pl = h->dp.plane;
    for (int c = 0; c < 2; ++c) {
        TmaMaps& M = h->maps[c];
        bool ok = make_map(&M.popF, dt, e, h->pop[c], nx, ny, 27, pl, L::FW, L::FH, 9) &&
                  make_map(&M.popG, dt, e, h->pop[c], nx, ny, 27, pl, kBX, kBY, 9) &&
                  make_map(&M.phiu, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->phiu, nx, ny, 2, pl, kBX, kBY, 2);
        if (kRef<S>) ok = ok && make_map(&M.ref, CU_TENSOR_MAP_DATA_TYPE_UINT64, 8, h->ref[c], nx, ny, 3, pl, L::RW, L::RH, 3);
        else M.ref = M.phiu;
        if (!ok) return;
    }
    // Tile list: first the rectangle's rows and columns that touch the lattice boundary
    // (only its first and last row and column can), then the others row by row, so that
    // no CTA's round-robin share holds more than one of the slower boundary tiles while
    // fewer of them than CTAs exist.
    {
        const int ntbx = h->ntbx, ntby = h->ntby;
        auto row_edge = [&](int b) { return b * kBY <= 1 || b * kBY + kBY >= ny - 1; };
        auto col_edge = [&](int b) { return b * kBX <= 1 || b * kBX + kBX >= nx - 1; };
        const bool fre = row_edge(by_lo), lre = ntby > 1 && row_edge(by_lo + ntby - 1);
        const bool fce = col_edge(bx_lo), lce = ntbx > 1 && col_edge(bx_lo + ntbx - 1);
        std::vector<int2> list;
        list.reserve((size_t)ntbx * ntby);
        auto add = [&](int bx, int by) { list.push_back(make_int2(bx * kBX, by * kBY)); };
        const int rlo = by_lo + (int)fre, rhi = by_lo + ntby - 1 - (int)lre;  // rows that are not boundary rows
        const int clo = bx_lo + (int)fce, chi = bx_lo + ntbx - 1 - (int)lce;
        if (fre) for (int bx = bx_lo; bx < bx_lo + ntbx; ++bx) add(bx, by_lo);
        if (lre) for (int bx = bx_lo; bx < bx_lo + ntbx; ++bx) add(bx, by_lo + ntby - 1);
        if (fce) for (int by = rlo; by <= rhi; ++by) add(bx_lo, by);
        if (lce) for (int by = rlo; by <= rhi; ++by) add(bx_lo + ntbx - 1, by);
        for (int by = rlo; by <= rhi; ++by)
            for (int bx = clo; bx <= chi; ++bx) add(bx, by);
        if ((long long)list.size() != (long long)ntbx * ntby) return;
        if (cudaMemcpy(h->tiles, list.data(), list.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    const int smem = 2 * L::STAGE;
    if (cudaFuncSetAttribute(k_step_tma<kBX, kBY, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_tma<kBX, kBY, S>, kBX * kBY, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return;
    }
    const int ntiles = ((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY);
    h->grid_tma = std::min(ntiles, per_sm * h->num_sms);
    h->tma = true;
}

int finish_create(tpflbm_t h, int nx, int ny, const tpflbm_params* p, void* ws, size_t bytes, bool owns)
{
    h->nx = nx; h->ny = ny; h->hp = *p;
    h->dp = make_dev_params(nx, ny, *p);
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    const Layout L = layout_of(nx, ny, p->storage);
    h->ws = ws; h->ws_bytes = bytes; h->owns = owns;
    char* b = (char*)ws;
    h->pop[0] = b + L.pop0;
    h->pop[1] = b + L.pop1;
    h->ref[0] = (RefT*)(b + L.ref0);
    h->ref[1] = (RefT*)(b + L.ref1);
    h->phiu = (float*)(b + L.phiu);
    h->stage = (float*)(b + L.stage);
    h->red = (double*)(b + L.red);
    h->err = (int*)(b + L.err);
    h->snap = (float*)(b + L.snap);
    h->tiles = (int2*)(b + L.tiles);
    if (cudaMemset(h->err, 0, sizeof(int)) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "cudaMemset");
    if (p->storage == TPF_STORAGE_FP16) setup_tma<StoreF16>(h);
    else setup_tma<StoreF32>(h);
    return TPF_OK;
}

template <class S>
void launch_step(tpflbm_t h)
{
    using E = typename S::elem;
    const DevParams& P = h->dp;
    const int c = h->cur;
    const E* A = (const E*)h->pop[c];
    E* B = (E*)h->pop[c ^ 1];
    if (h->tma) {
        using L = TmaLayout<kBX, kBY, S>;
        k_step_tma<kBX, kBY, S><<<h->grid_tma, kBX * kBY, 2 * L::STAGE, h->stream>>>(
            P, h->maps[c], A, B, h->phiu, h->ref[c], h->ref[c ^ 1], h->tiles, h->bx0, h->by0, h->ntbx, h->ntby,
            h->err);
    } else {
        dim3 grd((P.nx + kBX - 1) / kBX, (P.ny + kBY - 1) / kBY);
        k_step_general<kBX, kBY, S><<<grd, kBX * kBY, 0, h->stream>>>(P, A, B, h->phiu, h->ref[c], h->ref[c ^ 1]);
    }
    h->cur ^= 1;
}

// error raised by a step kernel (bounded waits that ran out)
int check_err(tpflbm_t h)
{
    int v = 0;
    TPF_CUDA(h, cudaMemcpyAsync(&v, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (v) return fail(h, TPF_ERR_TIMEOUT, "a step kernel gave up waiting for its shared-memory copies");
    return TPF_OK;
}

// copy a [ny][nx] float field (host or device, or NULL = constant `fill`) into staging plane k
int stage_in(tpflbm_t h, const float* src, int k, float fill)
{
    const long long N = (long long)h->nx * h->ny;
    float* dst = h->stage + k * h->dp.plane;
    if (src) {
        TPF_CUDA(h, cudaMemcpyAsync(dst, src, N * sizeof(float), cudaMemcpyDefault, h->stream));
        return TPF_OK;
    }
    if (fill == 0.f) {
        TPF_CUDA(h, cudaMemsetAsync(dst, 0, N * sizeof(float), h->stream));
        return TPF_OK;
    }
    float* tmp = new (std::nothrow) float[N];
    if (!tmp) return fail(h, TPF_ERR_OOM, "host allocation failed");
    for (long long i = 0; i < N; ++i) tmp[i] = fill;
    cudaError_t e = cudaMemcpyAsync(dst, tmp, N * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    delete[] tmp;
    if (e != cudaSuccess) return cuda_fail(h, e, "stage fill");
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "stage fill sync");
    return TPF_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

namespace {

// One block waits, with the step kernels' bounded wait, on an mbarrier that nothing
// completes (no arrival, no copy in flight), then votes and raises the flag the way a
// step kernel raises its error flag.
__global__ void k_wait_check(uint32_t polls, int* flag)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, polls);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(flag, 1);
}

}  // namespace

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
    rc = finish_create(h, nx, ny, p, ws, bytes, true);
    if (rc != TPF_OK) {
        g_create_error = h->err_msg;
        cudaFree(ws);
        delete h;
        return rc;
    }
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
    rc = finish_create(h, nx, ny, p, workspace, bytes, false);
    if (rc != TPF_OK) {
        g_create_error = h->err_msg;
        delete h;
        return rc;
    }
    *out = h;
    return TPF_OK;
}

int tpflbm_set_stream(tpflbm_t h, void* stream)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return TPF_OK;
}

static int init_impl(tpflbm_t h, const float* phi, const float* ux, const float* uy, const float* p, const float* T,
                     int which)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    const float* src[5] = {phi, ux, uy, p, T};
    for (int k = 0; k < 5; ++k) {
        int rc = stage_in(h, src[k], k, k == 0 ? 1.f : 0.f);
        if (rc) return rc;
    }
    const long long N = (long long)h->nx * h->ny;
    const int c = h->cur;
    const bool f16 = h->dp.storage == TPF_STORAGE_FP16;
    const bool half_src = which != 0;
    if (f16 && half_src)
        k_init<StoreF16, true><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->stage, (__half*)h->pop[c], h->ref[c], h->phiu, which);
    else if (f16)
        k_init<StoreF16, false><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->stage, (__half*)h->pop[c], h->ref[c], h->phiu);
    else if (half_src)
        k_init<StoreF32, true><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->stage, (float*)h->pop[c], h->ref[c], h->phiu, which);
    else
        k_init<StoreF32, false><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, h->stage, (float*)h->pop[c], h->ref[c], h->phiu);
    TPF_CUDA(h, cudaGetLastError());
    // init reads the caller's buffers asynchronously: finish before returning
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->t = 0;
    h->snap_t = -1;
    return TPF_OK;
}

int tpflbm_init(tpflbm_t h, const float* phi, const float* ux, const float* uy, const float* p, const float* T)
{
    return init_impl(h, phi, ux, uy, p, T, 0);
}

int tpflbm_init_forced(tpflbm_t h, const float* phi, const float* ux, const float* uy, const float* p, const float* T,
                       int which)
{
    if (which < 1 || which > 3) return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_init_forced: which must be 1, 2 or 3");
    return init_impl(h, phi, ux, uy, p, T, which);
}

int tpflbm_step(tpflbm_t h, long long nsteps)
{
    if (!h || nsteps < 0) return TPF_ERR_INVALID_ARG;
    // whole chunks from a CUDA graph when the stream can be captured (not the legacy
    // default stream); kGraphSteps is even, so a chunk leaves the parity unchanged
    while (h->stream && nsteps >= kGraphSteps) {
        cudaGraphExec_t g = h->graph[h->cur];
        if (!g) {
            const int c0 = h->cur;
            cudaGraph_t graph = nullptr;
            TPF_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            for (long long s = 0; s < kGraphSteps; ++s) {
                if (h->dp.storage == TPF_STORAGE_FP16) launch_step<StoreF16>(h);
                else launch_step<StoreF32>(h);
            }
            cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
            h->cur = c0;
            if (e != cudaSuccess) return fail(h, TPF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&h->graph[c0], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(h, TPF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            g = h->graph[c0];
        }
        TPF_CUDA(h, cudaGraphLaunch(g, h->stream));
        nsteps -= kGraphSteps;
        h->t += kGraphSteps;
    }
    for (long long s = 0; s < nsteps; ++s) {
        if (h->dp.storage == TPF_STORAGE_FP16) launch_step<StoreF16>(h);
        else launch_step<StoreF32>(h);
    }
    TPF_CUDA(h, cudaGetLastError());
    h->t += nsteps;
    return TPF_OK;
}

int tpflbm_status(tpflbm_t h)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    return check_err(h);
}

int tpflbm_status_async(tpflbm_t h, int* flag, void* copy_stream)
{
    if (!h || !flag) return TPF_ERR_INVALID_ARG;
    cudaStream_t cs = (cudaStream_t)copy_stream;
    if (!cs || cs == h->stream) {
        TPF_CUDA(h, cudaMemcpyAsync(flag, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        return TPF_OK;
    }
    // on the copy stream, behind an event on the handle's stream: the next steps do not
    // wait for the copy
    if (!h->status_ev) TPF_CUDA(h, cudaEventCreateWithFlags(&h->status_ev, cudaEventDisableTiming));
    TPF_CUDA(h, cudaEventRecord(h->status_ev, h->stream));
    TPF_CUDA(h, cudaStreamWaitEvent(cs, h->status_ev, 0));
    TPF_CUDA(h, cudaMemcpyAsync(flag, h->err, sizeof(int), cudaMemcpyDeviceToHost, cs));
    return TPF_OK;
}

int tpflbm_get_fields(tpflbm_t h, float* phi, float* ux, float* uy, float* p, float* T)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    int rc = check_err(h);
    if (rc) return rc;
    const long long N = (long long)h->nx * h->ny;
    const int c = h->cur;
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_fields<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const __half*)h->pop[c], h->ref[c], h->phiu, h->stage);
    else
        k_fields<StoreF32><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const float*)h->pop[c], h->ref[c], h->phiu, h->stage);
    TPF_CUDA(h, cudaGetLastError());
    float* dst[5] = {phi, ux, uy, p, T};
    for (int k = 0; k < 5; ++k)
        if (dst[k])
            TPF_CUDA(h, cudaMemcpyAsync(dst[k], h->stage + k * h->dp.plane, N * sizeof(float), cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    return TPF_OK;
}

int tpflbm_get_state(tpflbm_t h, float* f, float* g, float* hh, float* phiu)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    int rc = check_err(h);
    if (rc) return rc;
    const long long N = (long long)h->nx * h->ny;
    const long long pl = h->dp.plane;
    const int c = h->cur;
    float* dsts[3] = {f, g, hh};
    for (int k = 0; k < 3; ++k) {
        if (!dsts[k]) continue;
        if (h->dp.storage == TPF_STORAGE_FP16)
            k_lbe_decode<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, k, (const __half*)h->pop[c], h->ref[c], h->stage);
        else
            k_lbe_decode<StoreF32><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, k, (const float*)h->pop[c], h->ref[c], h->stage);
        TPF_CUDA(h, cudaGetLastError());
        for (int i = 0; i < 9; ++i)
            TPF_CUDA(h, cudaMemcpyAsync(dsts[k] + (long long)i * N, h->stage + i * pl, N * 4, cudaMemcpyDefault, h->stream));
        TPF_CUDA(h, cudaStreamSynchronize(h->stream));
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
    const int c = h->cur;
    const float* srcs[3] = {f, g, hh};
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i < 9; ++i)
            TPF_CUDA(h, cudaMemcpyAsync(h->stage + i * pl, srcs[k] + (long long)i * N, N * 4, cudaMemcpyDefault, h->stream));
        if (h->dp.storage == TPF_STORAGE_FP16) {
            k_lbe_ref<<<grid_1d(N), 256, 0, h->stream>>>(h->dp, k, h->stage, h->ref[c]);
            k_lbe_encode<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, k, h->stage, (__half*)h->pop[c], h->ref[c]);
        } else {
            k_lbe_encode<StoreF32><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, k, h->stage, (float*)h->pop[c], h->ref[c]);
        }
        TPF_CUDA(h, cudaGetLastError());
    }
    TPF_CUDA(h, cudaMemcpyAsync(h->phiu, phiu, N * 4, cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaMemcpyAsync(h->phiu + pl, phiu + N, N * 4, cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    return TPF_OK;
}

int tpflbm_diagnostics(tpflbm_t h, double out[8])
{
    if (!h || !out) return TPF_ERR_INVALID_ARG;
    int rc = check_err(h);
    if (rc) return rc;
    const long long N = (long long)h->nx * h->ny;
    long long b = (N + kRedThreads - 1) / kRedThreads;
    const int nb = (int)(b < kRedMaxBlocks ? b : kRedMaxBlocks);
    const int c = h->cur;
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_reduce_partial<StoreF16><<<nb, kRedThreads, 0, h->stream>>>(h->dp, (const __half*)h->pop[c], h->ref[c], h->phiu, h->red);
    else
        k_reduce_partial<StoreF32><<<nb, kRedThreads, 0, h->stream>>>(h->dp, (const float*)h->pop[c], h->ref[c], h->phiu, h->red);
    TPF_CUDA(h, cudaGetLastError());
    double* res = h->red + kRedMaxBlocks * 8;
    k_reduce_final<<<1, 256, 0, h->stream>>>(h->red, nb, res);
    TPF_CUDA(h, cudaGetLastError());
    TPF_CUDA(h, cudaMemcpyAsync(out, res, 8 * sizeof(double), cudaMemcpyDefault, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (out[7] > 0) return fail(h, TPF_ERR_NONFINITE, "non-finite values in the state");
    return TPF_OK;
}

int tpflbm_diagnostics_static(int nx, int ny, const tpflbm_params* p, const void* pop, long long plane,
                              const void* ref, const float* phiu, double out[8], void* stream)
{
    std::string why;
    int rc = validate(nx, ny, p, why);
    if (rc != TPF_OK) return fail(nullptr, rc, "tpflbm_diagnostics_static: " + why);
    if (!pop || !phiu || !out) return fail(nullptr, TPF_ERR_INVALID_ARG, "tpflbm_diagnostics_static: pop, phiu and out are required");
    if (plane < (long long)nx * ny) return fail(nullptr, TPF_ERR_INVALID_ARG, "tpflbm_diagnostics_static: plane must be >= nx * ny");
    const bool f16 = p->storage == TPF_STORAGE_FP16;
    if (f16 && !ref) return fail(nullptr, TPF_ERR_INVALID_ARG, "tpflbm_diagnostics_static: FP16 storage needs the reference records");

    // the scratch's device address in the context current now (a lookup, no allocation;
    // done on every call so that it follows the context after a reset or a switch)
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_diag_scratch);
    if (e != cudaSuccess) return fail(nullptr, TPF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    double* scratch = (double*)a;

    DevParams P = make_dev_params(nx, ny, *p);
    P.plane = plane;
    const long long N = (long long)nx * ny;
    const long long b = (N + kRedThreads - 1) / kRedThreads;
    const int nb = (int)(b < kRedMaxBlocks ? b : kRedMaxBlocks);
    cudaStream_t s = (cudaStream_t)stream;
    if (f16)
        k_reduce_partial<StoreF16><<<nb, kRedThreads, 0, s>>>(P, (const __half*)pop, (const RefT*)ref, phiu, scratch);
    else
        k_reduce_partial<StoreF32><<<nb, kRedThreads, 0, s>>>(P, (const float*)pop, (const RefT*)ref, phiu, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, TPF_ERR_CUDA, std::string("k_reduce_partial: ") + cudaGetErrorString(e));
    double* res = scratch + kRedMaxBlocks * 8;
    k_reduce_final<<<1, 256, 0, s>>>(scratch, nb, res);
    // one copy of the results on the caller's stream, then out from that host copy
    double v[8];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, res, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaPointerAttributes at{};
    if (e == cudaSuccess) e = cudaPointerGetAttributes(&at, out);
    if (e == cudaSuccess) {
        if (at.type == cudaMemoryTypeDevice) {
            e = cudaMemcpyAsync(out, v, sizeof(v), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        } else {
            std::memcpy(out, v, sizeof(v));
        }
    }
    if (e != cudaSuccess) return fail(nullptr, TPF_ERR_CUDA, std::string("tpflbm_diagnostics_static: ") + cudaGetErrorString(e));
    if (v[7] > 0) return fail(nullptr, TPF_ERR_NONFINITE, "non-finite values in the state");
    return TPF_OK;
}

int tpflbm_state_buffers(tpflbm_t h, void** pop, void** ref, void** phiu, long long* plane)
{
    if (!h) return TPF_ERR_INVALID_ARG;
    if (pop) *pop = h->pop[h->cur];
    if (ref) *ref = h->dp.storage == TPF_STORAGE_FP16 ? (void*)h->ref[h->cur] : nullptr;
    if (phiu) *phiu = h->phiu;
    if (plane) *plane = h->dp.plane;
    return TPF_OK;
}

int tpflbm_residual(tpflbm_t h, double dT, double out[3])
{
    if (!h || !out || !(dT > 0)) return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_residual needs out and dT > 0");
    int rc = check_err(h);
    if (rc) return rc;
    const long long N = (long long)h->nx * h->ny;
    long long b = (N + kRedThreads - 1) / kRedThreads;
    const int nb = (int)(b < kRedMaxBlocks ? b : kRedMaxBlocks);
    const int c = h->cur;
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_residual_partial<StoreF16><<<nb, kRedThreads, 0, h->stream>>>(h->dp, (const __half*)h->pop[c], h->ref[c], h->phiu, h->snap, h->red);
    else
        k_residual_partial<StoreF32><<<nb, kRedThreads, 0, h->stream>>>(h->dp, (const float*)h->pop[c], h->ref[c], h->phiu, h->snap, h->red);
    TPF_CUDA(h, cudaGetLastError());
    double* res = h->red + kRedMaxBlocks * 8;
    k_reduce_final<<<1, 256, 0, h->stream>>>(h->red, nb, res);
    TPF_CUDA(h, cudaGetLastError());
    double sums[8];
    TPF_CUDA(h, cudaMemcpyAsync(sums, res, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    const long long K = h->t - h->snap_t;
    const bool first = h->snap_t < 0;
    h->snap_t = h->t;
    if (first || K <= 0) {
        out[0] = out[1] = HUGE_VAL;
        out[2] = 0;
        return TPF_OK;
    }
    out[0] = sums[1] > 0 ? std::sqrt(sums[0]) / (K * std::sqrt(sums[1])) : (sums[0] > 0 ? HUGE_VAL : 0.0);
    out[1] = std::sqrt(sums[2]) / (K * dT * std::sqrt((double)N));
    out[2] = (double)K;
    return TPF_OK;
}

int tpflbm_project_phi(tpflbm_t h, const float* phi_pred, double target_sum, int mode, float* phi_out,
                       double* achieved)
{
    if (!h || !phi_pred || !phi_out) return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_project_phi needs phi_pred and phi_out");
    if (mode != TPF_PROJECT_ATANH && mode != TPF_PROJECT_CONTOUR)
        return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_project_phi: unknown mode");
    const long long N = (long long)h->nx * h->ny;
    if (!(std::fabs(target_sum) < (double)N)) return fail(h, TPF_ERR_INVALID_ARG, "target sum must lie strictly inside (-N, N)");
    // scaled distances in the last staging plane
    float* a = h->stage + 8 * h->dp.plane;
    if (mode == TPF_PROJECT_ATANH) {
        k_project_dist_atanh<<<grid_1d(N), 256, 0, h->stream>>>(phi_pred, N, a);
    } else {
        const float inv_sw = (float)(1.0 / (std::sqrt(2.0) * h->hp.W));
        k_project_dist_contour<<<(h->nx + 127) / 128, 128, 0, h->stream>>>(phi_pred, h->nx, h->ny, inv_sw, a);
    }
    TPF_CUDA(h, cudaGetLastError());
    const long long b = (N + kRedThreads - 1) / kRedThreads;
    const int nb = (int)(b < kRedMaxBlocks ? b : kRedMaxBlocks);
    double* res = h->red + kRedMaxBlocks * 8;
    double s = 0.0, sums[2] = {0.0, 0.0};
    const double tol = 1e-12 * (double)N;
    // Newton on S(s) = sum tanh(a_n + s), increasing in s
    int it = 0;
    for (; it < 100; ++it) {
        k_project_partial<<<nb, kRedThreads, 0, h->stream>>>(a, N, s, h->red);
        TPF_CUDA(h, cudaGetLastError());
        k_reduce_final<<<1, 256, 0, h->stream>>>(h->red, nb, res);
        TPF_CUDA(h, cudaGetLastError());
        TPF_CUDA(h, cudaMemcpyAsync(sums, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        TPF_CUDA(h, cudaStreamSynchronize(h->stream));
        const double r = sums[0] - target_sum;
        if (!std::isfinite(r)) return fail(h, TPF_ERR_NONFINITE, "tpflbm_project_phi: non-finite predicted phase field");
        if (std::fabs(r) <= tol) break;
        if (!(sums[1] > 0.0)) return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_project_phi: the field has no interface to move");
        double step = r / sums[1];
        if (step > 2.0) step = 2.0;  // keep the iterate inside tanh's useful range
        if (step < -2.0) step = -2.0;
        s -= step;
    }
    if (it == 100) return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_project_phi: no convergence");
    k_project_apply<<<grid_1d(N), 256, 0, h->stream>>>(a, N, s, phi_out);
    TPF_CUDA(h, cudaGetLastError());
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (achieved) *achieved = sums[0];
    return TPF_OK;
}

int tpflbm_bubbles(tpflbm_t h, int max_bubbles, double* out, int* count)
{
    if (!h || max_bubbles < 0 || (max_bubbles > 0 && !out) || !count)
        return fail(h, TPF_ERR_INVALID_ARG, "tpflbm_bubbles needs count, and out when max_bubbles > 0");
    int rc = check_err(h);
    if (rc) return rc;
    const long long N = (long long)h->nx * h->ny;
    const long long pl = h->dp.plane;
    const int c = h->cur;
    // phi, u_x, u_y of the current state into staging planes 0-2 (as tpflbm_get_fields)
    if (h->dp.storage == TPF_STORAGE_FP16)
        k_fields<StoreF16><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const __half*)h->pop[c], h->ref[c], h->phiu, h->stage);
    else
        k_fields<StoreF32><<<grid_1d(N), 256, 0, h->stream>>>(h->dp, (const float*)h->pop[c], h->ref[c], h->phiu, h->stage);
    TPF_CUDA(h, cudaGetLastError());
    int* lab = (int*)(h->stage + 5 * pl);
    int* roots = (int*)(h->stage + 6 * pl);  // kMaxBubbles entries
    int* flags = h->err + 1;                   // [0] changed, [1] root count
    k_lab_init<<<grid_1d(N), 256, 0, h->stream>>>(h->stage, N, lab);
    TPF_CUDA(h, cudaGetLastError());
    // propagate to the fixed point, checking for changes every 4 sweeps; a region of
    // n nodes settles within n sweeps (pointer jumping makes it far fewer)
    const long long max_sweeps = N + 8;
    long long sweeps = 0;
    for (;;) {
        int changed = 0;
        TPF_CUDA(h, cudaMemsetAsync(flags, 0, sizeof(int), h->stream));
        for (int k = 0; k < 4; ++k)
            k_lab_hook<<<grid_1d(N), 256, 0, h->stream>>>(h->nx, h->ny, h->dp.bc_x, h->dp.bc_y, lab, flags);
        TPF_CUDA(h, cudaGetLastError());
        TPF_CUDA(h, cudaMemcpyAsync(&changed, flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        TPF_CUDA(h, cudaStreamSynchronize(h->stream));
        sweeps += 4;
        if (!changed) break;
        if (sweeps > max_sweeps) return fail(h, TPF_ERR_UNSUPPORTED, "tpflbm_bubbles: labelling did not settle");
    }
    TPF_CUDA(h, cudaMemsetAsync(flags + 1, 0, sizeof(int), h->stream));
    k_lab_roots<<<grid_1d(N), 256, 0, h->stream>>>(lab, N, flags + 1, roots);
    TPF_CUDA(h, cudaGetLastError());
    RootList rl{};
    int nroots = 0;
    TPF_CUDA(h, cudaMemcpyAsync(&nroots, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    TPF_CUDA(h, cudaMemcpyAsync(rl.r, roots, sizeof(rl.r), cudaMemcpyDeviceToHost, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (nroots > kMaxBubbles)
        return fail(h, TPF_ERR_UNSUPPORTED, "tpflbm_bubbles: more than 32 separate regions of phi < 0");
    rl.n = nroots;
    std::sort(rl.r, rl.r + nroots);
    *count = nroots;
    if (nroots == 0 || max_bubbles == 0) return TPF_OK;
    double* part = h->red;
    double* res = h->red + kBubBlocks * kMaxBubbles * 6;
    k_bubble_partial<<<kBubBlocks, 256, 0, h->stream>>>(h->nx, h->ny, h->dp.bc_x, h->dp.bc_y, h->stage, h->stage + pl,
                                                        h->stage + 2 * pl, lab, rl, part);
    TPF_CUDA(h, cudaGetLastError());
    k_bubble_final<<<1, kMaxBubbles * 6, 0, h->stream>>>(part, kBubBlocks, nroots, res);
    TPF_CUDA(h, cudaGetLastError());
    double sums[kMaxBubbles * 6];
    TPF_CUDA(h, cudaMemcpyAsync(sums, res, nroots * 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TPF_CUDA(h, cudaStreamSynchronize(h->stream));
    // per bubble: nodes, sum phi, u_b, v_b, x_b, y_b; ordered by x_b, then y_b
    double rows[kMaxBubbles][6];
    for (int k = 0; k < nroots; ++k) {
        const double* v = sums + 6 * k;
        const int xr = rl.r[k] % h->nx, yr = rl.r[k] / h->nx;
        double xb = xr + v[4] / v[1], yb = yr + v[5] / v[1];
        if (h->dp.bc_x == 0) xb = std::fmod(xb + h->nx, (double)h->nx);
        if (h->dp.bc_y == 1) yb = std::fmod(yb + h->ny, (double)h->ny);
        const double r[6] = {v[0], v[1], v[2] / v[1], v[3] / v[1], xb, yb};
        std::memcpy(rows[k], r, sizeof(r));
    }
    int order[kMaxBubbles];
    for (int k = 0; k < nroots; ++k) order[k] = k;
    std::sort(order, order + nroots, [&](int a, int b) {
        return rows[a][4] < rows[b][4] || (rows[a][4] == rows[b][4] && rows[a][5] < rows[b][5]);
    });
    for (int k = 0; k < nroots && k < max_bubbles; ++k) std::memcpy(out + 6 * k, rows[order[k]], 6 * sizeof(double));
    return TPF_OK;
}

int tpflbm_check_bounded_wait(int polls, int* gave_up)
{
    if (polls < 1 || !gave_up) return fail(nullptr, TPF_ERR_INVALID_ARG, "tpflbm_check_bounded_wait: polls >= 1 and gave_up required");
    *gave_up = 0;
    int* flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_check<<<1, 256>>>((uint32_t)polls, flag);
        e = cudaGetLastError();
    }
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tpflbm_check_bounded_wait");
    *gave_up = v;
    return TPF_OK;
}

long long tpflbm_time(tpflbm_t h) { return h ? h->t : -1; }

void tpflbm_destroy(tpflbm_t h)
{
    if (!h) return;
    for (int c = 0; c < 2; ++c)
        if (h->graph[c]) cudaGraphExecDestroy(h->graph[c]);
    if (h->status_ev) cudaEventDestroy(h->status_ev);
    if (h->owns && h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
    }
    delete h;
}

const char* tpflbm_last_error(tpflbm_t h)
{
    return h ? h->err_msg.c_str() : g_create_error.c_str();
}

}  // extern "C"
