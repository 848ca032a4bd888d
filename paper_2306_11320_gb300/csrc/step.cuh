// The fused time step of the three coupled LBEs (arXiv 2306.11320, Sec. 3-4):
// a general tile routine (every boundary rule, thread loads) and a persistent
// kernel that stages interior tiles in shared memory with TMA, double buffered.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lattice.cuh"

namespace tpf {

// FP16 storage keeps the scaled deviation s_k (q_i - r_i) of each population from a
// reference r_i built from a record that the population's writer leaves for the next
// step:
//   f: r_i = w_i (phi + c_i . J_f / cs2)      h: r_i = w_i (T + c_i . J_h / cs2)
//   g: r_i = wg_i p / cs2 + w_i c_i . J_g / cs2   (wg_0 = w_0 - 1, wg_i = w_i)
// with phi, T, p the writer's moments and J_f, J_g, J_h the first moments of its
// post-collision f, g, h, i.e. the rest equilibrium plus the first-order Hermite term
// of what it emitted, so that only the higher-order non-equilibrium part is
// quantised.  The writer of population i at y is the node it streamed from, y - c_i
// (wrapped when periodic), except where y - c_i lies outside the fluid: a population
// reflected at a wall or at the inlet (and g reflected at the outflow) was written by
// y itself, and f, h entering through the outflow are the copies that the last
// column's node y - c_iy (same column) made of its own populations.  A record is one
// 8-byte word per LBE and node: the zeroth moment in float32 and J / cs2 as two
// halves; the writer encodes against the rounded record, so encoder and decoder see
// the same reference bit for bit.
template <class S>
constexpr bool kRef = std::is_same<S, StoreF16>::value;

using RefT = uint2;  // one reference record: float32 zeroth moment, half2 first moment / cs2
constexpr int kRecF = 0, kRecG = 1, kRecH = 2;  // record planes

struct RefVals {
    float m0, jx, jy;
};
__device__ __forceinline__ RefVals ref_unpack(RefT q)
{
    const float2 j = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    return {__uint_as_float(q.x), j.x, j.y};
}
// keeps m0, rounds (jx, jy) to halves; r receives the values the decoder will see
__device__ __forceinline__ RefT ref_pack(float m0, float jx, float jy, RefVals& r)
{
    const __half2 j = __floats2half2_rn(jx, jy);
    const float2 fj = __half22float2(j);
    r = {m0, fj.x, fj.y};
    RefT q;
    q.x = __float_as_uint(m0);
    q.y = *reinterpret_cast<const uint32_t*>(&j);
    return q;
}

// c_i . (vx, vy) for a moving direction i, adding only its nonzero components (after
// unrolling, i is a constant and the selects fold away)
__device__ __forceinline__ float cdot(int i, float vx, float vy)
{
    const float a = cx(i) > 0 ? vx : -vx, b = cy(i) > 0 ? vy : -vy;
    return cx(i) == 0 ? b : (cy(i) == 0 ? a : a + b);
}
// reference of population i of f or h from its writer's record
__device__ __forceinline__ float ref_pop(int i, const RefVals& r)
{
    return i == 0 ? wq(0) * r.m0 : wq(i) * (r.m0 + cdot(i, r.jx, r.jy));
}
// reference of population i of g (r.m0 = p / cs2)
__device__ __forceinline__ float ref_g(int i, const RefVals& r)
{
    return i == 0 ? wg(0) * r.m0 : fmaf(wg(i), r.m0, wq(i) * cdot(i, r.jx, r.jy));
}

// node that wrote population i at (x, y), whose record is its FP16 reference (for the
// g LBE when g_lbe: the outflow reflects g at the node itself)
__device__ __forceinline__ int ref_source(const DevParams& P, int x, int y, int i, bool g_lbe)
{
    int sx = x - cx(i), sy = y - cy(i);
    if (P.bc_x == 0) sx = wrap(sx, P.nx);
    if (P.bc_y == 1) sy = wrap(sy, P.ny);
    if (sy < 0 || sy >= P.ny || sx < 0 || (sx >= P.nx && g_lbe)) return y * P.nx + x;
    if (sx >= P.nx) return sy * P.nx + (P.nx - 1);  // outflow copy made by (nx - 1, sy)
    return sy * P.nx + sx;
}

// ref_source for a node of a TMA tile: the writer's slot in the tile's record box
// (origin x0 - 4, y0 - 2, RW x RH).  Records exist with FP16 storage only, whose TMA
// tiles never need a periodic wrap.  Every writer lies in the box; the clamps only keep
// the slot inside it when P itself is not to be trusted (a batched tile whose copies,
// parameters included, timed out).
__device__ __forceinline__ int ref_slot_box(const DevParams& P, int x, int y, int i, bool g_lbe, int x0, int y0,
                                            int RW, int RH)
{
    int sx = x - cx(i), sy = y - cy(i);
    if (sy < 0 || sy >= P.ny || sx < 0 || (sx >= P.nx && g_lbe)) {
        sx = x;
        sy = y;
    } else if (sx >= P.nx) {
        sx = P.nx - 1;
    }
    const int c = min(max(sx - x0 + 4, 0), RW - 1), r = min(max(sy - y0 + 2, 0), RH - 1);
    return r * RW + c;
}

// Decoded populations of node (x, y) read from global memory (general path).
template <class S, bool WANT_G = true>
__device__ __forceinline__ void load_node(const DevParams& P, const typename S::elem* __restrict__ A,
                                          const RefT* __restrict__ ref, int x, int y, float* f, float* g,
                                          float* h)
{
    const long long pl = P.plane;
    const int n = y * P.nx + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float rf = 0.f, rg = 0.f, rh = 0.f;
        if constexpr (kRef<S>) {
            const int s = ref_source(P, x, y, i, false);
            rf = ref_pop(i, ref_unpack(ref[kRecF * pl + s]));
            rh = ref_pop(i, ref_unpack(ref[kRecH * pl + s]));
            if constexpr (WANT_G) rg = ref_g(i, ref_unpack(ref[kRecG * pl + ref_source(P, x, y, i, true)]));
        }
        f[i] = S::ld(A + i * pl, n, P.is_f, rf);
        if constexpr (WANT_G) g[i] = S::ld(A + (9 + i) * pl, n, P.is_g, rg);
        h[i] = S::ld(A + (18 + i) * pl, n, P.is_h, rh);
    }
}

// Shared staging of phi, T, 1/(rho c_p) and pre-collision h for a tile and its ring.
template <int BX, int BY>
struct RingSmem {
    static constexpr int SX = BX + 2, SY = BY + 2, SN = SX * SY;
    float phi[SN];
    float T[SN];
    float irc[SN];
    float h[9][SN];
};

// Collide the node's populations and push them to their destinations, with every
// boundary rule; for FP16 also leave the node's reference records in refB (every
// population this node writes is encoded against them).  hold(i, k) and irc(k) give
// the pre-collision h_i and 1/(rho c_p) of the node in ring slot k.
template <class S, int SX, class HOLD, class IRC>
__device__ __forceinline__ void collide_push(const DevParams& P, typename S::elem* __restrict__ B,
                                             RefT* __restrict__ refB, int x, int y, int kown, bool interior,
                                             const Macro& m, float* f, float* g, float* h, HOLD hold, IRC irc)
{
    const long long pl = P.plane;
    const int n = y * P.nx + x;
    node_collide(P, m, f, g, h);
    // FP16 reference records of what this node emits (as the decoder sees them)
    RefVals rf{0.f, 0.f, 0.f}, rgv{0.f, 0.f, 0.f}, rh{0.f, 0.f, 0.f};
    if constexpr (kRef<S>) {
        float jfx, jfy, jgx, jgy, jhx, jhy;
        dq9_moment1(f, jfx, jfy);
        dq9_moment1(g, jgx, jgy);
        dq9_moment1(h, jhx, jhy);
        refB[kRecF * pl + n] = ref_pack(m.phi, jfx * kInvCs2, jfy * kInvCs2, rf);
        refB[kRecG * pl + n] = ref_pack(m.p * kInvCs2, jgx * kInvCs2, jgy * kInvCs2, rgv);
        refB[kRecH * pl + n] = ref_pack(m.T, jhx * kInvCs2, jhy * kInvCs2, rh);
    }
    if (interior) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int d = n + cy(i) * P.nx + cx(i);
            const int kd = kown + cy(i) * SX + cx(i);
            S::st(B + i * pl, d, f[i], P.s_f, ref_pop(i, rf));
            S::st(B + (9 + i) * pl, d, g[i], P.s_g, ref_g(i, rgv));
            const float ho = hold(i, kd);
            S::st(B + (18 + i) * pl, d, fmaf(h[i] - ho, irc(kd), ho), P.s_h, ref_pop(i, rh));
        }
        return;
    }
    const float irc_own = irc(kown);
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
            S::st(B + o * pl, n, f[i], P.s_f, ref_pop(o, rf));
            S::st(B + (9 + o) * pl, n, g[i], P.s_g, ref_g(o, rgv));
            const float ho = hold(o, kown);
            const float hin = -h[i] + 2.f * wq(o) * Tw;
            S::st(B + (18 + o) * pl, n, fmaf(hin - ho, irc_own, ho), P.s_h, ref_pop(o, rh));
        } else if (out_x && dx < 0) {
            // velocity inlet: bounce-back carrying the inlet momentum and phi_in
            const float ycr = (float)y + 0.5f + 0.5f * cy(i);
            const float cu = cx(o) * u_inlet(P, ycr);
            S::st(B + o * pl, n, f[i] + 2.f * wq(o) * P.phi_in * cu * kInvCs2, P.s_f, ref_pop(o, rf));
            S::st(B + (9 + o) * pl, n, g[i] + 2.f * wq(o) * m.rho * cu * kInvCs2, P.s_g, ref_g(o, rgv));
            const float ho = hold(o, kown);
            const float hin = -h[i] + 2.f * wq(o) * P.T_in;
            S::st(B + (18 + o) * pl, n, fmaf(hin - ho, irc_own, ho), P.s_h, ref_pop(o, rh));
        } else if (out_x) {
            // outflow: pressure anti-bounce-back of g (f and h arrive by the copy below)
            const float cu = cx(o) * m.ux + cy(o) * m.uy;
            const float sym = P.p_out * kInvCs2 +
                              m.rho * (0.5f * cu * cu * kInvCs2 * kInvCs2 - 0.5f * (m.ux * m.ux + m.uy * m.uy) * kInvCs2);
            S::st(B + (9 + o) * pl, n, -g[i] + 2.f * wq(o) * sym, P.s_g, ref_g(o, rgv));
        } else {
            const int d = dy * P.nx + dx;
            const int kd = kown + cy(i) * SX + cx(i);
            S::st(B + i * pl, d, f[i], P.s_f, ref_pop(i, rf));
            S::st(B + (9 + i) * pl, d, g[i], P.s_g, ref_g(i, rgv));
            const float ho = hold(i, kd);
            S::st(B + (18 + i) * pl, d, fmaf(h[i] - ho, irc(kd), ho), P.s_h, ref_pop(i, rh));
        }
        // zero-gradient outflow of f and h: the ghost column beyond x = nx-1 carries the
        // post-collision populations of the last column (this node wrote them, so they
        // are encoded against its own records).
        if (P.bc_x == 1 && x == P.nx - 1 && cx(i) < 0) {
            const int ey = y + cy(i);
            if (ey >= 0 && ey < P.ny) {
                const int d = ey * P.nx + x;
                const int kd = kown + cy(i) * SX;
                S::st(B + i * pl, d, f[i], P.s_f, ref_pop(i, rf));
                const float ho = hold(i, kd);
                S::st(B + (18 + i) * pl, d, fmaf(h[i] - ho, irc(kd), ho), P.s_h, ref_pop(i, rh));
            }
        }
    }
}

// One tile through the general path: thread loads, ghost values and every boundary
// rule.  Used for lattices whose rows do not meet TMA alignment, by the batched
// ensemble, and in the TMA kernel for the tiles next to a periodic seam and the ragged
// tiles.  (bx, by): tile coordinates.
template <int BX, int BY, class S>
__device__ __forceinline__ void step_tile_general(const DevParams& P, const typename S::elem* __restrict__ A,
                                                  typename S::elem* __restrict__ B, float* __restrict__ phiu,
                                                  const RefT* __restrict__ refA, RefT* __restrict__ refB,
                                                  RingSmem<BX, BY>& sm, int bx, int by)
{
    constexpr int SX = RingSmem<BX, BY>::SX, SN = RingSmem<BX, BY>::SN;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int x0 = bx * BX, y0 = by * BY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < P.nx && y < P.ny;
    const long long pl = P.plane;
    const int n = y * P.nx + x;
    const int kown = (ty + 1) * SX + tx + 1;
    const bool interior = x0 >= 1 && x0 + BX <= P.nx - 1 && y0 >= 1 && y0 + BY <= P.ny - 1;

    // Whole tiles: one thread per ring node issues that node's loads together with the
    // own node's, so the tile waits on one round trip to memory, and ghost ring nodes
    // take their mirror's values from shared memory once those are in.  Ragged tiles
    // walk every slot outside the lattice part of the tile.
    constexpr int kRing = 2 * (BX + BY) + 4;
    static_assert(kRing <= BX * BY, "one thread per ring node");
    const bool whole = x0 + BX <= P.nx && y0 + BY <= P.ny;
    int rx = 0, ry = 0, wx = 0, wy = 0;
    bool rload = false, rghost = false;
    float ra[9], rc[9];
    if (whole && (int)threadIdx.x < kRing) {
        const int r = threadIdx.x;
        if (r < SX) { rx = r; ry = 0; }
        else if (r < 2 * SX) { rx = r - SX; ry = BY + 1; }
        else if (r < 2 * SX + BY) { rx = 0; ry = r - 2 * SX + 1; }
        else { rx = BX + 1; ry = r - 2 * SX - BY + 1; }
        wx = x0 + rx - 1;
        wy = y0 + ry - 1;
        if (P.bc_x == 0) wx = wrap(wx, P.nx);
        if (P.bc_y == 1) wy = wrap(wy, P.ny);
        rload = wx >= 0 && wx < P.nx && wy >= 0 && wy < P.ny;
        rghost = !rload;
        if (rload) load_node<S, false>(P, A, refA, wx, wy, ra, nullptr, rc);
    }

    float f[9], g[9], h[9];
    if (active) {
        load_node<S>(P, A, refA, x, y, f, g, h);
        float sf = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            sf += f[i];
            sh += h[i];
        }
        sm.phi[kown] = sf;
        sm.T[kown] = sh;
        sm.irc[kown] = __frcp_rn(fmaf(P.rcp_b, clamp1(sf), P.rcp_a));
#pragma unroll
        for (int i = 0; i < 9; ++i) sm.h[i][kown] = h[i];
    }
    if (whole) {
        if (rload) {
            const int k = ry * SX + rx;
            float sf = 0.f, sh = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                sf += ra[i];
                sh += rc[i];
                sm.h[i][k] = rc[i];
            }
            sm.phi[k] = sf;
            sm.T[k] = sh;
            sm.irc[k] = __frcp_rn(fmaf(P.rcp_b, clamp1(sf), P.rcp_a));
        }
        // ghost ring nodes beyond walls, inlet and outflow (as phiT_at): phi mirrored,
        // T by the boundary's rule; the mirror is the adjacent slot inside the lattice
        if (__syncthreads_or(rghost) && rghost) {
            const int gx = x0 + rx - 1, gy = y0 + ry - 1;
            const int mx = min(max(wx, 0), P.nx - 1), my = min(max(wy, 0), P.ny - 1);
            const int km = (ry + my - wy) * SX + rx + mx - wx;
            const float tm = sm.T[km];
            const float tx = (wx < 0) ? 2.f * P.T_in - tm : tm;
            const bool oy = wy < 0 || wy >= P.ny;
            const int k = ry * SX + rx;
            sm.phi[k] = sm.phi[km];
            sm.T[k] = oy ? 2.f * (wy < 0 ? T_wall_bottom(P, (float)gx) : T_wall_top(P, (float)gx)) - tx : tx;
            sm.irc[k] = 0.f;
            (void)gy;
        }
    } else {
        auto get = [&](int gx, int gy, float& ph, float& tt) {
            float a[9], c[9];
            load_node<S, false>(P, A, refA, gx, gy, a, nullptr, c);
            float sf = 0.f, sh = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                sf += a[i];
                sh += c[i];
            }
            ph = sf;
            tt = sh;
        };
        for (int k = threadIdx.x; k < SN; k += BX * BY) {
            const int lx = k % SX, ly = k / SX;
            const bool own = lx >= 1 && lx <= BX && ly >= 1 && ly <= BY && (x0 + lx - 1) < P.nx && (y0 + ly - 1) < P.ny;
            if (own) continue;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            int qx = gx, qy = gy;
            if (P.bc_x == 0) qx = wrap(qx, P.nx);
            if (P.bc_y == 1) qy = wrap(qy, P.ny);
            const bool far = gx < -1 || gx > P.nx || gy < -1 || gy > P.ny;
            if (far) {
                sm.phi[k] = 0.f;
                sm.T[k] = 0.f;
                sm.irc[k] = 0.f;
                continue;
            }
            if (qx >= 0 && qx < P.nx && qy >= 0 && qy < P.ny) {
                float a[9], c[9];
                load_node<S, false>(P, A, refA, qx, qy, a, nullptr, c);
                float sf = 0.f, sh = 0.f;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    sf += a[i];
                    sh += c[i];
                    sm.h[i][k] = c[i];
                }
                sm.phi[k] = sf;
                sm.T[k] = sh;
                sm.irc[k] = __frcp_rn(fmaf(P.rcp_b, clamp1(sf), P.rcp_a));
            } else {
                float ph, tt;
                phiT_at(P, gx, gy, get, ph, tt);
                sm.phi[k] = ph;
                sm.T[k] = tt;
                sm.irc[k] = 0.f;
            }
        }
    }
    __syncthreads();
    if (active) {
        float phin[9], Tn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int k = kown + cy(i) * SX + cx(i);
            phin[i] = sm.phi[k];
            Tn[i] = sm.T[k];
        }
        const Macro m = node_macro(P, f, g, h, phin, Tn, phiu[n], phiu[pl + n]);
        phiu[n] = m.phi * m.ux;
        phiu[pl + n] = m.phi * m.uy;
        collide_push<S, SX>(
            P, B, refB, x, y, kown, interior, m, f, g, h, [&](int i, int k) { return sm.h[i][k]; },
            [&](int k) { return sm.irc[k]; });
    }
    __syncthreads();  // the caller may reuse sm for the next tile
}

template <int BX, int BY, class S>
__global__ void __launch_bounds__(BX * BY, 3)
k_step_general(const DevParams P, const typename S::elem* __restrict__ A, typename S::elem* __restrict__ B,
               float* __restrict__ phiu, const RefT* __restrict__ refA, RefT* __restrict__ refB)
{
    __shared__ RingSmem<BX, BY> sm;
    step_tile_general<BX, BY, S>(P, A, B, phiu, refA, refB, sm, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------ TMA kernel
//
// Persistent CTAs walk a tile list: first the TMA tiles, then the remaining tiles
// through the general path.  TMA tiles are the whole tiles whose halo lies inside the
// lattice along each periodic axis (x0 >= XP, x0 + BX + XP <= nx; y0 >= 2,
// y0 + BY + 2 <= ny), which along a walled or inlet/outflow axis are all whole tiles:
// there the box reaches past the lattice, the copy fills it with zeros, and the tile
// takes its ghost ring nodes and its boundary nodes' FP16 records by the boundary
// rules instead.  For a TMA tile one elected thread issues 3D bulk
// tensor copies (cp.async.bulk.tensor) of the 9 f planes and the 9 h planes over the
// tile plus a one-node ring (widened to XP columns each side for the 16-byte rule),
// the 9 g planes and the 2 (phi u) planes over the tile, and for FP16 the 3 planes of
// reference records over the tile plus a two-node ring, all completing on one mbarrier.  While a
// tile is computed, the next tile's copies are in flight into the other stage.

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// bounded wait: false after `limit` polls (about 2^22 in the step kernels; each
// try_wait suspends for a while)
constexpr uint32_t kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit)
{
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <int BX, int BY, class S>
struct TmaLayout {
    using E = typename S::elem;
    static constexpr int XP = 16 / (int)sizeof(E);           // column pad for 16-byte aligned boxes
    static constexpr int FW = BX + 2 * XP, FH = BY + 2;     // f/h box (tile + ring, widened)
    static constexpr int RW = BX + 8, RH = BY + 4;          // reference box (tile + 2-ring, widened)
    static constexpr int rnd(int b) { return (b + 127) / 128 * 128; }
    static constexpr int F_BYTES = 9 * FH * FW * (int)sizeof(E);
    static constexpr int G_BYTES = 9 * BY * BX * (int)sizeof(E);
    static constexpr int U_BYTES = 2 * BY * BX * 4;
    static constexpr int R_BYTES = kRef<S> ? 3 * RH * RW * (int)sizeof(RefT) : 0;
    static constexpr int OFF_F = 0, OFF_H = rnd(F_BYTES), OFF_G = OFF_H + rnd(F_BYTES), OFF_U = OFF_G + rnd(G_BYTES),
                         OFF_R = OFF_U + rnd(U_BYTES), STAGE = OFF_R + rnd(R_BYTES);
    static constexpr uint32_t TX_BYTES = 2 * F_BYTES + G_BYTES + U_BYTES + R_BYTES;
};

// Which side of a periodic x seam a TMA tile sits on: -1 its left ring column wraps to
// x = nx - 1, +1 its right one to x = 0, 0 neither.  Seam tiles are staged by TMA with
// FP32 storage only, and only in lattices at least two tiles wide (so no tile has both
// sides); otherwise they take the general path and this is 0 for every TMA tile.  With
// FP16 storage (records to patch as well) the seam code pushed the kernel to its
// 128-register cap and slowed every tile (the 2048 x 512 channel, which has no seam,
// by 3.5%).
template <int BX>
__device__ __forceinline__ int seam_side(const DevParams& P, int x0)
{
    if (P.bc_x != 0) return 0;
    return x0 == 0 ? -1 : (x0 + BX == P.nx ? 1 : 0);
}

struct TmaMaps {
    CUtensorMap popF;  // populations, box FW x FH x 9 (used for f at z = 0 and h at z = 18)
    CUtensorMap popG;  // populations, box BX x BY x 9 (g at z = 9)
    CUtensorMap phiu;  // (phi u) planes, box BX x BY x 2
    CUtensorMap ref;   // FP16 reference records (8-byte elements), box RW x RH x 3
};

// The copies of one TMA tile into stage st, completing on bar (one elected thread).
template <int BX, int BY, class S>
__device__ __forceinline__ void tma_issue_tile(const TmaMaps& M, unsigned char* st, uint64_t* bar, int x0, int y0)
{
    using L = TmaLayout<BX, BY, S>;
    fence_proxy_async();
    mbar_expect_tx(bar, L::TX_BYTES);
    tma_load_3d(st + L::OFF_F, &M.popF, bar, x0 - L::XP, y0 - 1, 0);
    tma_load_3d(st + L::OFF_H, &M.popF, bar, x0 - L::XP, y0 - 1, 18);
    tma_load_3d(st + L::OFF_G, &M.popG, bar, x0, y0, 9);
    tma_load_3d(st + L::OFF_U, &M.phiu, bar, x0, y0, 0);
    if constexpr (kRef<S>) tma_load_3d(st + L::OFF_R, &M.ref, bar, x0 - 4, y0 - 2, 0);
}

// phi, T and 1/(rho c_p) of a TMA tile and its ring
template <int BX, int BY>
struct PhiSmem {
    static constexpr int SN = (BX + 2) * (BY + 2);
    float phi[SN];
    float T[SN];
    float irc[SN];
};

// Periodic x seam (FP32 storage): the wrapped ring column of f and h from global memory
// A into the box, where the copies left zeros, before anything decodes it (rows beyond
// a wall stay zero: nothing decodes them).  Out of line: it runs for seam tiles only,
// which wait one memory round trip here, and the stages keep their size.  Ends with a
// block barrier.
template <int BX, int BY, class S>
__device__ __noinline__ void seam_patch(unsigned char* st, int seam, const typename S::elem* __restrict__ A, int nx,
                                        int ny, long long pl, int y0)
{
    static_assert(!kRef<S>, "FP16 tiles are not staged across a seam");
    using L = TmaLayout<BX, BY, S>;
    using E = typename S::elem;
    E* bF = (E*)(st + L::OFF_F);
    E* bH = (E*)(st + L::OFF_H);
    const int fc = seam < 0 ? L::XP - 1 : L::XP + BX, gx = seam < 0 ? nx - 1 : 0;
    for (int k = threadIdx.x; k < 9 * L::FH; k += BX * BY) {
        const int i = k / L::FH, y = y0 - 1 + k % L::FH;
        if (y < 0 || y >= ny) continue;
        const long long n = (long long)y * nx + gx;
        bF[k * L::FW + fc] = A[i * pl + n];
        bH[k * L::FW + fc] = A[(18 + i) * pl + n];
    }
    __syncthreads();
}

// The body of one TMA tile, shared by the single-lattice and the batched kernels: decode
// the staged populations of the tile (stage st, landed unless ok is false) and its
// ring, phi / T / 1/(rho c_p) into sm, one block barrier (which also votes on ok:
// on_abort() runs on every thread and the tile returns true when any wait ran out),
// after_ring() on every thread, then per node the macroscopic state, the collisions
// and the push to B.  EDGE: the tile touches the lattice boundary (ghost ring nodes,
// boundary records, boundary-aware push for every node); seam (seam_side): the wrapped
// column of a periodic x seam comes from A first.  EDGE and seam must be the
// same on every thread and must not come from a staged P (it is not to be trusted
// before the vote).
template <int BX, int BY, class S, bool EDGE, bool PRELOAD, class OnAbort, class AfterRing>
__device__ __forceinline__ bool tma_tile(const DevParams& P, const typename S::elem* __restrict__ A,
                                         typename S::elem* __restrict__ B, float* __restrict__ phiu,
                                         RefT* __restrict__ refB,
                                         unsigned char* st, PhiSmem<BX, BY>& sm, int x0, int y0, int seam, bool ok,
                                         OnAbort on_abort, AfterRing after_ring)
{
    using L = TmaLayout<BX, BY, S>;
    using E = typename S::elem;
    constexpr int SX = BX + 2;
    constexpr int kRing = 2 * (BX + BY) + 4;
    static_assert(2 * kRing <= BX * BY, "one thread per ring moment");
    const int tid = threadIdx.x;
    const long long pl = P.plane;
    const E* sF = (const E*)(st + L::OFF_F);
    const E* sH = (const E*)(st + L::OFF_H);
    const E* sG = (const E*)(st + L::OFF_G);
    const float* sU = (const float*)(st + L::OFF_U);
    const RefT* sR = (const RefT*)(st + L::OFF_R);
    (void)sR;
    constexpr bool edge = EDGE;
    // nodes on a walled, inlet or outflow boundary (a periodic one has none), and ring
    // nodes beyond one.  Only FP32 TMA tiles reach a periodic edge (x seams): the other
    // TMA tiles keep one node clear of every periodic edge, where the plain tests agree.
    constexpr bool kSeams = !kRef<S>;
    auto on_boundary = [&](int gx, int gy) {
        return ((!kSeams || P.bc_x != 0) && (gx == 0 || gx == P.nx - 1)) || gy == 0 || gy == P.ny - 1;
    };
    auto is_ghost = [&](int gx, int gy) {
        return ((!kSeams || P.bc_x != 0) && (gx < 0 || gx >= P.nx)) || gy < 0 || gy >= P.ny;
    };
    if constexpr (edge) {
        if constexpr (!kRef<S>) {
            if (seam) {
                // vote first: a batched tile's P and buffer pointers arrive with its copies
                if (__syncthreads_or(!ok)) {
                    on_abort();
                    return true;
                }
                seam_patch<BX, BY, S>(st, seam, A, P.nx, P.ny, P.plane, y0);
            }
        }
    }

    // decoded population i of ring slot (lx, ly) from the f (or h) box
    auto decF = [&](const E* box, float is, int rplane, int i, int lx, int ly, bool bnode) {
        float r = 0.f;
        if constexpr (kRef<S>) {
            const int k = bnode ? ref_slot_box(P, x0 + lx - 1, y0 + ly - 1, i, false, x0, y0, L::RW, L::RH)
                                : (ly + 1 - cy(i)) * L::RW + lx + 3 - cx(i);
            r = ref_pop(i, ref_unpack(sR[rplane * L::RH * L::RW + k]));
        }
        return S::lds(box, (i * L::FH + ly) * L::FW + lx - 1 + L::XP, is, r);
    };

    // own node: decoded populations, phi, T, 1/(rho c_p)
    const int tx = tid % BX, ty = tid / BX;
    const int lx = tx + 1, ly = ty + 1, kown = ly * SX + lx;
    const int x = x0 + tx, y = y0 + ty;
    const int n = y * P.nx + x;
    const bool bnode = edge && on_boundary(x, y);
    float f[9], g[9], h[9], phin[9], Tn[9];
    {
        float sf = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float rf = 0.f, rg = 0.f, rh = 0.f;
            if constexpr (kRef<S>) {
                int k = (ly + 1 - cy(i)) * L::RW + lx + 3 - cx(i), kg = k;
                if (bnode) {
                    k = ref_slot_box(P, x, y, i, false, x0, y0, L::RW, L::RH);
                    kg = ref_slot_box(P, x, y, i, true, x0, y0, L::RW, L::RH);
                }
                rf = ref_pop(i, ref_unpack(sR[kRecF * L::RH * L::RW + k]));
                rg = ref_g(i, ref_unpack(sR[kRecG * L::RH * L::RW + kg]));
                rh = ref_pop(i, ref_unpack(sR[kRecH * L::RH * L::RW + k]));
            }
            f[i] = S::lds(sF, (i * L::FH + ly) * L::FW + lx - 1 + L::XP, P.is_f, rf);
            h[i] = S::lds(sH, (i * L::FH + ly) * L::FW + lx - 1 + L::XP, P.is_h, rh);
            g[i] = S::lds(sG, (i * BY + ty) * BX + tx, P.is_g, rg);
            sf += f[i];
            sh += h[i];
        }
        sm.phi[kown] = sf;
        sm.T[kown] = sh;
        sm.irc[kown] = __frcp_rn(fmaf(P.rcp_b, clamp1(sf), P.rcp_a));
    }
    // PRELOAD (tiles without boundary nodes): the rest of the tile's reads of the stage,
    // done before the ring barrier so that the stage is free after it: the destinations'
    // pre-collision h_i for the push (each came from this node, so for FP16 its
    // reference is this node's record) and the previous (phi u)
    constexpr bool kPre = PRELOAD && !EDGE;
    float hold_r[9], pu_x = 0.f, pu_y = 0.f;
    RefVals rown_h{0.f, 0.f, 0.f};
    (void)hold_r;
    if constexpr (kPre) {
        if constexpr (kRef<S>) rown_h = ref_unpack(sR[(kRecH * L::RH + ly + 1) * L::RW + lx + 3]);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int kd = kown + cy(i) * SX + cx(i);
            float r = 0.f;
            if constexpr (kRef<S>) r = ref_pop(i, rown_h);
            hold_r[i] = S::lds(sH, (i * L::FH + kd / SX) * L::FW + kd % SX - 1 + L::XP, P.is_h, r);
        }
        pu_x = sU[ty * BX + tx];
        pu_y = sU[(BY + ty) * BX + tx];
    }
    // ring: 2 (BX + BY) + 4 nodes, one zeroth moment (f or h) per thread
    if (tid < 2 * kRing) {
        const int r = tid < kRing ? tid : tid - kRing;
        int rx, ry;
        if (r < SX) { rx = r; ry = 0; }
        else if (r < 2 * SX) { rx = r - SX; ry = BY + 1; }
        else if (r < 2 * SX + BY) { rx = 0; ry = r - 2 * SX + 1; }
        else { rx = BX + 1; ry = r - 2 * SX - BY + 1; }
        const int k = ry * SX + rx;
        const int gx = x0 + rx - 1, gy = y0 + ry - 1;
        const bool ghost = edge && is_ghost(gx, gy);
        const bool rb = edge && on_boundary(gx, gy);
        float s = 0.f;
        if (ghost) {
            // filled below from the node it mirrors
        } else if (tid < kRing) {
#pragma unroll
            for (int i = 0; i < 9; ++i) s += decF(sF, P.is_f, kRecF, i, rx, ry, rb);
            sm.phi[k] = s;
            sm.irc[k] = __frcp_rn(fmaf(P.rcp_b, clamp1(s), P.rcp_a));
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) s += decF(sH, P.is_h, kRecH, i, rx, ry, rb);
            sm.T[k] = s;
        }
    }
    if constexpr (edge) {
        // ghost ring nodes beyond walls, inlet and outflow: phi mirrored, T by the
        // boundary's rule (as phiT_at does for the general path)
        __syncthreads();
        if (tid < kRing) {
            const int r = tid;
            int rx, ry;
            if (r < SX) { rx = r; ry = 0; }
            else if (r < 2 * SX) { rx = r - SX; ry = BY + 1; }
            else if (r < 2 * SX + BY) { rx = 0; ry = r - 2 * SX + 1; }
            else { rx = BX + 1; ry = r - 2 * SX - BY + 1; }
            const int gx = x0 + rx - 1, gy = y0 + ry - 1;
            const bool ox = (!kSeams || P.bc_x != 0) && (gx < 0 || gx >= P.nx), oy = gy < 0 || gy >= P.ny;
            if (ox || oy) {
                const int mx = ox ? (gx < 0 ? 0 : P.nx - 1) : gx;
                const int my = oy ? (gy < 0 ? 0 : P.ny - 1) : gy;
                // (the clamp only matters when P is not to be trusted, as above)
                const int km = min(max((my - y0 + 1) * SX + mx - x0 + 1, 0), PhiSmem<BX, BY>::SN - 1);
                const float tm = sm.T[km];
                const float tx = (ox && gx < 0) ? 2.f * P.T_in - tm : tm;
                const int k = ry * SX + rx;
                sm.phi[k] = sm.phi[km];
                sm.T[k] = oy ? 2.f * (gy < 0 ? T_wall_bottom(P, (float)gx) : T_wall_top(P, (float)gx)) - tx : tx;
                sm.irc[k] = 0.f;
            }
        }
    }
    if (__syncthreads_or(!ok)) {
        on_abort();
        return true;
    }
    after_ring();
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int k = kown + cy(i) * SX + cx(i);
        phin[i] = sm.phi[k];
        Tn[i] = sm.T[k];
    }
    if constexpr (!kPre) {
        pu_x = sU[ty * BX + tx];
        pu_y = sU[(BY + ty) * BX + tx];
    }
    const Macro m = node_macro(P, f, g, h, phin, Tn, pu_x, pu_y);
    phiu[n] = m.phi * m.ux;
    phiu[pl + n] = m.phi * m.uy;
    if constexpr (kRef<S> && !kPre) rown_h = ref_unpack(sR[(kRecH * L::RH + ly + 1) * L::RW + lx + 3]);
    collide_push<S, SX>(
        P, B, refB, x, y, kown, !edge, m, f, g, h,
        [&](int i, int kd) {
            if constexpr (kPre) {
                return hold_r[i];  // interior tiles push only to kd = own + c_i
            } else {
                // h_i of destination kd came from this node: its reference is this node's record
                float r = 0.f;
                if constexpr (kRef<S>) r = ref_pop(i, rown_h);
                return S::lds(sH, (i * L::FH + kd / SX) * L::FW + kd % SX - 1 + L::XP, P.is_h, r);
            }
        },
        [&](int kd) { return sm.irc[kd]; });
    return false;
}

// CTAs per SM the TMA kernel is built for (shared memory allows up to 2 for FP32 and
// 3 for FP16; more CTAs means fewer registers per thread).
#ifndef TPF_TMA_BLOCKS_F32
#define TPF_TMA_BLOCKS_F32 2
#endif
#ifndef TPF_TMA_BLOCKS_F16
#define TPF_TMA_BLOCKS_F16 2
#endif
template <class S>
constexpr int kTmaMinBlocks = kRef<S> ? TPF_TMA_BLOCKS_F16 : TPF_TMA_BLOCKS_F32;

template <int BX, int BY, class S>
__global__ void __launch_bounds__(BX * BY, kTmaMinBlocks<S>)
k_step_tma(const DevParams P, const __grid_constant__ TmaMaps maps, const typename S::elem* __restrict__ A,
           typename S::elem* __restrict__ B, float* __restrict__ phiu, const RefT* __restrict__ refA,
           RefT* __restrict__ refB, const int2* __restrict__ tiles, int bx0, int by0, int ntbx, int ntby,
           int* __restrict__ err)
{
    using L = TmaLayout<BX, BY, S>;
    static_assert(sizeof(RingSmem<BX, BY>) <= 2 * L::STAGE, "general-path tiles reuse the stages");
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar[2];
    // Where a tile's copies are issued: tile t + 2 (this CTA's after next) goes into the
    // stage of tile t as soon as tile t no longer reads it.  Tiles without boundary
    // nodes read everything they need from the stage before their ring barrier
    // (PRELOAD), so their stage is refilled right after it and the tile ends without a
    // block barrier; boundary tiles end with one and refill after it.  phi, T and
    // 1/(rho c_p) are double buffered: a warp may start the next tile while others still
    // push (it cannot get two tiles ahead: the next ring barrier waits for them).
    __shared__ PhiSmem<BX, BY> smb[2];

    const int ntma = ntbx * ntby;  // TMA tiles: bx in [bx0, bx0 + ntbx), by in [by0, by0 + ntby)
    const int tilesx = (P.nx + BX - 1) / BX, tilesy = (P.ny + BY - 1) / BY;
    const int nall = tilesx * tilesy;
    const int nedge = nall - ntma;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto tile_of = [&](int t, int k, int& x0, int& y0) {
        const int2 v = __ldg(tiles + t);
        x0 = v.x;
        y0 = v.y;
    };

    auto issue = [&](int t, int k, int s) {
        int x0, y0;
        tile_of(t, k, x0, y0);
        tma_issue_tile<BX, BY, S>(maps, dsm + s * L::STAGE, &bar[s], x0, y0);
    };

    int it = 0;
    int t = blockIdx.x;
    if (tid == 0) {
        if (t < ntma) issue(t, 0, 0);
        if (t + (int)gridDim.x < ntma) issue(t + gridDim.x, 1, 1);
    }
    for (; t < ntma; t += gridDim.x, ++it) {
        const int s = it & 1;
        const int tn = t + gridDim.x, t2 = t + 2 * gridDim.x;
        PhiSmem<BX, BY>& sm = smb[s];
        // every thread waits for the stage itself; a thread whose wait ran out reads
        // stale (in-bounds) shared memory until the block votes at the next barrier
        const bool ok = mbar_wait_bounded(&bar[s], (it >> 1) & 1);
        int x0, y0;
        tile_of(t, it, x0, y0);
        // the tile body is compiled twice: for tiles touching the lattice boundary and
        // for all others, which keep the plain interior code
        auto on_abort = [&]() {
            if (tid == 0) {
                atomicExch(err, 1);
                // let this CTA's copies in flight land (bounded) before leaving
                mbar_wait_bounded(&bar[s], (it >> 1) & 1);
                if (tn < ntma) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1);
            }
        };
        auto refill = [&]() {
            if (t2 < ntma && tid == 0) issue(t2, it + 2, s);
        };
        auto no_refill = [&]() {};
        unsigned char* st = dsm + s * L::STAGE;
        const bool edge_tile = x0 <= 1 || x0 + BX >= P.nx - 1 || y0 <= 1 || y0 + BY >= P.ny - 1;
        const int seam = seam_side<BX>(P, x0);
        if (edge_tile) {
            if (tma_tile<BX, BY, S, true, false>(P, A, B, phiu, refB, st, sm, x0, y0, seam, ok, on_abort, no_refill))
                return;
            __syncthreads();  // every warp is done with stage s
            refill();
        } else if (tma_tile<BX, BY, S, false, true>(P, A, B, phiu, refB, st, sm, x0, y0, 0, ok, on_abort, refill)) {
            return;
        }
    }

    // the tiles outside the TMA rectangle (periodic seams, ragged edges) through the
    // general path, continuing this CTA's round-robin share; their ring lives in the
    // stages, which the last TMA tile may still be reading
    if (t - ntma < nedge) __syncthreads();
    for (int e = t - ntma; e < nedge; e += gridDim.x) {
        // map edge index e to the e-th tile outside the TMA rectangle
        int idx = e, bx = 0, by = 0;
        {
            // tiles in row-major order, skipping the TMA rectangle
            int row = 0;
            for (row = 0; row < tilesy; ++row) {
                const bool inner = row >= by0 && row < by0 + ntby;
                const int cnt = inner ? tilesx - ntbx : tilesx;
                if (idx < cnt) break;
                idx -= cnt;
            }
            by = row;
            const bool inner = by >= by0 && by < by0 + ntby;
            bx = (inner && idx >= bx0) ? idx + ntbx : idx;
        }
        step_tile_general<BX, BY, S>(P, A, B, phiu, refA, refB, *reinterpret_cast<RingSmem<BX, BY>*>(dsm), bx, by);
    }
}

}  // namespace tpf
