// Training and inference kernels of the warm-start U-Net (no counterpart in the
// paper): 3x3 convolutions as implicit GEMMs on the tensor cores (BF16 operands,
// FP32 accumulation, mma.sync m16n8k16), their data and weight gradients, pooling,
// upsampling, channel concatenation, the 1x1 head, the MSE loss and Adam.
// Activations are NHWC bfloat16 with channel counts that are multiples of 32;
// 3x3 weights are [9][Cout][Cin] (tap = (dh + 1) * 3 + (dw + 1)).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "../../include/tpflbm.h"
#include "../../include/tpfnet.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kBM = 64;  // output pixels per CTA (one row segment)
constexpr int kKC = 32;  // input channels per K chunk
constexpr int kPad = 8;  // smem row padding (bf16) against bank conflicts

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// y[n, h, w, co] = act(b[co] + sum_tap sum_ci x[n, h+dh, w+dw, ci] W[tap][co][ci]).
// CTA: 64 pixels of one image row x BN output channels; 4 warps, 16 pixels each.
template <int BN>
__global__ void __launch_bounds__(128)
k_conv3x3(const bf16* __restrict__ x, int N, int H, int W, int Cin, const bf16* __restrict__ wt,
          const float* __restrict__ bias, int Cout, int relu, bf16* __restrict__ y)
{
    __shared__ __align__(16) bf16 As[kBM][kKC + kPad];
    __shared__ __align__(16) bf16 Bs[BN][kKC + kPad];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tig = lane & 3;
    const int wblocks = (W + kBM - 1) / kBM;
    const int row = blockIdx.x / wblocks, w0 = (blockIdx.x % wblocks) * kBM;
    const int n = row / H, h = row % H;
    const int co0 = blockIdx.y * BN;
    constexpr int NT = BN / 8;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    for (int tap = 0; tap < 9; ++tap) {
        const int dh = tap / 3 - 1, dw = tap % 3 - 1;
        const int hh = h + dh;
        for (int c0 = 0; c0 < Cin; c0 += kKC) {
            // A: 64 pixels x 32 channels (4 x 16-byte pieces per pixel)
            for (int k = tid; k < kBM * 4; k += 128) {
                const int m = k >> 2, q = k & 3;
                const int ww = w0 + m + dw;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (hh >= 0 && hh < H && ww >= 0 && ww < W)
                    v = *reinterpret_cast<const uint4*>(x + (((size_t)n * H + hh) * W + ww) * Cin + c0 + q * 8);
                *reinterpret_cast<uint4*>(&As[m][q * 8]) = v;
            }
            // B: BN output channels x 32 input channels
            for (int k = tid; k < BN * 4; k += 128) {
                const int co = k >> 2, q = k & 3;
                *reinterpret_cast<uint4*>(&Bs[co][q * 8]) =
                    *reinterpret_cast<const uint4*>(wt + ((size_t)tap * Cout + co0 + co) * Cin + c0 + q * 8);
            }
            __syncthreads();
#pragma unroll
            for (int ks = 0; ks < kKC; ks += 16) {
                uint32_t a[4];
                const int r0 = warp * 16 + g;
                a[0] = ld_pair(&As[r0][ks + 2 * tig]);
                a[1] = ld_pair(&As[r0 + 8][ks + 2 * tig]);
                a[2] = ld_pair(&As[r0][ks + 2 * tig + 8]);
                a[3] = ld_pair(&As[r0 + 8][ks + 2 * tig + 8]);
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    uint32_t b[2];
                    b[0] = ld_pair(&Bs[j * 8 + g][ks + 2 * tig]);
                    b[1] = ld_pair(&Bs[j * 8 + g][ks + 2 * tig + 8]);
                    mma_bf16(acc[j], a, b);
                }
            }
            __syncthreads();
        }
    }
    // epilogue: bias, optional ReLU, bf16 store
#pragma unroll
    for (int j = 0; j < NT; ++j) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int m = warp * 16 + g + 8 * r;
            const int ww = w0 + m;
            if (ww >= W) continue;
            const int co = co0 + j * 8 + 2 * tig;
            float v0 = acc[j][2 * r] + (bias ? bias[co] : 0.f);
            float v1 = acc[j][2 * r + 1] + (bias ? bias[co + 1] : 0.f);
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            __nv_bfloat162 o;
            o.x = __float2bfloat16_rn(v0);
            o.y = __float2bfloat16_rn(v1);
            *reinterpret_cast<__nv_bfloat162*>(y + (((size_t)n * H + h) * W + ww) * Cout + co) = o;
        }
    }
}

// ------------------------------------------------ tcgen05 forward convolution
//
// The same convolution on the fifth-generation tensor cores: an implicit GEMM with
// M = 128 output pixels (a BW x BH block of one image, BW * BH = 128), N = BN output
// channels and K = 9 taps x Cin.  Operands are staged by TMA in swizzled K-major tiles
// of KC channels per row (64 channels: 128-byte rows and swizzle when Cin allows, else
// 32 channels: 64-byte rows and swizzle): the activation tile of a tap is the
// pixel block shifted by (dh, dw), read through a 4-D tensor map whose out-of-range
// rows and columns come back as zeros (the padding); the weight tile is BN rows of
// [9 Cout][Cin].  One thread issues the copies into a ring of kTcStages stages, one
// thread issues tcgen05.mma (M = 128, N = BN, K = 16, BF16 in, FP32 accumulated in
// tensor memory) and frees each stage with tcgen05.commit; the four warps then read
// the accumulator (warp w owns TMEM lanes 32w..32w+31, i.e. pixels), add the bias,
// apply the ReLU and store bf16.  Every wait is bounded; a wait that runs out sets
// the error flag and the CTA still releases its tensor memory.
constexpr int kTcStages = 4;
__device__ int g_tc_err;                     // a bounded wait of the tcgen05 kernel ran out

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity)
{
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(sa(b)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    atomicExch(&g_tc_err, 1);
    return false;
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* m, uint64_t* b, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            sa(dst)),
        "l"((uint64_t)m), "r"(c0), "r"(c1), "r"(sa(b))
        : "memory");
}
__device__ __forceinline__ void tma_4d(void* dst, const CUtensorMap* m, uint64_t* b, int c0, int c1, int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(sa(dst)),
        "l"((uint64_t)m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(sa(b))
        : "memory");
}
// shared-memory matrix descriptor of a K-major tile with KC bf16 (2 KC bytes) per row,
// swizzled over the row width (64 bytes: mode 4, 128 bytes: mode 2), 8-row groups
// 16 KC bytes apart (start address and strides in 16-byte units; descriptor version 1)
template <int KC>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr)
{
    static_assert(KC == 32 || KC == 64, "64- or 128-byte rows");
    constexpr uint64_t mode = KC == 64 ? 2 : 4;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(16 * KC >> 4) << 32) |
           ((uint64_t)1 << 46) | (mode << 61);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int BN, int KC>
__global__ void __launch_bounds__(128, 1)
k_conv3x3_tc(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw, int H, int W, int Cin,
             int Cout, int BW, int BH, const float* __restrict__ bias, int relu, bf16* __restrict__ y)
{
    static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "TMEM columns: a power of two from 32");
    constexpr int kABytes = 128 * KC * 2, kBBytes = BN * KC * 2;
    constexpr int kStage = kABytes + kBBytes;  // multiple of 1024
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 1024-byte aligned stages (the swizzle pattern repeats every 512 bytes)
    unsigned char* st0 = tsm + ((1024 - (sa(tsm) & 1023)) & 1023);
    const int bpr = W / BW, bpi = bpr * (H / BH);  // pixel blocks per row of blocks, per image
    const int n = blockIdx.x / bpi, rem = blockIdx.x % bpi;
    const int h0 = (rem / bpr) * BH, w0 = (rem % bpr) * BW;
    const int co0 = blockIdx.y * BN;
    const int kc = Cin / KC, ksteps = 9 * kc;

    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        mb_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer: stage k % S holds tap k / kc, channels (k % kc) * 32
        int issued = 0;
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kTcStages;
            if (k >= kTcStages && !mb_wait(&empty[s], ((k / kTcStages) - 1) & 1)) break;
            unsigned char* a = st0 + s * kStage;
            const int tap = k / kc, c0 = (k % kc) * KC;
            mb_expect_tx(&full[s], kStage);
            tma_4d(a, &mx, &full[s], c0, w0 + tap % 3 - 1, h0 + tap / 3 - 1, n);
            tma_2d(a + kABytes, &mw, &full[s], c0, tap * Cout + co0);
            issued = k + 1;
        }
        // copies still in flight (only after a wait ran out) land before the CTA ends
        for (int k = issued > kTcStages ? issued - kTcStages : 0; k < issued; ++k)
            mb_wait(&full[k % kTcStages], (k / kTcStages) & 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = tc_idesc(128, BN);
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kTcStages;
            if (!mb_wait(&full[s], (k / kTcStages) & 1)) break;
            tc_fence_after();
            const uint32_t a = sa(st0 + s * kStage), b = a + kABytes;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
                const uint64_t ad = kmajor_desc<KC>(a + 32 * kk), bd = kmajor_desc<KC>(b + 32 * kk);
                const uint32_t acc = (k | kk) != 0;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            // stage s is free once these MMAs have read it
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             sa(&empty[s]))
                         : "memory");
        }
        // the accumulator is complete once every MMA issued has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(&done))
                     : "memory");
    }
    __syncwarp();

    // epilogue: thread (warp w, lane l) owns pixel 32 w + l of the block
    mb_wait(&done, 0);
    tc_fence_after();
    const int m = warp * 32 + lane;
    const int hh = h0 + m / BW, ww = w0 + m % BW;
    bf16* out = y + (((size_t)n * H + hh) * W + ww) * Cout + co0;
#pragma unroll 1
    for (int c = 0; c < BN; c += 8) {
        uint32_t r[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v0 = __uint_as_float(r[2 * j]) + (bias ? bias[co0 + c + 2 * j] : 0.f);
            float v1 = __uint_as_float(r[2 * j + 1]) + (bias ? bias[co0 + c + 2 * j + 1] : 0.f);
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            __nv_bfloat162 t;
            t.x = __float2bfloat16_rn(v0);
            t.y = __float2bfloat16_rn(v1);
            o[j] = *reinterpret_cast<uint32_t*>(&t);
        }
        *reinterpret_cast<uint4*>(out + c) = make_uint4(o[0], o[1], o[2], o[3]);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// dW[tap][co][ci] += sum_p dz[p][co] x[p + off(tap)][ci], db[co] += sum_p dz[p][co].
// CTA: one tap, WM co x 32 ci, a chunk of 32 pixels at a time over its pixel range;
// accumulates in FP32 and adds into dW with atomics.  4 warps: WM/16 row blocks of
// 16 output channels times 64/WM groups of n-tiles.
constexpr int kWN = 32, kWK = 32;
template <int WM>
__global__ void __launch_bounds__(128)
k_conv3x3_wgrad(const bf16* __restrict__ x, const bf16* __restrict__ dz, int N, int H, int W, int Cin, int Cout,
                int pix_per_cta, float* __restrict__ dw, float* __restrict__ db)
{
    constexpr int RB = WM / 16;        // row blocks
    constexpr int NG = 4 / RB;         // n-tile groups
    constexpr int NTW = 4 / NG;        // n-tiles (of 8 ci) per warp
    __shared__ __align__(16) bf16 Az[WM][kWK + kPad];   // [co][p]
    __shared__ __align__(16) bf16 Bx[kWN][kWK + kPad];  // [ci][p]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tig = lane & 3;
    const int rb = warp % RB, ng = warp / RB;
    const int tap = blockIdx.z % 9, split = blockIdx.z / 9;
    const int dh = tap / 3 - 1, dwd = tap % 3 - 1;
    const int co0 = blockIdx.y * WM, ci0 = blockIdx.x * kWN;
    const long long P = (long long)N * H * W;
    const long long p_begin = (long long)split * pix_per_cta;
    const long long p_end = p_begin + pix_per_cta < P ? p_begin + pix_per_cta : P;
    float acc[NTW][4];
#pragma unroll
    for (int j = 0; j < NTW; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    float bacc = 0.f;
    const bool do_bias = db && tap == 4 && blockIdx.x == 0;

    for (long long p0 = p_begin; p0 < p_end; p0 += kWK) {
        // dz tile: 32 pixels x WM co -> Az[co][p]
        for (int k = tid; k < kWK * WM; k += 128) {
            const int pl = k / WM, co = k % WM;
            const long long p = p0 + pl;
            bf16 v = __float2bfloat16_rn(0.f);
            if (p < p_end) v = dz[p * Cout + co0 + co];
            Az[co][pl] = v;
        }
        // x tile at the tap offset: 32 pixels x 32 ci -> Bx[ci][p]
        for (int k = tid; k < kWK * kWN; k += 128) {
            const int pl = k / kWN, ci = k % kWN;
            const long long p = p0 + pl;
            bf16 v = __float2bfloat16_rn(0.f);
            if (p < p_end) {
                const int w = (int)(p % W), hrow = (int)((p / W) % H), nn = (int)(p / ((long long)W * H));
                const int hh = hrow + dh, ww = w + dwd;
                if (hh >= 0 && hh < H && ww >= 0 && ww < W) v = x[(((long long)nn * H + hh) * W + ww) * Cin + ci0 + ci];
            }
            Bx[ci][pl] = v;
        }
        __syncthreads();
        if (do_bias && tid < WM) {
            for (int pl = 0; pl < kWK; ++pl) bacc += __bfloat162float(Az[tid][pl]);
        }
#pragma unroll
        for (int ks = 0; ks < kWK; ks += 16) {
            uint32_t a[4];
            const int r0 = rb * 16 + g;
            a[0] = ld_pair(&Az[r0][ks + 2 * tig]);
            a[1] = ld_pair(&Az[r0 + 8][ks + 2 * tig]);
            a[2] = ld_pair(&Az[r0][ks + 2 * tig + 8]);
            a[3] = ld_pair(&Az[r0 + 8][ks + 2 * tig + 8]);
#pragma unroll
            for (int j = 0; j < NTW; ++j) {
                const int nt = ng * NTW + j;
                uint32_t b[2];
                b[0] = ld_pair(&Bx[nt * 8 + g][ks + 2 * tig]);
                b[1] = ld_pair(&Bx[nt * 8 + g][ks + 2 * tig + 8]);
                mma_bf16(acc[j], a, b);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int co = co0 + rb * 16 + g + 8 * r;
            const int ci = ci0 + (ng * NTW + j) * 8 + 2 * tig;
            float* dst = dw + ((size_t)tap * Cout + co) * Cin + ci;
            atomicAdd(dst, acc[j][2 * r]);
            atomicAdd(dst + 1, acc[j][2 * r + 1]);
        }
    }
    if (do_bias && tid < WM) atomicAdd(db + co0 + tid, bacc);
}

// ------------------------------------------------ tcgen05 weight gradient
//
// dW[tap][co][ci] += sum_p dz[p][co] x[p + off(tap)][ci] as GEMMs with M = 128 output
// channels (co), N = 64 input channels (ci) and K = pixels, over a range of 64-pixel
// row segments per CTA (split over CTAs, partial sums added with FP32 atomics), for one
// tap or for the three taps of one column offset, which share each dz box (one 64-column
// TMEM accumulator per tap).  The reduction runs over pixels, which NHWC stores outermost, so both
// operands are staged MN-major: a TMA box of 64 channels (128 bytes, 128-byte
// swizzle) by 64 pixels puts one pixel's channels in each 128-byte row.  A is two such
// boxes of dz (co0 and co0 + 64), B one box of x at the tap's shifted pixels
// (w0 + dw, h + dh), whose out-of-range pixels and channels arrive as zeros (the
// padding, and the channels past Cin or Cout).  The tap's shift is on the pixel
// coordinates, never on the innermost (channel) one, so every copy starts on a
// 16-byte boundary.  Same roles as the forward kernel: one thread copies, one thread
// issues tcgen05.mma (FP32 accumulator in 64 TMEM columns), four warps read TMEM and
// add into dW.
constexpr int kWgStages = 4;
constexpr int kWgPix = 64;   // pixels per K step (one row segment)
// taps per CTA: one, or the three rows (dh) of one column offset (dw), which share their
// dz boxes; three measured faster from 2^17 pixels up (the 512 x 128 level), one below
constexpr long long kWgTaps3Pixels = 1 << 17;

// shared-memory matrix descriptor of an MN-major tile: 128-byte rows of 64 bf16 along
// M (or N), one row per K index, 128-byte swizzle; blocks of 64 along M lbo bytes
// apart, groups of 8 rows 1024 bytes apart (descriptor version 1)
__device__ __forceinline__ uint64_t mnmajor_desc(uint32_t addr, uint32_t lbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

template <int TAPS>
__global__ void __launch_bounds__(128, 1)
k_conv3x3_wgrad_tc(const __grid_constant__ CUtensorMap mdz, const __grid_constant__ CUtensorMap mx, int N, int H,
                   int W, int Cin, int Cout, int chunks_per_cta, float* __restrict__ dw)
{
    static_assert(TAPS == 1 || TAPS == 3, "one tap, or the three rows of one column offset");
    constexpr int kBlk = kWgPix * 128;      // one 64-channel x 64-pixel box
    constexpr int kStage = (2 + TAPS) * kBlk;  // A: two boxes (128 co), B: one box (64 ci) per tap
    constexpr uint32_t kCols = TAPS == 1 ? 64 : 256;  // TMEM columns: 64 per tap, a power of two
    // MN-major A and B (transpose bits), FP32 accumulator, BF16 operands, M 128, N 64
    constexpr uint32_t idesc = tc_idesc(128, 64) | (1u << 15) | (1u << 16);
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t full[kWgStages], empty[kWgStages], done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* st0 = tsm + ((1024 - (sa(tsm) & 1023)) & 1023);
    const int co0 = blockIdx.x * 128, ci0 = blockIdx.y * 64;
    // TAPS 1: tap = z % 9; TAPS 3: taps dwi, dwi + 3, dwi + 6 (dh = -1, 0, 1) with dwi = z % 3
    constexpr int kGroups = 9 / TAPS;
    const int g = blockIdx.z % kGroups, split = blockIdx.z / kGroups;
    const int tap0 = g;  // the CTA's first tap (dh = -1 when TAPS is 3)
    const int dwd = tap0 % 3 - 1;
    const int segs = W / kWgPix, nchunks = N * H * segs;
    const int c_begin = split * chunks_per_cta;
    const int c_end = min(c_begin + chunks_per_cta, nchunks);
    const int ksteps = c_end > c_begin ? c_end - c_begin : 0;

    if (tid == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        mb_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kWgStages;
            if (k >= kWgStages && !mb_wait(&empty[s], ((k / kWgStages) - 1) & 1)) break;
            const int c = c_begin + k, row = c / segs;  // row = n * H + h
            const int w0 = (c - row * segs) * kWgPix, n = row / H, h = row - n * H;
            unsigned char* a = st0 + s * kStage;
            // the second dz box only when it holds channels: otherwise TMEM lanes 64-127
            // accumulate whatever that smem holds and are never read
            const bool a2 = co0 + 64 < Cout;
            mb_expect_tx(&full[s], a2 ? kStage : kStage - kBlk);
            tma_4d(a, &mdz, &full[s], co0, w0, h, n);
            if (a2) tma_4d(a + kBlk, &mdz, &full[s], co0 + 64, w0, h, n);
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const int dh = (tap0 + 3 * t) / 3 - 1;
                tma_4d(a + (2 + t) * kBlk, &mx, &full[s], ci0, w0 + dwd, h + dh, n);
            }
            issued = k + 1;
        }
        for (int k = issued > kWgStages ? issued - kWgStages : 0; k < issued; ++k)
            mb_wait(&full[k % kWgStages], (k / kWgStages) & 1);
    } else if (warp == 1 && lane == 0) {
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kWgStages;
            if (!mb_wait(&full[s], (k / kWgStages) & 1)) break;
            tc_fence_after();
            const uint32_t a = sa(st0 + s * kStage);
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const uint32_t b = a + (2 + t) * kBlk;
#pragma unroll
                for (int kk = 0; kk < kWgPix / 16; ++kk) {
                    // 16 K rows = two 8-row groups
                    const uint64_t ad = mnmajor_desc(a + 2048 * kk, kBlk), bd = mnmajor_desc(b + 2048 * kk, kBlk);
                    const uint32_t acc = (k | kk) != 0;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 64 * t),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             sa(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(&done))
                     : "memory");
    }
    __syncwarp();

    // thread (warp w, lane l) owns output channel co0 + 32 w + l (TMEM lane 32 w + l)
    mb_wait(&done, 0);
    tc_fence_after();
    const int co = co0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < 64 * TAPS; c += 8) {
        uint32_t r[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int tap = tap0 + 3 * (c / 64), cc = c % 64;
        if (ksteps > 0 && co < Cout) {
            float* dst = dw + ((size_t)tap * Cout + co) * Cin + ci0 + cc;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (ci0 + cc + j < Cin) atomicAdd(dst + j, __uint_as_float(r[j]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// db[co] += sum_p dz[p][co]: one thread per channel per pixel range
__global__ void k_bias_grad(const bf16* __restrict__ dz, long long P, int Cout, long long per, float* __restrict__ db)
{
    const int co = blockIdx.x * blockDim.x + threadIdx.x;
    if (co >= Cout) return;
    const long long p0 = (long long)blockIdx.y * per, p1 = p0 + per < P ? p0 + per : P;
    float acc = 0.f;
    for (long long p = p0; p < p1; ++p) acc += __bfloat162float(dz[p * Cout + co]);
    atomicAdd(db + co, acc);
}

// flipped transpose for the data gradient: wd[tap][ci][co] = w[8 - tap][co][ci]
__global__ void k_flip_weights(const bf16* __restrict__ w, int Cin, int Cout, bf16* __restrict__ wd)
{
    const long long total = 9LL * Cin * Cout;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(k % Cout);
        const long long r = k / Cout;
        const int ci = (int)(r % Cin), tap = (int)(r / Cin);
        wd[k] = w[((size_t)(8 - tap) * Cout + co) * Cin + ci];
    }
}

__global__ void k_relu_mask(bf16* __restrict__ d, const bf16* __restrict__ y, long long count)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(y[k]) > 0.f)) d[k] = __float2bfloat16_rn(0.f);
}

// 2x2 average pooling and its adjoint; nearest upsampling and its adjoint
__global__ void k_pool(const bf16* __restrict__ x, int N, int H, int W, int C, bf16* __restrict__ y)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Ho * Wo * C;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        long long r = k / C;
        const int wo = (int)(r % Wo); r /= Wo;
        const int ho = (int)(r % Ho);
        const int n = (int)(r / Ho);
        const size_t b = (((size_t)n * H + 2 * ho) * W + 2 * wo) * C + c;
        const float s = __bfloat162float(x[b]) + __bfloat162float(x[b + C]) + __bfloat162float(x[b + (size_t)W * C]) +
                        __bfloat162float(x[b + (size_t)W * C + C]);
        y[k] = __float2bfloat16_rn(0.25f * s);
    }
}
// dx[fine] (+)= dy[coarse] / 4
__global__ void k_pool_back(const bf16* __restrict__ dy, int N, int H, int W, int C, bf16* __restrict__ dx, int accumulate)
{
    const long long total = (long long)N * H * W * C;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        long long r = k / C;
        const int w = (int)(r % W); r /= W;
        const int hh = (int)(r % H);
        const int n = (int)(r / H);
        float v = 0.25f * __bfloat162float(dy[(((size_t)n * (H / 2) + hh / 2) * (W / 2) + w / 2) * C + c]);
        if (accumulate) v += __bfloat162float(dx[k]);
        dx[k] = __float2bfloat16_rn(v);
    }
}
// y[n, h, w, cofs + c] = x[n, h/2, w/2, c] : upsampled x into channels [cofs, cofs + C) of a Ctot tensor
__global__ void k_up_into(const bf16* __restrict__ x, int N, int H, int W, int C, bf16* __restrict__ y, int Ctot, int cofs)
{
    const long long total = (long long)N * H * W * C;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        long long r = k / C;
        const int w = (int)(r % W); r /= W;
        const int hh = (int)(r % H);
        const int n = (int)(r / H);
        y[(((size_t)n * H + hh) * W + w) * Ctot + cofs + c] = x[(((size_t)n * (H / 2) + hh / 2) * (W / 2) + w / 2) * C + c];
    }
}
// dx[coarse] = sum of the 4 fine dy values in channels [cofs, cofs + C) of a Ctot tensor
__global__ void k_up_back(const bf16* __restrict__ dy, int N, int H, int W, int Ctot, int cofs, int C, bf16* __restrict__ dx)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Ho * Wo * C;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        long long r = k / C;
        const int wo = (int)(r % Wo); r /= Wo;
        const int ho = (int)(r % Ho);
        const int n = (int)(r / Ho);
        const size_t b = (((size_t)n * H + 2 * ho) * W + 2 * wo) * Ctot + cofs + c;
        const float s = __bfloat162float(dy[b]) + __bfloat162float(dy[b + Ctot]) +
                        __bfloat162float(dy[b + (size_t)W * Ctot]) + __bfloat162float(dy[b + (size_t)W * Ctot + Ctot]);
        dx[k] = __float2bfloat16_rn(s);
    }
}
// copy channels [sofs, sofs + C) of an Sc-channel tensor into channels [dofs, dofs + C) of a Dc-channel
// tensor (concatenation and its adjoint split); accumulate adds into the destination
__global__ void k_channels(const bf16* __restrict__ src, int Sc, int sofs, long long pixels, int C, bf16* __restrict__ dst,
                           int Dc, int dofs, int accumulate)
{
    const long long total = pixels * C;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        const long long p = k / C;
        float v = __bfloat162float(src[p * Sc + sofs + c]);
        bf16* d = dst + p * Dc + dofs + c;
        if (accumulate) v += __bfloat162float(*d);
        *d = __float2bfloat16_rn(v);
    }
}

// 1x1 head: out[p][o] = b[o] + sum_c x[p][c] W[c][o] (FP32 weights and output)
__global__ void k_head(const bf16* __restrict__ x, long long pixels, int C, const float* __restrict__ Wt,
                       const float* __restrict__ b, int Cout, float* __restrict__ out)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < pixels * Cout; k += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(k % Cout);
        const long long p = k / Cout;
        float s = b[o];
        for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(x[p * C + c]), Wt[c * Cout + o], s);
        out[k] = s;
    }
}
// head gradients: dx[p][c] = sum_o dout[p][o] W[c][o]; dW[c][o] += sum_p x[p][c] dout[p][o]; db[o] += sum_p dout[p][o]
__global__ void k_head_back(const bf16* __restrict__ x, const float* __restrict__ dout, long long pixels, int C,
                            const float* __restrict__ Wt, int Cout, bf16* __restrict__ dx, float* __restrict__ dW,
                            float* __restrict__ db)
{
    extern __shared__ float sh[];  // C * Cout + Cout partial sums
    for (int k = threadIdx.x; k < C * Cout + Cout; k += blockDim.x) sh[k] = 0.f;
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pixels; p += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < C; ++c) {
            float s = 0.f;
            const float xv = __bfloat162float(x[p * C + c]);
            for (int o = 0; o < Cout; ++o) {
                const float d = dout[p * Cout + o];
                s = fmaf(d, Wt[c * Cout + o], s);
                atomicAdd(&sh[c * Cout + o], xv * d);
            }
            dx[p * C + c] = __float2bfloat16_rn(s);
        }
        for (int o = 0; o < Cout; ++o) atomicAdd(&sh[C * Cout + o], dout[p * Cout + o]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C * Cout; k += blockDim.x) atomicAdd(&dW[k], sh[k]);
    for (int k = threadIdx.x; k < Cout; k += blockDim.x) atomicAdd(&db[k], sh[C * Cout + k]);
}

// mean squared error with channel weights; grad = d loss / d pred; loss accumulated in FP64
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, const float* __restrict__ wch,
                      long long count, int C, float* __restrict__ grad, double* __restrict__ loss)
{
    double acc = 0.0;
    const float inv = 1.f / (float)count;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x) {
        const float wc = wch ? wch[k % C] : 1.f;
        const float d = pred[k] - target[k];
        acc += (double)d * d * wc;
        if (grad) grad[k] = 2.f * d * wc * inv;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (double)count);
}

// Adam on FP32 master weights, refreshing the bf16 copy used by the convolutions
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       long long count, float lr, float b1, float b2, float eps, float c1, float c2,
                       bf16* __restrict__ pb)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x) {
        const float gk = gr[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float pk = p[k] - lr * (mk * c1) / (sqrtf(vk * c2) + eps);
        p[k] = pk;
        if (pb) pb[k] = __float2bfloat16_rn(pk);
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, long long count, bf16* __restrict__ y)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x)
        y[k] = __float2bfloat16_rn(x[k]);
}

// planar float fields <-> interleaved NHWC tensors, with a per-channel affine map
constexpr int kMaxPackC = 8;
struct Affine {
    float scale[kMaxPackC], shift[kMaxPackC];
};
__global__ void k_pack(const float* __restrict__ src, const float* __restrict__ base, long long plane, int C,
                       long long pixels, Affine a, void* __restrict__ dst, int Cd, int bf)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < pixels * C; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        const long long p = k / C;
        const float d = src[c * plane + p] - (base ? base[c * plane + p] : 0.f);
        const float v = fmaf(d, a.scale[c], a.shift[c]);
        if (bf) ((bf16*)dst)[p * Cd + c] = __float2bfloat16_rn(v);
        else ((float*)dst)[p * Cd + c] = v;
    }
}
__global__ void k_unpack(const float* __restrict__ src, long long pixels, int C, Affine a, const float* __restrict__ base,
                         float* __restrict__ dst, long long plane)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < pixels * C; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        const long long p = k / C;
        dst[c * plane + p] = fmaf(src[k], a.scale[c], a.shift[c]) + (base ? base[c * plane + p] : 0.f);
    }
}

int grid_of(long long count)
{
    long long b = (count + 255) / 256;
    return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

int status(cudaError_t e) { return e == cudaSuccess ? TPF_OK : TPF_ERR_CUDA; }

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

// Shapes the tcgen05 convolution takes: pixel blocks of BW x BH = 128 (BW = W up to
// 128, dividing W; BH dividing H).  BN: the largest of 256, 128, 64, 32 that divides
// Cout and still gives at least one CTA per SM (else 32).  0 when the shape is not
// taken.
int tc_bn(int N, int H, int W, int Cout, int& BW, int& BH)
{
    BW = W < 128 ? W : 128;
    if (128 % BW != 0 || W % BW != 0) return 0;
    BH = 128 / BW;
    if (H % BH != 0) return 0;
    const long long mtiles = (long long)N * (H / BH) * (W / BW);
    for (int bn = 256; bn > 32; bn /= 2)
        if (Cout % bn == 0 && mtiles * (Cout / bn) >= 152) return bn;
    return 32;
}

// The tcgen05 convolution for 16-byte aligned tensors of a shape tc_bn takes; returns
// false (nothing launched) otherwise.
template <int BN, int KC>
bool launch_tc(const bf16* x, int N, int H, int W, int Cin, const bf16* wt, const float* bias, int Cout, int relu,
               bf16* y, cudaStream_t s, int BW, int BH)
{
    auto fn = encode_fn();
    if (!fn) return false;
    CUtensorMap mx, mw;
    {
        cuuint64_t dims[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
        cuuint64_t strides[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
        cuuint32_t box[4] = {(cuuint32_t)KC, (cuuint32_t)BW, (cuuint32_t)BH, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (fn(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)x, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               KC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return false;
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)Cin, (cuuint64_t)9 * Cout};
        cuuint64_t strides[1] = {(cuuint64_t)Cin * 2};
        cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)BN};
        cuuint32_t es[2] = {1, 1};
        if (fn(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)wt, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               KC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return false;
    }
    const int smem = kTcStages * (128 + BN) * KC * 2 + 1024;
    // set on every call: the attribute belongs to the current device
    if (cudaFuncSetAttribute(k_conv3x3_tc<BN, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    dim3 grd(N * (H / BH) * (W / BW), Cout / BN);
    k_conv3x3_tc<BN, KC><<<grd, 128, smem, s>>>(mx, mw, H, W, Cin, Cout, BW, BH, bias, relu, y);
    return true;
}

bool conv_tc(const bf16* x, int N, int H, int W, int Cin, const bf16* wt, const float* bias, int Cout, int relu,
             bf16* y, cudaStream_t s)
{
    int BW = 0, BH = 0;
    const int bn = tc_bn(N, H, W, Cout, BW, BH);
    if (!bn || (((uintptr_t)x | (uintptr_t)wt | (uintptr_t)y) & 15)) return false;
    if (Cin % 64 == 0) {
        switch (bn) {
        case 256: return launch_tc<256, 64>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
        case 128: return launch_tc<128, 64>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
        case 64: return launch_tc<64, 64>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
        default: return launch_tc<32, 64>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
        }
    }
    switch (bn) {
    case 256: return launch_tc<256, 32>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
    case 128: return launch_tc<128, 32>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
    case 64: return launch_tc<64, 32>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
    default: return launch_tc<32, 32>(x, N, H, W, Cin, wt, bias, Cout, relu, y, s, BW, BH);
    }
}

// The tcgen05 weight gradient for W a multiple of 64 and 16-byte aligned tensors;
// false (nothing launched) otherwise.  Adds into dw (and db).
bool wgrad_tc(const bf16* x, const bf16* dz, int N, int H, int W, int Cin, int Cout, float* dw, float* db,
              cudaStream_t s)
{
    if (W % kWgPix != 0 || (((uintptr_t)x | (uintptr_t)dz) & 15)) return false;
    auto fn = encode_fn();
    if (!fn) return false;
    CUtensorMap mdz, mx;
    auto make = [&](CUtensorMap* m, const bf16* base, int C) {
        cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
        cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
        cuuint32_t box[4] = {64, (cuuint32_t)kWgPix, 1, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!make(&mdz, dz, Cout) || !make(&mx, x, Cin)) return false;
    const long long P = (long long)N * H * W;
    const int taps = P >= kWgTaps3Pixels ? 3 : 1;
    const int smem = kWgStages * (2 + taps) * kWgPix * 128 + 1024;
    if (cudaFuncSetAttribute(taps == 3 ? (const void*)k_conv3x3_wgrad_tc<3> : (const void*)k_conv3x3_wgrad_tc<1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // split the pixel segments so that the grid fills the GPU about twice
    const long long nchunks = (long long)N * H * (W / kWgPix);
    const int ctiles = (Cout + 127) / 128, itiles = (Cin + 63) / 64;
    const long long base = (9 / taps) * (long long)ctiles * itiles;
    const long long target = taps == 1 ? 2 * 152 : 152;  // CTAs per SM the shared memory allows
    long long splits = (target + base - 1) / base;
    if (splits > nchunks) splits = nchunks;
    if (splits < 1) splits = 1;
    const long long per = (nchunks + splits - 1) / splits;
    splits = (nchunks + per - 1) / per;
    dim3 grd(ctiles, itiles, (9 / taps) * (unsigned)splits);
    if (taps == 3)
        k_conv3x3_wgrad_tc<3><<<grd, 128, smem, s>>>(mdz, mx, N, H, W, Cin, Cout, (int)per, dw);
    else
        k_conv3x3_wgrad_tc<1><<<grd, 128, smem, s>>>(mdz, mx, N, H, W, Cin, Cout, (int)per, dw);
    if (db) {
        const long long ys = P < 256 ? P : 256, pper = (P + ys - 1) / ys;
        k_bias_grad<<<dim3((Cout + 127) / 128, (unsigned)((P + pper - 1) / pper)), 128, 0, s>>>(dz, P, Cout, pper, db);
    }
    return true;
}

}  // namespace

extern "C" {

int tpfnet_conv3x3(const void* x, int N, int H, int W, int Cin, const void* wt, const float* bias, int Cout, int relu,
                   void* y, void* stream)
{
    if (!x || !wt || !y || N < 1 || H < 1 || W < 1 || Cin % kKC || Cout % 32) return TPF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (conv_tc((const bf16*)x, N, H, W, Cin, (const bf16*)wt, bias, Cout, relu, (bf16*)y, s))
        return status(cudaGetLastError());
    const int wblocks = (W + kBM - 1) / kBM;
    if (Cout % 64 == 0) {
        dim3 grd(wblocks * N * H, Cout / 64);
        k_conv3x3<64><<<grd, 128, 0, s>>>((const bf16*)x, N, H, W, Cin, (const bf16*)wt, bias, Cout, relu, (bf16*)y);
    } else {
        dim3 grd(wblocks * N * H, Cout / 32);
        k_conv3x3<32><<<grd, 128, 0, s>>>((const bf16*)x, N, H, W, Cin, (const bf16*)wt, bias, Cout, relu, (bf16*)y);
    }
    return status(cudaGetLastError());
}

int tpfnet_conv3x3_tcgen05(int N, int H, int W, int Cin, int Cout)
{
    int BW = 0, BH = 0;
    if (N < 1 || H < 1 || W < 1 || Cin % kKC || Cout % 32 || !encode_fn()) return 0;
    return tc_bn(N, H, W, Cout, BW, BH);
}

int tpfnet_conv3x3_wgrad_tcgen05(int N, int H, int W, int Cin, int Cout)
{
    return N >= 1 && H >= 1 && W >= 1 && Cin % 32 == 0 && Cout % 32 == 0 && W % kWgPix == 0 && encode_fn() ? 1 : 0;
}

int tpfnet_status(void)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(int)) != cudaSuccess) return TPF_ERR_CUDA;
    return v ? TPF_ERR_TIMEOUT : TPF_OK;
}

int tpfnet_conv3x3_dgrad(const void* dz, int N, int H, int W, int Cout, const void* wt, int Cin, void* wflip, void* dx,
                         void* stream)
{
    if (!dz || !wt || !wflip || !dx || Cin % 32 || Cout % kKC) return TPF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_flip_weights<<<grid_of(9LL * Cin * Cout), 256, 0, s>>>((const bf16*)wt, Cin, Cout, (bf16*)wflip);
    int rc = status(cudaGetLastError());
    if (rc) return rc;
    return tpfnet_conv3x3(dz, N, H, W, Cout, wflip, nullptr, Cin, 0, dx, stream);
}

int tpfnet_conv3x3_wgrad(const void* x, const void* dz, int N, int H, int W, int Cin, int Cout, float* dw, float* db,
                         void* stream)
{
    if (!x || !dz || !dw || Cin % kWN || Cout % 32) return TPF_ERR_INVALID_ARG;
    if (wgrad_tc((const bf16*)x, (const bf16*)dz, N, H, W, Cin, Cout, dw, db, (cudaStream_t)stream))
        return status(cudaGetLastError());
    const int WM = Cout % 64 == 0 ? 64 : 32;
    const long long P = (long long)N * H * W;
    // split the pixels so that the grid fills the GPU a few times over
    const long long ctas_per_split = 9LL * (Cin / kWN) * (Cout / WM);
    long long splits = (152LL * 8 + ctas_per_split - 1) / ctas_per_split;
    const long long maxsplits = (P + kWK - 1) / kWK;
    if (splits > maxsplits) splits = maxsplits;
    if (splits < 1) splits = 1;
    long long per = (P + splits - 1) / splits;
    per = (per + kWK - 1) / kWK * kWK;
    splits = (P + per - 1) / per;
    dim3 grd(Cin / kWN, Cout / WM, 9 * (int)splits);
    if (WM == 64)
        k_conv3x3_wgrad<64><<<grd, 128, 0, (cudaStream_t)stream>>>((const bf16*)x, (const bf16*)dz, N, H, W, Cin, Cout,
                                                                   (int)per, dw, db);
    else
        k_conv3x3_wgrad<32><<<grd, 128, 0, (cudaStream_t)stream>>>((const bf16*)x, (const bf16*)dz, N, H, W, Cin, Cout,
                                                                   (int)per, dw, db);
    return status(cudaGetLastError());
}

int tpfnet_relu_mask(void* d, const void* y, long long count, void* stream)
{
    k_relu_mask<<<grid_of(count), 256, 0, (cudaStream_t)stream>>>((bf16*)d, (const bf16*)y, count);
    return status(cudaGetLastError());
}

int tpfnet_pool(const void* x, int N, int H, int W, int C, void* y, void* stream)
{
    if (H % 2 || W % 2) return TPF_ERR_INVALID_ARG;
    k_pool<<<grid_of((long long)N * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, N, H, W, C, (bf16*)y);
    return status(cudaGetLastError());
}

int tpfnet_pool_back(const void* dy, int N, int H, int W, int C, void* dx, int accumulate, void* stream)
{
    k_pool_back<<<grid_of((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, N, H, W, C, (bf16*)dx,
                                                                                    accumulate);
    return status(cudaGetLastError());
}

int tpfnet_up_into(const void* x, int N, int H, int W, int C, void* y, int Ctot, int cofs, void* stream)
{
    k_up_into<<<grid_of((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, N, H, W, C, (bf16*)y,
                                                                                  Ctot, cofs);
    return status(cudaGetLastError());
}

int tpfnet_up_back(const void* dy, int N, int H, int W, int Ctot, int cofs, int C, void* dx, void* stream)
{
    k_up_back<<<grid_of((long long)N * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, N, H, W, Ctot, cofs,
                                                                                       C, (bf16*)dx);
    return status(cudaGetLastError());
}

int tpfnet_channels(const void* src, int Sc, int sofs, long long pixels, int C, void* dst, int Dc, int dofs,
                    int accumulate, void* stream)
{
    k_channels<<<grid_of(pixels * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)src, Sc, sofs, pixels, C, (bf16*)dst, Dc,
                                                                     dofs, accumulate);
    return status(cudaGetLastError());
}

int tpfnet_head(const void* x, long long pixels, int C, const float* Wt, const float* b, int Cout, float* out,
                void* stream)
{
    k_head<<<grid_of(pixels * Cout), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, pixels, C, Wt, b, Cout, out);
    return status(cudaGetLastError());
}

int tpfnet_head_back(const void* x, const float* dout, long long pixels, int C, const float* Wt, int Cout, void* dx,
                     float* dW, float* db, void* stream)
{
    const int smem = (C * Cout + Cout) * (int)sizeof(float);
    if (smem > 48 * 1024) return TPF_ERR_INVALID_ARG;
    k_head_back<<<grid_of(pixels) < 304 ? grid_of(pixels) : 304, 256, smem, (cudaStream_t)stream>>>(
        (const bf16*)x, dout, pixels, C, Wt, Cout, (bf16*)dx, dW, db);
    return status(cudaGetLastError());
}

int tpfnet_mse(const float* pred, const float* target, const float* wch, long long count, int C, float* grad,
               double* loss, void* stream)
{
    k_mse<<<grid_of(count) < 1024 ? grid_of(count) : 1024, 256, 0, (cudaStream_t)stream>>>(pred, target, wch, count, C, grad,
                                                                                          loss);
    return status(cudaGetLastError());
}

int tpfnet_adam(float* p, const float* g, float* m, float* v, long long count, float lr, float b1, float b2, float eps,
                int step, void* pb, void* stream)
{
    const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    k_adam<<<grid_of(count), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2, (bf16*)pb);
    return status(cudaGetLastError());
}

static int affine_of(int C, const float* scale, const float* shift, Affine* a)
{
    if (C < 1 || C > kMaxPackC) return TPF_ERR_INVALID_ARG;
    for (int c = 0; c < C; ++c) {
        a->scale[c] = scale ? scale[c] : 1.f;
        a->shift[c] = shift ? shift[c] : 0.f;
    }
    return TPF_OK;
}

int tpfnet_pack(const float* src, const float* base, long long plane, int C, long long pixels, const float* scale,
                const float* shift, void* dst, int Cd, int dst_bf16, void* stream)
{
    Affine a;
    if (!src || !dst || Cd < C || plane < pixels || affine_of(C, scale, shift, &a)) return TPF_ERR_INVALID_ARG;
    k_pack<<<grid_of(pixels * C), 256, 0, (cudaStream_t)stream>>>(src, base, plane, C, pixels, a, dst, Cd,
                                                                 dst_bf16 ? 1 : 0);
    return status(cudaGetLastError());
}

int tpfnet_unpack(const float* src, long long pixels, int C, const float* scale, const float* shift, const float* base,
                  float* dst, long long plane, void* stream)
{
    Affine a;
    if (!src || !dst || plane < pixels || affine_of(C, scale, shift, &a)) return TPF_ERR_INVALID_ARG;
    k_unpack<<<grid_of(pixels * C), 256, 0, (cudaStream_t)stream>>>(src, pixels, C, a, base, dst, plane);
    return status(cudaGetLastError());
}

int tpfnet_to_bf16(const float* x, long long count, void* y, void* stream)
{
    k_to_bf16<<<grid_of(count), 256, 0, (cudaStream_t)stream>>>(x, count, (bf16*)y);
    return status(cudaGetLastError());
}

}  // extern "C"
