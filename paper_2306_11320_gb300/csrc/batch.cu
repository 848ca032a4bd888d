// Batched ensemble: many independent lattices of uneven sizes and parameters
// advanced together by one persistent step launch per time step, replayed from a
// CUDA graph, with the tile shape chosen by timing every compiled shape.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/tpflbm.h"
#include "handle.h"
#include "lattice.cuh"
#include "step.cuh"

using namespace tpf;

namespace {

// One lattice of the ensemble as the batch kernel sees it.
struct InstDesc {
    DevParams P;
    void* pop[2];
    RefT* ref[2];
    float* phiu;
};

// Variants the autotuner chooses from: four tile shapes of the general tile path (BX x
// BY nodes, one thread per node) and, last, the TMA-staged path with 32 x 8 tiles.
constexpr int kNumVariants = 5;
constexpr int kTmaVariant = 4;
constexpr int kVarBX[kNumVariants] = {32, 32, 32, 64, kStepBX};
constexpr int kVarBY[kNumVariants] = {4, 8, 16, 4, kStepBY};

// Persistent CTAs walk the work list of (instance, tile) pairs; each tile goes
// through the general tile routine with its instance's parameters and buffers.
// resident threads per SM the batch kernel is built for: the general tile path is
// latency-bound, and FP32 at 2 CTAs of 256 threads per SM (107 registers) ran 20% slower
// than at 3; FP16 keeps 2 (at 80 registers it spills)
template <class S>
constexpr int kBatchThreadsPerSM = kRef<S> ? 512 : 768;
// The instance descriptor of a work item is copied word by word by warp 0 (32-bit words;
// InstDesc is plain data).  The next item's copy is loaded into registers while the
// current tile runs and stored into the other shared buffer after it, so no tile waits
// on a global load for its parameters.
constexpr int kDescWords = (int)(sizeof(InstDesc) / 4);
constexpr int kDescPerLane = (kDescWords + 31) / 32;
static_assert(sizeof(InstDesc) % 4 == 0, "descriptor copied in 32-bit words");

template <int BX, int BY, class S>
__global__ void __launch_bounds__(BX * BY, kBatchThreadsPerSM<S> / (BX * BY) > 0 ? kBatchThreadsPerSM<S> / (BX * BY) : 1)
k_step_batch(const InstDesc* __restrict__ inst, const int2* __restrict__ work, int nwork, int parity)
{
    __shared__ RingSmem<BX, BY> sm;
    __shared__ __align__(16) InstDesc dsc[2];
    const int lane = threadIdx.x;  // warp 0 copies the descriptors
    uint32_t nxt[kDescPerLane];
    auto load = [&](int w) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(inst + work[w].x);
#pragma unroll
        for (int j = 0; j < kDescPerLane; ++j) {
            const int k = lane + 32 * j;
            nxt[j] = k < kDescWords ? __ldg(src + k) : 0u;
        }
    };
    auto store = [&](int b) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(&dsc[b]);
#pragma unroll
        for (int j = 0; j < kDescPerLane; ++j) {
            const int k = lane + 32 * j;
            if (k < kDescWords) dst[k] = nxt[j];
        }
    };
    int w = blockIdx.x, b = 0;
    if (w < nwork && threadIdx.x < 32) {
        load(w);
        store(0);
    }
    __syncthreads();
    for (; w < nwork; w += gridDim.x, b ^= 1) {
        const int2 item = work[w];
        const int wn = w + gridDim.x;
        if (wn < nwork && threadIdx.x < 32) load(wn);  // lands while this tile runs
        const InstDesc& d = dsc[b];
        const typename S::elem* A = (const typename S::elem*)d.pop[parity];
        typename S::elem* B = (typename S::elem*)d.pop[parity ^ 1];
        step_tile_general<BX, BY, S>(d.P, A, B, d.phiu, d.ref[parity], d.ref[parity ^ 1], sm, item.y & 0xffff,
                                     item.y >> 16);
        // step_tile_general ends with a barrier: buffer b ^ 1 is free (its tile ended a
        // barrier ago), and after this one the next descriptor is visible
        if (wn < nwork && threadIdx.x < 32) store(b ^ 1);
        __syncthreads();
    }
}

// ------------------------------------------------ TMA-staged batch kernel
//
// The tiles of every lattice whose rows meet the 16-byte rule and that lie in its TMA
// rectangle (the single-lattice kernel's) are staged by TMA from that lattice's own
// tensor maps, double buffered across lattices, and run through the single-lattice
// kernel's tile body; the lattice's parameters and buffer pointers arrive in the same
// stage by a bulk copy on the same mbarrier.  The remaining tiles follow through the
// general tile path.

// What a tile needs of its lattice besides the staged populations (a 16-byte multiple,
// copied into the stage).
struct __align__(16) BatchTileDesc {
    DevParams P;
    void* pop[2];
    RefT* ref[2];
    float* phiu;
    int* err;
};
struct BatchTmaInst {  // aligned as its tensor maps
    TmaMaps maps[2];      // by parity: the copies of a step at parity p read pop[p]
    BatchTileDesc d;
};
// the bulk copy wants 16-byte aligned addresses and a 16-byte multiple; the tensor maps
// in the device array want 64-byte alignment
static_assert(sizeof(BatchTileDesc) % 16 == 0, "bulk copy size");
static_assert(offsetof(BatchTmaInst, d) % 16 == 0, "bulk copy source alignment");
static_assert(alignof(BatchTmaInst) % 64 == 0 && sizeof(BatchTmaInst) % 64 == 0, "tensor map alignment");

// tile of the TMA-staged batch kernel: the single-lattice step tile, in which each
// lattice's TMA rectangle is laid out
constexpr int kTBX = kStepBX, kTBY = kStepBY;

template <class S>
struct BatchLayout {
    using L = TmaLayout<kTBX, kTBY, S>;
    static constexpr int OFF_D = L::STAGE;
    static constexpr int STAGE = L::STAGE + L::rnd((int)sizeof(BatchTileDesc));
};

__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

template <class S>
__global__ void __launch_bounds__(kTBX * kTBY, kTmaMinBlocks<S>)
k_step_batch_tma(const BatchTmaInst* __restrict__ inst, const int4* __restrict__ titem, int nt,
                 const int2* __restrict__ gitem, int ng, int parity)
{
    constexpr int BX = kTBX, BY = kTBY;
    using L = TmaLayout<BX, BY, S>;
    using BL = BatchLayout<S>;
    using E = typename S::elem;
    static_assert(sizeof(RingSmem<BX, BY>) <= 2 * BL::STAGE, "general-path tiles reuse the stages");
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar[2];
    // issue placement and staging as in k_step_tma
    constexpr bool kLate = kRef<S>;
    __shared__ PhiSmem<BX, BY> smb[kLate ? 2 : 1];
    __shared__ BatchTileDesc gdesc;  // general-path tiles
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int t, int s) {
        // item: lattice, tile (bx | by << 16), seam side, boundary tile
        const int4 item = titem[t];
        const BatchTmaInst& I = inst[item.x];
        const TmaMaps& M = I.maps[parity];
        const int x0 = (item.y & 0xffff) * BX, y0 = (item.y >> 16) * BY;
        unsigned char* st = dsm + s * BL::STAGE;
        // the descriptor's bytes join the tile's on the same mbarrier (expected without an
        // arrival; the tile's copies bring the one arrival)
        fence_proxy_async();
        mbar_expect_tx_only(&bar[s], (uint32_t)sizeof(BatchTileDesc));
        bulk_load(st + BL::OFF_D, &I.d, (uint32_t)sizeof(BatchTileDesc), &bar[s]);
        tma_issue_tile<BX, BY, S>(M, st, &bar[s], x0, y0);
    };

    int it = 0;
    int t = blockIdx.x;
    int4 cur = t < nt ? titem[t] : make_int4(0, 0, 0, 0);
    if (t < nt && tid == 0) issue(t, 0);
    for (; t < nt; t += gridDim.x, ++it) {
        const int s = it & 1;
        const int tn = t + gridDim.x;
        const int4 nxt = tn < nt ? titem[tn] : make_int4(0, 0, 0, 0);
        if constexpr (!kLate) {
            if (tn < nt && tid == 0) issue(tn, s ^ 1);
        }
        PhiSmem<BX, BY>& sm = smb[kLate ? s : 0];
        const bool ok = mbar_wait_bounded(&bar[s], (it >> 1) & 1);
        unsigned char* st = dsm + s * BL::STAGE;
        // the lattice's parameters and buffers, landed with the populations (read before
        // the block's vote only for shared-memory indices the tile body keeps in range)
        const BatchTileDesc& D = *reinterpret_cast<const BatchTileDesc*>(st + BL::OFF_D);
        const DevParams& P = D.P;
        const int x0 = (cur.y & 0xffff) * BX, y0 = (cur.y >> 16) * BY;
        auto on_abort = [&]() {
            if (tid == 0) {
                atomicExch(inst[cur.x].d.err, 1);
                mbar_wait_bounded(&bar[s], (it >> 1) & 1);
                if (!kLate && tn < nt) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1);
            }
        };
        auto after_ring = [&]() {
            if constexpr (kLate) {
                if (tn < nt && tid == 0) issue(tn, s ^ 1);
            }
        };
        // the buffers are read only after the block's vote; which body runs and whether the
        // seam patch does come from the work item, the same on every thread
        const E* A = (const E*)D.pop[parity];
        E* B = (E*)D.pop[parity ^ 1];
        RefT* refB = D.ref[parity ^ 1];
        if (cur.w ? tma_tile<BX, BY, S, true, false>(P, A, B, D.phiu, refB, st, sm, x0, y0, cur.z, ok, on_abort,
                                                     after_ring)
                  : tma_tile<BX, BY, S, false, false>(P, A, B, D.phiu, refB, st, sm, x0, y0, 0, ok, on_abort,
                                                      after_ring))
            return;
        if constexpr (!kLate) __syncthreads();  // stage s and sm are free for the next copies
        cur = nxt;
    }

    // general-path tiles; their ring lives in the stages, which the last TMA tile may
    // still be reading
    if (t - nt < ng) __syncthreads();
    for (int w = t - nt; w < ng; w += gridDim.x) {
        const int2 item = gitem[w];
        if (tid == 0) gdesc = inst[item.x].d;
        __syncthreads();
        const DevParams& P = gdesc.P;
        step_tile_general<BX, BY, S>(P, (const E*)gdesc.pop[parity], (E*)gdesc.pop[parity ^ 1], gdesc.phiu,
                                     gdesc.ref[parity], gdesc.ref[parity ^ 1],
                                     *reinterpret_cast<RingSmem<BX, BY>*>(dsm), item.y & 0xffff, item.y >> 16);
        // step_tile_general ends with a barrier: gdesc is free again
    }
}

template <class S>
void launch_tma(const BatchTmaInst* inst, const int4* titem, int nt, const int2* gitem, int ng, int parity, int grid,
                cudaStream_t s)
{
    k_step_batch_tma<S><<<grid, kTBX * kTBY, 2 * BatchLayout<S>::STAGE, s>>>(inst, titem, nt, gitem, ng, parity);
}

template <class S>
int occupancy_tma()
{
    const int smem = 2 * BatchLayout<S>::STAGE;
    if (cudaFuncSetAttribute(k_step_batch_tma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batch_tma<S>, kTBX * kTBY, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

template <int V, class S>
void launch_variant(const InstDesc* inst, const int2* work, int nwork, int parity, int grid, cudaStream_t s)
{
    constexpr int BX = kVarBX[V], BY = kVarBY[V];
    k_step_batch<BX, BY, S><<<grid, BX * BY, 0, s>>>(inst, work, nwork, parity);
}

template <class S>
void launch(int v, const InstDesc* inst, const int2* work, int nwork, int parity, int grid, cudaStream_t s)
{
    switch (v) {
        case 0: launch_variant<0, S>(inst, work, nwork, parity, grid, s); break;
        case 1: launch_variant<1, S>(inst, work, nwork, parity, grid, s); break;
        case 2: launch_variant<2, S>(inst, work, nwork, parity, grid, s); break;
        case 3: launch_variant<3, S>(inst, work, nwork, parity, grid, s); break;
        default: break;  // kTmaVariant: launch_tma
    }
}

template <int V, class S>
int occupancy_variant()
{
    constexpr int BX = kVarBX[V], BY = kVarBY[V];
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batch<BX, BY, S>, BX * BY, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, per_sm);
}

template <class S>
int occupancy(int v)
{
    switch (v) {
        case 0: return occupancy_variant<0, S>();
        case 1: return occupancy_variant<1, S>();
        case 2: return occupancy_variant<2, S>();
        case 3: return occupancy_variant<3, S>();
        default: return std::max(1, occupancy_tma<S>());
    }
}

}  // namespace

struct tpflbm_batch {
    int n = 0;
    int storage = 0;
    int num_sms = 0;
    std::vector<tpflbm_t> inst;
    InstDesc* d_inst = nullptr;
    BatchTmaInst* d_tinst = nullptr;  // TMA-staged variant: per-lattice maps and descriptors,
    int4* d_titem = nullptr;          // its ntma TMA items (d_work[kTmaVariant] holds the rest)
    int ntma = 0;
    int2* d_work[kNumVariants] = {};
    int nwork[kNumVariants] = {};
    int grid[kNumVariants] = {};
    int variant = 1;
    int parity = 0;
    long long t = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[kNumVariants][2] = {};  // two steps, starting at parity 0 / 1
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(tpflbm_batch_t b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return code;
}

#define TPF_BCUDA(b, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return bfail((b), TPF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void launch_batch(tpflbm_batch_t b, int v, int parity)
{
    if (v == kTmaVariant) {
        const int ng = b->nwork[v] - b->ntma;
        if (b->storage == TPF_STORAGE_FP16)
            launch_tma<StoreF16>(b->d_tinst, b->d_titem, b->ntma, b->d_work[v], ng, parity, b->grid[v], b->stream);
        else
            launch_tma<StoreF32>(b->d_tinst, b->d_titem, b->ntma, b->d_work[v], ng, parity, b->grid[v], b->stream);
        return;
    }
    if (b->storage == TPF_STORAGE_FP16)
        launch<StoreF16>(v, b->d_inst, b->d_work[v], b->nwork[v], parity, b->grid[v], b->stream);
    else
        launch<StoreF32>(v, b->d_inst, b->d_work[v], b->nwork[v], parity, b->grid[v], b->stream);
}

void sync_instances(tpflbm_batch_t b)
{
    for (tpflbm_t h : b->inst) {
        h->cur = b->parity;
        h->t = b->t;
    }
}

void drop_graphs(tpflbm_batch_t b)
{
    for (int v = 0; v < kNumVariants; ++v)
        for (int p = 0; p < 2; ++p)
            if (b->graph[v][p]) {
                cudaGraphExecDestroy(b->graph[v][p]);
                b->graph[v][p] = nullptr;
            }
}

// two steps of variant v starting at parity p, captured once into a graph
int graph_for(tpflbm_batch_t b, int v, int p, cudaGraphExec_t* out)
{
    if (!b->graph[v][p]) {
        cudaGraph_t g = nullptr;
        TPF_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        launch_batch(b, v, p);
        launch_batch(b, v, p ^ 1);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess) return bfail(b, TPF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph[v][p], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, TPF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    *out = b->graph[v][p];
    return TPF_OK;
}

}  // namespace

extern "C" {

int tpflbm_batch_create(int n, const int* nx, const int* ny, const tpflbm_params* params, tpflbm_batch_t* out)
{
    if (!out) return bfail(nullptr, TPF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !nx || !ny || !params) return bfail(nullptr, TPF_ERR_INVALID_ARG, "need n >= 1 lattices with sizes and parameters");
    for (int k = 0; k < n; ++k) {
        if (params[k].storage != params[0].storage)
            return bfail(nullptr, TPF_ERR_INVALID_ARG, "every lattice of a batch has the same storage");
        if (nx[k] >= 65536 || ny[k] >= 65536)
            return bfail(nullptr, TPF_ERR_INVALID_ARG, "batch lattices must have nx, ny < 65536");
    }
    tpflbm_batch_t b = new (std::nothrow) tpflbm_batch;
    if (!b) return bfail(nullptr, TPF_ERR_OOM, "host allocation failed");
    b->n = n;
    b->storage = params[0].storage;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<InstDesc> desc(n);
    for (int k = 0; k < n; ++k) {
        tpflbm_t h = nullptr;
        int rc = tpflbm_create(nx[k], ny[k], &params[k], &h);
        if (rc != TPF_OK) {
            std::string why = std::string("lattice ") + std::to_string(k) + ": " + tpflbm_last_error(nullptr);
            tpflbm_batch_destroy(b);
            return bfail(nullptr, rc, why);
        }
        b->inst.push_back(h);
        desc[k].P = h->dp;
        desc[k].pop[0] = h->pop[0];
        desc[k].pop[1] = h->pop[1];
        desc[k].ref[0] = h->ref[0];
        desc[k].ref[1] = h->ref[1];
        desc[k].phiu = h->phiu;
    }
    cudaError_t e = cudaMalloc(&b->d_inst, n * sizeof(InstDesc));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_inst, desc.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice);
    // the TMA-staged variant: each lattice's own tensor maps (built by its handle when its
    // rows meet the 16-byte rule) and descriptor
    std::vector<BatchTmaInst> tdesc(n);
    for (int k = 0; k < n; ++k) {
        tpflbm_t h = b->inst[k];
        std::memset(&tdesc[k], 0, sizeof(BatchTmaInst));
        if (h->tma) {
            tdesc[k].maps[0] = h->maps[0];
            tdesc[k].maps[1] = h->maps[1];
        }
        tdesc[k].d.P = h->dp;
        tdesc[k].d.pop[0] = h->pop[0];
        tdesc[k].d.pop[1] = h->pop[1];
        tdesc[k].d.ref[0] = h->ref[0];
        tdesc[k].d.ref[1] = h->ref[1];
        tdesc[k].d.phiu = h->phiu;
        tdesc[k].d.err = h->err;
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tinst, n * sizeof(BatchTmaInst));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tinst, tdesc.data(), n * sizeof(BatchTmaInst), cudaMemcpyHostToDevice);
    for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
        std::vector<int2> work;
        const int BX = kVarBX[v], BY = kVarBY[v];
        // tiles of all lattices, lattice by lattice and row by row: the CTAs take
        // consecutive items in the same round, so neighbouring tiles run together (their
        // shared halo rows hit L2) and each lattice's edge tiles spread over the CTAs
        std::vector<int> tx(n), ty(n);
        long long total = 0;
        for (int k = 0; k < n; ++k) {
            tx[k] = (nx[k] + BX - 1) / BX;
            ty[k] = (ny[k] + BY - 1) / BY;
            total += (long long)tx[k] * ty[k];
        }
        work.reserve(total);
        if (v == kTmaVariant) {
            // TMA items first: every lattice's boundary tiles, interleaved over the lattices
            // (at most one per CTA while there are fewer of them than CTAs), then the other
            // TMA tiles lattice by lattice and row by row, as above; then the general-path
            // items
            std::vector<std::vector<int2>> edge(n), tma(n), rest(n);
            for (int k = 0; k < n; ++k) {
                tpflbm_t h = b->inst[k];
                for (int by = 0; by < ty[k]; ++by)
                    for (int bx = 0; bx < tx[k]; ++bx) {
                        const int2 it = make_int2(k, bx | (by << 16));
                        const bool in = h->tma && bx >= h->bx0 && bx < h->bx0 + h->ntbx && by >= h->by0 &&
                                        by < h->by0 + h->ntby;
                        if (!in) {
                            rest[k].push_back(it);
                            continue;
                        }
                        const int x0 = bx * BX, y0 = by * BY;
                        const bool eg = x0 <= 1 || x0 + BX >= nx[k] - 1 || y0 <= 1 || y0 + BY >= ny[k] - 1;
                        (eg ? edge[k] : tma[k]).push_back(it);
                    }
            }
            size_t most = 0;
            for (auto& l : edge) most = std::max(most, l.size());
            for (size_t i = 0; i < most; ++i)
                for (auto& l : edge)
                    if (i < l.size()) work.push_back(l[i]);
            auto concat = [&](std::vector<std::vector<int2>>& lists) {
                for (auto& l : lists) work.insert(work.end(), l.begin(), l.end());
            };
            concat(tma);
            // TMA items also carry the tile's seam side (as seam_side) and whether it
            // touches the lattice boundary (as the single-lattice kernel decides it)
            std::vector<int4> titem(work.size());
            for (size_t i = 0; i < work.size(); ++i) {
                const int k = work[i].x, x0 = (work[i].y & 0xffff) * BX, y0 = (work[i].y >> 16) * BY;
                const int seam = b->inst[k]->hp.bc_x != 0 ? 0 : (x0 == 0 ? -1 : (x0 + BX == nx[k] ? 1 : 0));
                const bool eg = x0 <= 1 || x0 + BX >= nx[k] - 1 || y0 <= 1 || y0 + BY >= ny[k] - 1;
                titem[i] = make_int4(k, work[i].y, seam, eg ? 1 : 0);
            }
            b->ntma = (int)titem.size();
            work.clear();
            concat(rest);
            e = cudaMalloc(&b->d_titem, std::max<size_t>(1, titem.size()) * sizeof(int4));
            if (e == cudaSuccess && !titem.empty())
                e = cudaMemcpy(b->d_titem, titem.data(), titem.size() * sizeof(int4), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
        } else {
            for (int k = 0; k < n; ++k)
                for (int by = 0; by < ty[k]; ++by)
                    for (int bx = 0; bx < tx[k]; ++bx) work.push_back(make_int2(k, bx | (by << 16)));
        }
        b->nwork[v] = (int)work.size() + (v == kTmaVariant ? b->ntma : 0);
        if (b->storage == TPF_STORAGE_FP16) b->grid[v] = occupancy<StoreF16>(v) * b->num_sms;
        else b->grid[v] = occupancy<StoreF32>(v) * b->num_sms;
        b->grid[v] = std::min(b->grid[v], b->nwork[v]);
        e = cudaMalloc(&b->d_work[v], std::max<size_t>(1, work.size()) * sizeof(int2));
        if (e == cudaSuccess && !work.empty())
            e = cudaMemcpy(b->d_work[v], work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        std::string why = std::string("batch set-up: ") + cudaGetErrorString(e);
        tpflbm_batch_destroy(b);
        return bfail(nullptr, TPF_ERR_CUDA, why);
    }
    b->own_stream = true;
    for (tpflbm_t h : b->inst) h->stream = b->stream;
    *out = b;
    return TPF_OK;
}

int tpflbm_batch_set_stream(tpflbm_batch_t b, void* stream)
{
    if (!b || !stream) return bfail(b, TPF_ERR_INVALID_ARG, "a batch needs a non-default stream (graph capture)");
    drop_graphs(b);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->own_stream = false;
    b->stream = (cudaStream_t)stream;
    for (tpflbm_t h : b->inst) h->stream = b->stream;
    return TPF_OK;
}

int tpflbm_batch_size(tpflbm_batch_t b) { return b ? b->n : -1; }

int tpflbm_batch_lattice(tpflbm_batch_t b, int k, tpflbm_t* out)
{
    if (!b || !out || k < 0 || k >= b->n) return bfail(b, TPF_ERR_INVALID_ARG, "no such lattice");
    sync_instances(b);
    *out = b->inst[k];
    return TPF_OK;
}

int tpflbm_batch_init(tpflbm_batch_t b, int k, const float* phi, const float* ux, const float* uy, const float* p,
                      const float* T)
{
    if (!b || k < 0 || k >= b->n) return bfail(b, TPF_ERR_INVALID_ARG, "no such lattice");
    sync_instances(b);
    tpflbm_t h = b->inst[k];
    int rc = tpflbm_init(h, phi, ux, uy, p, T);
    if (rc != TPF_OK) return bfail(b, rc, tpflbm_last_error(h));
    h->t = b->t;
    return TPF_OK;
}

int tpflbm_batch_step(tpflbm_batch_t b, long long nsteps)
{
    if (!b || nsteps < 0) return bfail(b, TPF_ERR_INVALID_ARG, "nsteps must be >= 0");
    const int v = b->variant;
    while (nsteps >= 2) {
        cudaGraphExec_t g = nullptr;
        int rc = graph_for(b, v, b->parity, &g);
        if (rc != TPF_OK) return rc;
        TPF_BCUDA(b, cudaGraphLaunch(g, b->stream));
        nsteps -= 2;
        b->t += 2;
    }
    if (nsteps == 1) {
        launch_batch(b, v, b->parity);
        TPF_BCUDA(b, cudaGetLastError());
        b->parity ^= 1;
        b->t += 1;
    }
    sync_instances(b);
    return TPF_OK;
}

int tpflbm_batch_get_fields(tpflbm_batch_t b, int k, float* phi, float* ux, float* uy, float* p, float* T)
{
    if (!b || k < 0 || k >= b->n) return bfail(b, TPF_ERR_INVALID_ARG, "no such lattice");
    sync_instances(b);
    int rc = tpflbm_get_fields(b->inst[k], phi, ux, uy, p, T);
    return rc == TPF_OK ? rc : bfail(b, rc, tpflbm_last_error(b->inst[k]));
}

int tpflbm_batch_diagnostics(tpflbm_batch_t b, double* out)
{
    if (!b || !out) return bfail(b, TPF_ERR_INVALID_ARG, "out is NULL");
    sync_instances(b);
    int worst = TPF_OK;
    for (int k = 0; k < b->n; ++k) {
        int rc = tpflbm_diagnostics(b->inst[k], out + 8 * k);
        if (rc == TPF_ERR_NONFINITE) worst = rc;
        else if (rc != TPF_OK) return bfail(b, rc, tpflbm_last_error(b->inst[k]));
    }
    if (worst != TPF_OK) return bfail(b, worst, "non-finite values in some lattice");
    return TPF_OK;
}

int tpflbm_batch_residual(tpflbm_batch_t b, const double* dT, double* out)
{
    if (!b || !dT || !out) return bfail(b, TPF_ERR_INVALID_ARG, "dT and out are required");
    sync_instances(b);
    for (int k = 0; k < b->n; ++k) {
        int rc = tpflbm_residual(b->inst[k], dT[k], out + 3 * k);
        if (rc != TPF_OK) return bfail(b, rc, tpflbm_last_error(b->inst[k]));
    }
    return TPF_OK;
}

int tpflbm_batch_variants(int* count, int* bx, int* by)
{
    if (count) *count = kNumVariants;
    for (int v = 0; v < kNumVariants; ++v) {
        if (bx) bx[v] = kVarBX[v];
        if (by) by[v] = kVarBY[v];
    }
    return TPF_OK;
}

int tpflbm_batch_set_variant(tpflbm_batch_t b, int v)
{
    if (!b || v < 0 || v >= kNumVariants) return bfail(b, TPF_ERR_INVALID_ARG, "no such tile shape");
    b->variant = v;
    return TPF_OK;
}

int tpflbm_batch_tune(tpflbm_batch_t b, int steps, double* ms_per_step, int* best)
{
    if (!b || steps < 2) return bfail(b, TPF_ERR_INVALID_ARG, "tuning needs steps >= 2");
    steps &= ~1;
    cudaEvent_t e0, e1;
    TPF_BCUDA(b, cudaEventCreate(&e0));
    TPF_BCUDA(b, cudaEventCreate(&e1));
    int arg = b->variant;
    double bestt = 1e300;
    for (int v = 0; v < kNumVariants; ++v) {
        b->variant = v;
        int rc = tpflbm_batch_step(b, 2);  // capture and warm up
        if (rc != TPF_OK) return rc;
        TPF_BCUDA(b, cudaEventRecord(e0, b->stream));
        rc = tpflbm_batch_step(b, steps);
        if (rc != TPF_OK) return rc;
        TPF_BCUDA(b, cudaEventRecord(e1, b->stream));
        TPF_BCUDA(b, cudaEventSynchronize(e1));
        float ms = 0.f;
        TPF_BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
        const double per = ms / steps;
        if (ms_per_step) ms_per_step[v] = per;
        if (per < bestt) {
            bestt = per;
            arg = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->variant = arg;
    if (best) *best = arg;
    return TPF_OK;
}

long long tpflbm_batch_time(tpflbm_batch_t b) { return b ? b->t : -1; }

void tpflbm_batch_destroy(tpflbm_batch_t b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (tpflbm_t h : b->inst) {
        h->stream = nullptr;
        tpflbm_destroy(h);
    }
    for (int v = 0; v < kNumVariants; ++v) cudaFree(b->d_work[v]);
    cudaFree(b->d_inst);
    cudaFree(b->d_tinst);
    cudaFree(b->d_titem);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* tpflbm_batch_last_error(tpflbm_batch_t b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
