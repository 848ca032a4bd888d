// Internal definition of a lattice handle, shared by the library's translation
// units (the single-lattice API and the batched ensemble).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/tpflbm.h"
#include "lattice.cuh"
#include "step.cuh"

#ifndef TPF_TILE_BY
#define TPF_TILE_BY 8
#endif
namespace tpf {
// Tile of the single-lattice step kernels and of the TMA-staged batch kernel, one
// thread per node; a lattice's TMA rectangle is laid out in these tiles (measured on
// the 2048 x 512 channel: 32 x 16 tiles run at 18.8 / 14.8 GLUPS against 21.3 / 16.7
// for 32 x 8, FP32 / FP16).
constexpr int kStepBX = 32, kStepBY = TPF_TILE_BY;
}  // namespace tpf

struct tpflbm {
    int nx = 0, ny = 0;
    tpflbm_params hp{};
    tpf::DevParams dp{};
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool owns = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* pop[2] = {nullptr, nullptr};  // population buffers; pop[cur] holds time t
    tpf::RefT* ref[2] = {nullptr, nullptr}; // FP16 reference records, paired with pop
    int cur = 0;
    float* phiu = nullptr;
    float* stage = nullptr;             // 9 float planes: fields and state I/O
    double* red = nullptr;              // per-block partials and results of the reductions
    int* err = nullptr;                 // device error flag of the step kernels
    float* snap = nullptr;              // u_x, u_y, T at the last residual call
    long long snap_t = -1;              // its time step (-1: none)
    // TMA step kernel
    bool tma = false;
    tpf::TmaMaps maps[2]{};             // maps[c]: reading pop[c]
    int bx0 = 0, by0 = 0, ntbx = 0, ntby = 0, grid_tma = 0;
    int2* tiles = nullptr;              // (x0, y0) of the TMA tiles in the order the kernel walks them
    // CUDA graphs of kGraphSteps steps starting from pop[0] / pop[1] (captured on first use)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // marks the steps enqueued so far for tpflbm_status_async's copy stream (created on first use)
    cudaEvent_t status_ev = nullptr;
    long long t = 0;
    std::string err_msg;
};
