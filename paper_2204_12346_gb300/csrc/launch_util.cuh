// launch_util.cuh -- helpers shared by the FP32 evaluation and iteration kernels: the staging of
// a window's observations in shared memory and the launch-shape helpers.
#pragma once

#include "kernels.h"

namespace sird {

// Copies the observations (all stacked series) into shared memory; returns the reciprocal table
// (or ys).
template <int COST>
__device__ __forceinline__ float* stage_obs_f32(float* smem, const WindowDev& w, const ModelDev& m, const ObsDev& o) {
    float* ys = smem;
    float* invys = (variant_cost(COST) == COST_MAPE) ? ys + obs_span_pad(w, m) : ys;
    const int span = obs_span(w, m);
    for (int i = threadIdx.x; i < span; i += blockDim.x) {
        ys[i] = o.yf[i];
        if (variant_cost(COST) == COST_MAPE) invys[i] = o.invyf[i];
    }
    return invys;
}

template <int COST>
__device__ __forceinline__ float* after_obs_f32(float* smem, const WindowDev& w, const ModelDev& m) {
    return smem + obs_span_pad(w, m) * (variant_cost(COST) == COST_MAPE ? 2 : 1);
}

template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline unsigned grid_for(int M, int block) {
    (void)cudaGetLastError();  // launch errors are read right after each launch; start clean
    return (unsigned)((M + block - 1) / block);
}

// FP32 eval / iteration kernels: two particles per thread
inline unsigned grid_for_pairs(int M, int block) { return grid_for(M, 2 * block); }

// Threads per block the batched kernels are compiled for: 768 (80 registers) for PWC beta and
// F_D, 384 (up to 168) for the ramp and for F_IRD, whose per-step coefficients and three misfits
// need more registers than 80.
__host__ __device__ constexpr int batch_launch_bound(int variant) { return variant_form(variant) == 0 ? 768 : 384; }
// The flat form keeps its items' window constants in registers as well: 512 threads (128
// registers) for PWC beta and F_D, so that it runs without spilling.
__host__ __device__ constexpr int flat_launch_bound(int variant) { return variant_form(variant) == 0 ? 512 : 384; }

// Blocks of `block` threads a kernel can keep per SM; 0 when the block exceeds the kernel's
// compiled limit (its launch bound) or anything else fails.
template <class K>
inline int blocks_per_sm_of(K kern, int block, size_t sm) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || block > fa.maxThreadsPerBlock) return 0;
    if (sm > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int per = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, block, sm) == cudaSuccess ? per : 0;
}

}  // namespace sird
