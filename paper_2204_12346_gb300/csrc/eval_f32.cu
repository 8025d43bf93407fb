// eval_f32.cu -- FP32 fitness evaluation of parameter vectors (one window, or a table of windows).
//
// Layout as in the iteration kernels: parameter vectors are structure-of-arrays, entry d of
// vector p at [d*ld + p]; one thread evaluates two vectors in packed f32x2 form, the window's
// observations and the block's parameters staged in shared memory.
#include "kernels.h"
#include "launch_util.cuh"

namespace sird {

namespace {

// A thread evaluates two parameter vectors, p0 = blk * 2B + thread and p1 = p0 + B, together
// in packed f32x2 form (each loss equal to the one-at-a-time evaluation bit for bit).
template <int SPD, int COST>
__device__ __forceinline__ void eval_f32_body(const WindowDev& w, const ModelDev& m, const ObsDev& o,
                                              const float* __restrict__ theta, int ld, int M,
                                              float* __restrict__ loss, int blk) {
    extern __shared__ float smem[];
    float* ys = smem;
    float* invys = stage_obs_f32<COST>(smem, w, m, o);
    float* th_s = after_obs_f32<COST>(smem, w, m);  // [P][2B]
    const int B = blockDim.x, B2 = 2 * B, tid = threadIdx.x;
    const int p0 = blk * B2 + tid, p1 = p0 + B;
    for (int d = 0; d < m.P; ++d) {
        if (p0 < M) th_s[d * B2 + tid] = theta[(size_t)d * ld + p0];
        if (p1 < M) th_s[d * B2 + B + tid] = theta[(size_t)d * ld + p1];
    }
    __syncthreads();
    if (p1 < M) {
        float fa, fb;
        fitness_f32x2<SPD, COST>(w, m, ys, invys, th_s + tid, th_s + B + tid, B2, fa, fb);
        loss[p0] = fa;
        loss[p1] = fb;
    } else if (p0 < M) {
        loss[p0] = fitness_f32<SPD, COST>(w, m, ys, invys, th_s + tid, B2);
    }
}

template <int SPD, int COST>
__global__ void __launch_bounds__(kF32IterMaxBlock, 1) eval_f32_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                         const float* __restrict__ theta, int ld, int M,
                                                         float* __restrict__ loss) {
    eval_f32_body<SPD, COST>(w, m, o, theta, ld, M, loss, blockIdx.x);
}

// Table form: block row blockIdx.y evaluates window blockIdx.y's vectors with its constants.
template <int SPD, int COST>
__global__ void __launch_bounds__(kF32IterMaxBlock, 1) eval_f32_tab_kernel(const PolishWin* __restrict__ tab,
                                                             ModelDev m, const float* __restrict__ theta,
                                                             long long th_ws, int ld, int M,
                                                             float* __restrict__ loss, long long loss_ws) {
    const int i = blockIdx.y;
    const WindowDev w = tab[i].w;
    const ObsDev o = tab[i].o;
    eval_f32_body<SPD, COST>(w, m, o, theta + i * th_ws, ld, M, loss + i * loss_ws, blockIdx.x);
}

}  // namespace

size_t smem_bytes_f32(const WindowDev& w, const ModelDev& m, int block, bool with_theta) {
    size_t n = (size_t)obs_span_pad(w, m) * (m.cost == COST_MAPE ? 2 : 1);
    if (with_theta) n += (size_t)m.P * 2 * block + 3 * kMaxParams;  // theta of two particles per thread
    return n * sizeof(float);
}

cudaError_t launch_eval_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const float* theta, int ld,
                            int M, float* loss, int block, unsigned*, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (block > kF32IterMaxBlock) block = kF32IterMaxBlock;  // results do not depend on the block shape
    const size_t sm = smem_bytes_f32(w, m, block, true);
    cudaError_t e = cudaSuccess;
    SIRD_DISPATCH_F32(m, {
        auto kern = eval_f32_kernel<S_, C_>;
        e = set_smem(kern, sm);
        if (e == cudaSuccess) kern<<<grid_for_pairs(M, block), block, sm, s>>>(w, m, o, theta, ld, M, loss);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_eval_f32_tab(const PolishWin* tab, int nw, int n_max, const ModelDev& m, const float* theta,
                                long long th_ws, int ld, int M, float* loss, long long loss_ws, int block,
                                cudaStream_t s) {
    if (M <= 0 || nw <= 0) return cudaSuccess;
    if (nw > 65535) return cudaErrorInvalidValue;
    if (block > kF32IterMaxBlock) block = kF32IterMaxBlock;
    WindowDev wmax{};
    wmax.n_obs = n_max;
    const size_t sm = smem_bytes_f32(wmax, m, block, true);
    cudaError_t e = cudaSuccess;
    SIRD_DISPATCH_F32(m, {
        auto kern = eval_f32_tab_kernel<S_, C_>;
        e = set_smem(kern, sm);
        if (e == cudaSuccess)
            kern<<<dim3(grid_for_pairs(M, block), (unsigned)nw), block, sm, s>>>(tab, m, theta, th_ws, ld, M, loss,
                                                                              loss_ws);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sird
