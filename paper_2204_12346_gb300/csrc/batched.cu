// batched.cu -- many calibration windows in one persistent launch.
//
// The paper calibrates every rolling window I_i = [T_i, T_i + tau] separately (Sec. 3.1).  Here
// W windows of uneven length and swarm size run in one launch: each block takes the next
// window from an atomic queue (windows sorted longest first, so the tail of the run is made of
// short ones), runs that window's whole PSO -- initialisation and every iteration -- and takes
// the next.  A window's swarm never leaves its block, so the synchronous global best is a
// block-level minimum and no block ever waits for another.  Thread t takes particles t,
// t + 2 blockDim, ... and, where they exist, their partners t + blockDim, t + 3 blockDim, ...;
// a pair's trajectories are integrated together in packed f32x2 arithmetic.
//
// Every window uses the same Philox counters, arithmetic and order of updates as a
// single-window calibration, so its result equals that of sird_pso_calibrate with the same
// seed and stream word.
#include <cmath>

#include "kernels.h"
#include "launch_util.cuh"

namespace sird {

namespace {

__host__ __device__ __forceinline__ int pad4(int n) { return (n + 3) & ~3; }

// A last wave of at most this many particles runs one particle per thread.
constexpr int kSingleWaveMax = 384;

template <int SPD, int COST>
__global__ void __launch_bounds__(batch_launch_bound(COST)) pso_batch_f32(const BatchWindow* __restrict__ wins, const int* __restrict__ order,
                                                     int W, ModelDev m, PsoCoeffs<float> c, const float* __restrict__ yf_all,
                                                     const float* __restrict__ invy_all, float* __restrict__ swarm,
                                                     unsigned* __restrict__ queue, BatchOut* __restrict__ out, int iters,
                                                     int n_max) {
    extern __shared__ float smem[];
    __shared__ unsigned long long wk[32];
    __shared__ int s_win;
    const int B = blockDim.x, B2 = 2 * B, tid = threadIdx.x, P = m.P;
    float* ys = smem;
    const int obs_region = pad4(n_max) * (m.ird ? 3 : 1);  // the stacked series of the longest window
    float* invys = (variant_cost(COST) == COST_MAPE) ? ys + obs_region : ys;
    float* th_s = smem + obs_region * (variant_cost(COST) == COST_MAPE ? 2 : 1);  // [P][2B] theta
    float* zs_s = th_s + P * B2;                                                   // [P][2B] z
    float* g_s = zs_s + P * B2;
    float* lb_s = g_s + kMaxParams;
    float* ub_s = lb_s + kMaxParams;
    if (tid < P) {
        lb_s[tid] = c.zlb[tid];
        ub_s[tid] = c.zub[tid];
    }
    for (;;) {
        if (tid == 0) {
            const unsigned q = atomicAdd(queue, 1u);
            s_win = q < (unsigned)W ? order[q] : -1;
        }
        __syncthreads();
        const int wi = s_win;
        if (wi < 0) break;
        const BatchWindow bw = wins[wi];
        const WindowDev& w = bw.w;
        for (int i = tid, span = obs_span(w, m); i < span; i += B) {
            ys[i] = yf_all[bw.obs_off + i];
            if (variant_cost(COST) == COST_MAPE) invys[i] = invy_all[bw.obs_off + i];
        }
        float* X = swarm + bw.sw_off;
        float* V = X + (size_t)P * bw.ld;
        float* PB = V + (size_t)P * bw.ld;
        float* PBF = PB + (size_t)P * bw.ld;
        const int M = bw.M, ld = bw.ld;
        __syncthreads();
        unsigned long long gkey = ~0ull;
        for (int it = 0; it <= iters; ++it) {
            unsigned long long key = ~0ull;
            // The update (initialisation at it == 0) of particle j: the new position goes to
            // column col of th_s decoded (theta, which the fitness reads) and of zs_s as search
            // coordinates (what settle copies into the personal best, with no reload from global
            // memory).  Dimensions go in pairs (one Philox draw), a pair's swarm state loaded
            // before its stores, so a pair of dimensions costs one round trip to L2, not two.
            auto update = [&](int j, int col) {
                for (int d0 = 0; d0 < P; d0 += 2) {
                    const bool second = d0 + 1 < P;
                    float x[2] = {0.f, 0.f}, v[2] = {0.f, 0.f}, pbv[2] = {0.f, 0.f};
                    if (it > 0) {
                        const size_t o = (size_t)d0 * ld + j;
                        x[0] = X[o];
                        v[0] = V[o];
                        pbv[0] = PB[o];
                        if (second) {
                            x[1] = X[o + ld];
                            v[1] = V[o + ld];
                            pbv[1] = PB[o + ld];
                        }
                    }
                    const uint4 rnd = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)it, (uint32_t)(d0 >> 1), bw.stream_id),
                                                    bw.key0, bw.key1);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (q == 1 && !second) break;
                        const int d = d0 + q;
                        const float ua = u01f(q ? rnd.z : rnd.x);
                        const float ub = u01f(q ? rnd.w : rnd.y);
                        const float lo = lb_s[d], hi = ub_s[d];
                        float xn, vn;
                        if (it == 0) {
                            const float range = __fsub_rn(hi, lo);
                            xn = fminf(__fmaf_rn(range, ua, lo), hi);
                            vn = __fmul_rn(range, __fmaf_rn(2.f, ub, -1.f));
                        } else {
                            const float t = __fmaf_rn(__fmul_rn(c.c1, ua), __fsub_rn(pbv[q], x[q]), __fmul_rn(c.w, v[q]));
                            vn = __fmaf_rn(__fmul_rn(c.c2, ub), __fsub_rn(g_s[d], x[q]), t);
                            xn = fminf(fmaxf(__fadd_rn(x[q], vn), lo), hi);
                        }
                        const size_t o = (size_t)d * ld + j;
                        X[o] = xn;
                        V[o] = vn;
                        zs_s[d * B2 + col] = xn;
                        th_s[d * B2 + col] = ((c.logmask >> d) & 1u) ? expf(xn) : xn;
                    }
                }
            };
            // personal best (its position from zs_s column col) and the running block minimum
            auto settle = [&](int j, int col, float f) {
                if (f != f) f = INFINITY;
                float best = f;
                if (it == 0 || f < PBF[j]) {
                    PBF[j] = f;
                    for (int d = 0; d < P; ++d) PB[(size_t)d * ld + j] = zs_s[d * B2 + col];
                } else {
                    best = PBF[j];
                }
                const unsigned long long kj = argmin_key(best, (uint32_t)j);
                key = kj < key ? kj : key;
            };
            // waves of 2B particles, thread t taking particle t of the wave and particle B + t
            // with it -- a pair, integrated together in packed form (one instruction stream for
            // both).  The last wave holds the rest: its Tw threads take particle t and, for
            // t < cnt - Tw, also Tw + t, with Tw = cnt/2 rounded up to whole groups of four warps,
            // so its pairs sit in the lowest warps and every warp scheduler gets the same share;
            // a small rest runs one particle per thread on as many warps as it fills.
            for (int base = 0; base < M; base += B2) {
                const int cnt = M - base < B2 ? M - base : B2;
                int Tw = B;
                if (cnt < B2) {
                    Tw = cnt;
                    if (cnt > kSingleWaveMax && cnt > 1) {
                        Tw = (((cnt + 1) >> 1) + 127) & ~127;
                        if (Tw > B) Tw = B;
                        if (Tw > cnt) Tw = cnt;
                    }
                    if (Tw > B) Tw = B;
                }
                if (tid >= Tw || tid >= cnt) continue;
                const int j0 = base + tid, j1 = base + Tw + tid;
                update(j0, tid);
                float fa, fb;
                if (Tw + tid < cnt) {
                    update(j1, B + tid);
                    fitness_f32x2<SPD, COST, true>(w, m, ys, invys, th_s + tid, th_s + B + tid, B2, fa, fb);
                    settle(j0, tid, fa);
                    settle(j1, B + tid, fb);
                } else {
                    fa = fitness_f32<SPD, COST, true>(w, m, ys, invys, th_s + tid, B2);
                    settle(j0, tid, fa);
                }
            }
            key = warp_min_key(key);
            if ((tid & 31) == 0) wk[tid >> 5] = key;
            __syncthreads();
            gkey = warp_min_key((tid & 31) < (B + 31) / 32 ? wk[tid & 31] : ~0ull);
            if (tid < P) g_s[tid] = PB[(size_t)tid * ld + (int)(gkey & 0xFFFFFFFFu)];
            __syncthreads();
        }
        if (tid == 0) {
            out[wi].index = (int)(gkey & 0xFFFFFFFFu);
            out[wi].loss = from_ordered_bits((uint32_t)(gkey >> 32));
        }
        if (tid < P) out[wi].z[tid] = g_s[tid];
        __syncthreads();  // smem is reused by the next window
    }
}

__global__ void batch_reeval_kernel(const BatchWindow* __restrict__ wins, int W, ModelDev m, uint32_t logmask,
                                    const double* __restrict__ yd_all, BatchOut* __restrict__ out) {
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    if (wi >= W) return;
    const BatchWindow bw = wins[wi];
    double th[kMaxParams];
    for (int d = 0; d < m.P; ++d) {
        const double z = (double)out[wi].z[d];
        th[d] = ((logmask >> d) & 1u) ? exp(z) : z;
        out[wi].theta[d] = th[d];
    }
    double sse = 0.0, f = 0.0;
    const double* ys = yd_all + bw.obs_off;
    switch (m.cost) {
        case COST_MSE: f = fitness_f64<COST_MSE>(bw.w, m, ys, th, 1, &sse); break;
        case COST_MXSE: f = fitness_f64<COST_MXSE>(bw.w, m, ys, th, 1, &sse); break;
        case COST_MAE: f = fitness_f64<COST_MAE>(bw.w, m, ys, th, 1, &sse); break;
        default: f = fitness_f64<COST_MAPE>(bw.w, m, ys, th, 1, &sse); break;
    }
    out[wi].loss64 = f;
    out[wi].sse = sse;
}

}  // namespace

size_t batch_smem_bytes(const ModelDev& m, int block, int n_max) {
    return ((size_t)pad4(n_max) * (m.ird ? 3 : 1) * (m.cost == COST_MAPE ? 2 : 1) + (size_t)m.P * 4 * block +
            3 * kMaxParams) *
           sizeof(float);
}

int batch_blocks_per_sm(const ModelDev& m, int block, int n_max) {
    const size_t sm = batch_smem_bytes(m, block, n_max);
    int per = 0;
    SIRD_DISPATCH_F32(m, { per = blocks_per_sm_of(pso_batch_f32<S_, C_>, block, sm); });
    (void)cudaGetLastError();
    return per;
}

cudaError_t launch_batch(const BatchWindow* wins, const int* order, int W, const ModelDev& m, const PsoCoeffs<float>& c,
                         const float* yf_all, const float* invy_all, const double* yd_all, float* swarm,
                         unsigned* queue, BatchOut* out, int iters, int n_max, int block, int grid, bool reeval,
                         cudaStream_t s) {
    const size_t sm = batch_smem_bytes(m, block, n_max);
    (void)cudaGetLastError();
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    SIRD_DISPATCH_F32(m, {
        auto kern = pso_batch_f32<S_, C_>;
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            kern<<<grid, block, sm, s>>>(wins, order, W, m, c, yf_all, invy_all, swarm, queue, out, iters, n_max);
    });
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && reeval) e = launch_batch_reeval(wins, W, m, c.logmask, yd_all, out, s);
    return e;
}

cudaError_t launch_batch_reeval(const BatchWindow* wins, int W, const ModelDev& m, uint32_t logmask,
                                const double* yd_all, BatchOut* out, cudaStream_t s) {
    (void)cudaGetLastError();
    batch_reeval_kernel<<<(W + 63) / 64, 64, 0, s>>>(wins, W, m, logmask, yd_all, out);
    return cudaGetLastError();
}

}  // namespace sird
