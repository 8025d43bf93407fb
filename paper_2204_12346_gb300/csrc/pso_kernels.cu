// pso_kernels.cu -- fitness evaluation, fused PSO iteration, top-k and FP64 re-evaluation.
//
// Layout: the swarm is structure-of-arrays, entry d of particle p at [d*ld + p], so every
// per-dimension load and store of a warp is one coalesced 128-byte transaction.  One thread
// owns one particle for the whole iteration (Sec. 3.3: particles are independent), staging
// its decoded parameters in shared memory next to the window's observations.
#include <cmath>

#include "kernels.h"
#include "launch_util.cuh"

namespace sird {

namespace {

constexpr int kTopkThreads = 1024;
constexpr int kTopkChunk = 4096;

// ------------------------------------------------------------------ FP32 PSO iteration

template <int SPD, int COST>
__global__ void __launch_bounds__(kF32IterMaxBlock, 1) pso_f32_kernel(WindowDev w, ModelDev m, ObsDev o, PsoCoeffs<float> c,
                                                        SwarmDev<float> sw, ReduceScratch r, int iter) {
    extern __shared__ float smem[];
    __shared__ unsigned long long wk[32];
    __shared__ int last;
    const int B = blockDim.x, B2 = 2 * B, tid = threadIdx.x, P = m.P;
    float* ys = smem;
    float* invys = stage_obs_f32<COST>(smem, w, m, o);
    float* th_s = after_obs_f32<COST>(smem, w, m);  // [P][2B]
    float* g_s = th_s + P * B2;
    float* lb_s = g_s + kMaxParams;
    float* ub_s = lb_s + kMaxParams;
    if (tid < P) {
        g_s[tid] = sw.gbest[tid];  // global best of the previous iteration
        lb_s[tid] = c.zlb[tid];
        ub_s[tid] = c.zub[tid];
    }
    __syncthreads();

    // particles p0 = block * 2B + thread and p1 = p0 + B; a pair is integrated together in
    // packed f32x2 form
    const int p0 = blockIdx.x * B2 + tid, p1 = p0 + B;
    unsigned long long key = ~0ull;
    auto update = [&](int p, int col) {
        uint4 rnd = make_uint4(0, 0, 0, 0);
        for (int d = 0; d < P; ++d) {
            // one Philox call per (particle, iteration, dimension pair); a shard counts its
            // particles from its global offset
            if ((d & 1) == 0)
                rnd = philox4x32_10(make_uint4((uint32_t)p + c.p_off, (uint32_t)iter, (uint32_t)(d >> 1), c.stream_id),
                                    c.key0, c.key1);
            const float ua = u01f((d & 1) ? rnd.z : rnd.x);
            const float ub = u01f((d & 1) ? rnd.w : rnd.y);
            const size_t off = (size_t)d * sw.ld + p;
            const float lo = lb_s[d], hi = ub_s[d];
            float xn, vn;
            if (iter == 0) {
                const float range = __fsub_rn(hi, lo);
                xn = fminf(__fmaf_rn(range, ua, lo), hi);
                vn = __fmul_rn(range, __fmaf_rn(2.f, ub, -1.f));
            } else {
                // v <- w v + c1 r1 (pbest - x) + c2 r2 (gbest - x);  x <- x + v, set to the bound
                // when outside the box (Sec. 3.3); the velocity is kept.
                const float x = sw.x[off], v = sw.v[off], pbv = sw.pb[off];
                const float t = __fmaf_rn(__fmul_rn(c.c1, ua), __fsub_rn(pbv, x), __fmul_rn(c.w, v));
                vn = __fmaf_rn(__fmul_rn(c.c2, ub), __fsub_rn(g_s[d], x), t);
                xn = fminf(fmaxf(__fadd_rn(x, vn), lo), hi);
            }
            sw.x[off] = xn;
            sw.v[off] = vn;
            th_s[d * B2 + col] = ((c.logmask >> d) & 1u) ? expf(xn) : xn;
        }
    };
    auto settle = [&](int p, float f) {
        if (f != f) f = INFINITY;
        float best = f;
        const bool improve = (iter == 0) || (f < sw.pbf[p]);
        if (improve) {
            sw.pbf[p] = f;
            for (int d = 0; d < P; ++d) sw.pb[(size_t)d * sw.ld + p] = sw.x[(size_t)d * sw.ld + p];
        } else {
            best = sw.pbf[p];
        }
        const unsigned long long kp = argmin_key(best, (uint32_t)p + c.p_off);
        key = kp < key ? kp : key;
    };
    if (p0 < sw.M) {
        update(p0, tid);
        if (p1 < sw.M) {
            update(p1, B + tid);
            float fa, fb;
            fitness_f32x2<SPD, COST>(w, m, ys, invys, th_s + tid, th_s + B + tid, B2, fa, fb);
            settle(p0, fa);
            settle(p1, fb);
        } else {
            settle(p0, fitness_f32<SPD, COST>(w, m, ys, invys, th_s + tid, B2));
        }
    }

    // block minimum -> one atomicMin per block -> the last block publishes the global best
    key = warp_min_key(key);
    if ((tid & 31) == 0) wk[tid >> 5] = key;
    __syncthreads();
    if (tid < 32) {
        const unsigned long long k2 = warp_min_key((tid < (B + 31) / 32) ? wk[tid] : ~0ull);
        if (tid == 0) {
            atomicMin(r.gkey, k2);
            __threadfence();
            last = (atomicAdd(r.counter, 1u) == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (tid == 0) {
            const unsigned long long g = atomicExch(r.gkey, ~0ull);
            *r.counter = 0u;
            *r.gbest_idx = (int)(g & 0xFFFFFFFFu);
            *(float*)r.gbest_f = from_ordered_bits((uint32_t)(g >> 32));
            wk[0] = g;
        }
        __syncthreads();
        const int gi = (int)((uint32_t)(wk[0] & 0xFFFFFFFFu) - c.p_off);  // local index of the best
        if (tid < P) sw.gbest[tid] = __ldcg(&sw.pb[(size_t)tid * sw.ld + gi]);
    }
}

// ------------------------------------------------------------------ FP64 eval / PSO

template <int COST>
__global__ void __launch_bounds__(256) eval_f64_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                        const double* __restrict__ theta, int ld, int M,
                                                        double* __restrict__ loss) {
    extern __shared__ double dsm[];
    double* ys = dsm;
    double* th_s = dsm + obs_span(w, m);
    const int B = blockDim.x, tid = threadIdx.x;
    for (int i = tid, span = obs_span(w, m); i < span; i += B) ys[i] = o.yd[i];
    const int p = blockIdx.x * B + tid;
    if (p < M)
        for (int d = 0; d < m.P; ++d) th_s[d * B + tid] = theta[(size_t)d * ld + p];
    __syncthreads();
    if (p < M) loss[p] = fitness_f64<COST>(w, m, ys, th_s + tid, B, nullptr);
}

template <int COST>
__global__ void __launch_bounds__(256) pso_f64_kernel(WindowDev w, ModelDev m, ObsDev o, PsoCoeffs<double> c,
                                                       SwarmDev<double> sw, ReduceScratch r, int iter) {
    extern __shared__ double dsm[];
    __shared__ double wf[32];
    __shared__ int wi[32];
    __shared__ int last;
    const int B = blockDim.x, tid = threadIdx.x, P = m.P;
    double* ys = dsm;
    double* th_s = dsm + obs_span(w, m);
    double* g_s = th_s + P * B;
    for (int i = tid, span = obs_span(w, m); i < span; i += B) ys[i] = o.yd[i];
    if (tid < P) g_s[tid] = sw.gbest[tid];
    __syncthreads();

    const int p = blockIdx.x * B + tid;
    double best = INFINITY;
    int bidx = INT_MAX;
    if (p < sw.M) {
        uint4 rnd = make_uint4(0, 0, 0, 0);
        for (int d = 0; d < P; ++d) {
            if ((d & 1) == 0) rnd = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)iter, (uint32_t)(d >> 1), c.stream_id),
                                                 c.key0, c.key1);
            const double ua = u01d((d & 1) ? rnd.z : rnd.x);
            const double ub = u01d((d & 1) ? rnd.w : rnd.y);
            const size_t off = (size_t)d * sw.ld + p;
            const double lo = c.zlb[d], hi = c.zub[d];
            double xn, vn;
            if (iter == 0) {
                const double range = __dsub_rn(hi, lo);
                xn = __dadd_rn(lo, __dmul_rn(range, ua));
                if (xn > hi) xn = hi;
                vn = __dmul_rn(range, __dsub_rn(__dmul_rn(2.0, ub), 1.0));
            } else {
                // same update as FP32, in the order (w v) + (c1 r1)(pbest - x) + (c2 r2)(gbest - x)
                const double x = sw.x[off], v = sw.v[off], pbv = sw.pb[off];
                vn = __dadd_rn(__dadd_rn(__dmul_rn(c.w, v), __dmul_rn(__dmul_rn(c.c1, ua), __dsub_rn(pbv, x))),
                               __dmul_rn(__dmul_rn(c.c2, ub), __dsub_rn(g_s[d], x)));
                xn = __dadd_rn(x, vn);
                if (xn < lo) xn = lo;
                if (xn > hi) xn = hi;
            }
            sw.x[off] = xn;
            sw.v[off] = vn;
            th_s[d * B + tid] = ((c.logmask >> d) & 1u) ? exp(xn) : xn;
        }
        double f = fitness_f64<COST>(w, m, ys, th_s + tid, B, nullptr);
        if (f != f) f = INFINITY;
        best = f;
        if (iter == 0 || f < sw.pbf[p]) {
            sw.pbf[p] = f;
            for (int d = 0; d < P; ++d) sw.pb[(size_t)d * sw.ld + p] = sw.x[(size_t)d * sw.ld + p];
        } else {
            best = sw.pbf[p];
        }
        bidx = p;
    }
    warp_min_pair(best, bidx);
    if ((tid & 31) == 0) {
        wf[tid >> 5] = best;
        wi[tid >> 5] = bidx;
    }
    __syncthreads();
    if (tid < 32) {
        double f2 = (tid < (B + 31) / 32) ? wf[tid] : INFINITY;
        int i2 = (tid < (B + 31) / 32) ? wi[tid] : INT_MAX;
        warp_min_pair(f2, i2);
        if (tid == 0) {
            r.partial[blockIdx.x].f = f2;
            r.partial[blockIdx.x].idx = i2;
            __threadfence();
            last = (atomicAdd(r.counter, 1u) == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double f2 = INFINITY;
        int i2 = INT_MAX;
        for (int b = tid; b < (int)gridDim.x; b += B) {
            const double fb = __ldcg(&r.partial[b].f);
            const int ib = __ldcg(&r.partial[b].idx);
            if (pair_less(fb, ib, f2, i2)) {
                f2 = fb;
                i2 = ib;
            }
        }
        warp_min_pair(f2, i2);
        if ((tid & 31) == 0) {
            wf[tid >> 5] = f2;
            wi[tid >> 5] = i2;
        }
        __syncthreads();
        if (tid < 32) {
            double f3 = (tid < (B + 31) / 32) ? wf[tid] : INFINITY;
            int i3 = (tid < (B + 31) / 32) ? wi[tid] : INT_MAX;
            warp_min_pair(f3, i3);
            if (tid == 0) {
                *r.counter = 0u;
                *r.gbest_idx = i3;
                *(double*)r.gbest_f = f3;
                wi[0] = i3;
            }
        }
        __syncthreads();
        const int gi = wi[0];
        if (tid < P) sw.gbest[tid] = __ldcg(&sw.pb[(size_t)tid * sw.ld + gi]);
    }
}

// ------------------------------------------------------------------ top-k

// Sorts the kTopkChunk keys of s ascending (bitonic network); ends with a block barrier.
__device__ __forceinline__ void bitonic_sort_chunk(unsigned long long* s, int tid) {
    for (int size = 2; size <= kTopkChunk; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < kTopkChunk / 2; i += kTopkThreads) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long a = s[lo], b = s[hi];
                if ((a > b) == asc) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Sorts a chunk of kTopkChunk keys ascending in shared memory and writes the first k.  Keys come
// from the personal-best values (pbf != nullptr) or from a previous pass.
__global__ void __launch_bounds__(kTopkThreads) topk_kernel(const float* __restrict__ pbf,
                                                             const unsigned long long* __restrict__ in, int n, int k,
                                                             unsigned long long* __restrict__ out) {
    __shared__ unsigned long long s[kTopkChunk];
    const int tid = threadIdx.x;
    const long long base = (long long)blockIdx.x * kTopkChunk;
    for (int i = tid; i < kTopkChunk; i += kTopkThreads) {
        const long long j = base + i;
        unsigned long long v = ~0ull;
        if (j < n) v = pbf ? argmin_key(pbf[j], (uint32_t)j) : in[j];
        s[i] = v;
    }
    __syncthreads();
    bitonic_sort_chunk(s, tid);
    for (int i = tid; i < k; i += kTopkThreads) out[(size_t)blockIdx.x * k + i] = s[i];
}

// Table form, one block per window: s[0, k) holds the window's k smallest keys so far and is
// sorted together with the next kTopkChunk - k keys of its personal bests, chunk by chunk.  The k
// smallest keys are unique (the index breaks ties), so they equal the chunked passes' result.
__global__ void __launch_bounds__(kTopkThreads) topk_tab_kernel(const PolishWin* __restrict__ tab, int k,
                                                                 unsigned long long* __restrict__ keys) {
    __shared__ unsigned long long s[kTopkChunk];
    const int tid = threadIdx.x, per = kTopkChunk - k;
    const float* pbf = tab[blockIdx.x].pbf;
    const int M = tab[blockIdx.x].M;
    for (int i = tid; i < k; i += kTopkThreads) s[i] = ~0ull;
    for (int base = 0; base < M; base += per) {
        for (int i = tid; i < per; i += kTopkThreads) {
            const int j = base + i;
            s[k + i] = j < M ? argmin_key(pbf[j], (uint32_t)j) : ~0ull;
        }
        __syncthreads();
        bitonic_sort_chunk(s, tid);
    }
    for (int i = tid; i < k; i += kTopkThreads) keys[(size_t)blockIdx.x * k + i] = s[i];
}

// ------------------------------------------------------------------ FP64 re-evaluation

__global__ void __launch_bounds__(1024) reeval_kernel(WindowDev w, ModelDev m, ObsDev o, uint32_t logmask, int is64,
                                                       const void* pb, const void* pbf, int ld,
                                                       const unsigned long long* keys, int k, const int* gbest_idx,
                                                       ResultDev* res) {
    extern __shared__ double dsm[];
    __shared__ double wf[32];
    __shared__ int wi[32];
    double* ys = dsm;
    double* th_s = dsm + obs_span(w, m);
    const int B = blockDim.x, tid = threadIdx.x, P = m.P;
    for (int i = tid, span = obs_span(w, m); i < span; i += B) ys[i] = o.yd[i];
    int idx = INT_MAX;
    if (tid < k) {
        idx = keys ? (int)(keys[tid] & 0xFFFFFFFFu) : *gbest_idx;
        for (int d = 0; d < P; ++d) {
            const size_t off = (size_t)d * ld + idx;
            const double z = is64 ? ((const double*)pb)[off] : (double)((const float*)pb)[off];
            th_s[d * B + tid] = ((logmask >> d) & 1u) ? exp(z) : z;
        }
    }
    __syncthreads();
    double f = INFINITY, sse = 0.0;
    if (tid < k) {
        switch (m.cost) {
            case COST_MSE: f = fitness_f64<COST_MSE>(w, m, ys, th_s + tid, B, &sse); break;
            case COST_MXSE: f = fitness_f64<COST_MXSE>(w, m, ys, th_s + tid, B, &sse); break;
            case COST_MAE: f = fitness_f64<COST_MAE>(w, m, ys, th_s + tid, B, &sse); break;
            default: f = fitness_f64<COST_MAPE>(w, m, ys, th_s + tid, B, &sse); break;
        }
    }
    double bf = f;
    int bi = idx;
    warp_min_pair(bf, bi);
    if ((tid & 31) == 0) {
        wf[tid >> 5] = bf;
        wi[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid < 32) {
        double f2 = (tid < (B + 31) / 32) ? wf[tid] : INFINITY;
        int i2 = (tid < (B + 31) / 32) ? wi[tid] : INT_MAX;
        warp_min_pair(f2, i2);
        if (tid == 0) wi[0] = i2;
    }
    __syncthreads();
    if (tid < k && idx == wi[0]) {
        for (int d = 0; d < P; ++d) res->theta[d] = th_s[d * B + tid];
        res->loss = f;
        res->sse = sse;
        res->index = idx;
        res->count = k;
        res->loss_search = is64 ? ((const double*)pbf)[idx] : (double)((const float*)pbf)[idx];
    }
}

__global__ void topk_gather_kernel(const unsigned long long* __restrict__ keys, int k, const float* __restrict__ pb,
                                   const float* __restrict__ pbf, int ld, int P, uint32_t logmask,
                                   double* __restrict__ theta_out, double* __restrict__ loss_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const int idx = (int)(keys[j] & 0xFFFFFFFFu);
    for (int d = 0; d < P; ++d) {
        const double z = (double)pb[(size_t)d * ld + idx];
        theta_out[(size_t)j * P + d] = ((logmask >> d) & 1u) ? exp(z) : z;
    }
    loss_out[j] = (double)pbf[idx];
}

}  // namespace

static size_t smem_bytes_f64(const WindowDev& w, const ModelDev& m, int block, bool with_g) {
    return ((size_t)obs_span(w, m) + (size_t)m.P * block + (with_g ? kMaxParams : 0)) * sizeof(double);
}

#define SIRD_DISPATCH_COST(COSTV, ...)                          \
    switch (COSTV) {                                            \
        case COST_MSE: { constexpr int C_ = COST_MSE; __VA_ARGS__; } break;   \
        case COST_MXSE: { constexpr int C_ = COST_MXSE; __VA_ARGS__; } break; \
        case COST_MAE: { constexpr int C_ = COST_MAE; __VA_ARGS__; } break;   \
        default: { constexpr int C_ = COST_MAPE; __VA_ARGS__; } break;        \
    }

cudaError_t launch_eval_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const double* theta, int ld,
                            int M, double* loss, int block, unsigned*, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    const size_t sm = smem_bytes_f64(w, m, block, false);
    cudaError_t e = cudaSuccess;
    SIRD_DISPATCH_COST(m.cost, {
        auto kern = eval_f64_kernel<C_>;
        e = set_smem(kern, sm);
        if (e == cudaSuccess) kern<<<grid_for(M, block), block, sm, s>>>(w, m, o, theta, ld, M, loss);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_pso_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<float>& c,
                           const SwarmDev<float>& sw, const ReduceScratch& r, int iter, int block, cudaStream_t s) {
    if (block > kF32IterMaxBlock) block = kF32IterMaxBlock;  // results do not depend on the block shape
    const size_t sm = smem_bytes_f32(w, m, block, true);
    cudaError_t e = cudaSuccess;
    SIRD_DISPATCH_F32(m, {
        auto kern = pso_f32_kernel<S_, C_>;
        e = set_smem(kern, sm);
        if (e == cudaSuccess) kern<<<grid_for_pairs(sw.M, block), block, sm, s>>>(w, m, o, c, sw, r, iter);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_pso_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<double>& c,
                           const SwarmDev<double>& sw, const ReduceScratch& r, int iter, int block, cudaStream_t s) {
    const size_t sm = smem_bytes_f64(w, m, block, true);
    cudaError_t e = cudaSuccess;
    SIRD_DISPATCH_COST(m.cost, {
        auto kern = pso_f64_kernel<C_>;
        e = set_smem(kern, sm);
        if (e == cudaSuccess) kern<<<grid_for(sw.M, block), block, sm, s>>>(w, m, o, c, sw, r, iter);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

size_t topk_scratch_keys(int M, int k) {
    const size_t blocks = ((size_t)M + kTopkChunk - 1) / kTopkChunk;
    return blocks * (size_t)k + kTopkChunk;
}

cudaError_t launch_topk_f32(const float* pbf, int M, int k, unsigned long long* tmp_a, unsigned long long* tmp_b,
                            unsigned long long** out, cudaStream_t s) {
    if (k < 1 || k > kTopkChunk / 2) return cudaErrorInvalidValue;
    int n = M;
    const float* src_f = pbf;
    const unsigned long long* src = nullptr;
    unsigned long long* dst = tmp_a;
    (void)cudaGetLastError();
    for (;;) {
        const unsigned blocks = (unsigned)((n + kTopkChunk - 1) / kTopkChunk);
        topk_kernel<<<blocks, kTopkThreads, 0, s>>>(src_f, src, n, k, dst);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (blocks == 1) {
            *out = dst;
            return cudaSuccess;
        }
        n = (int)(blocks * (unsigned)k);
        src_f = nullptr;
        src = dst;
        dst = (dst == tmp_a) ? tmp_b : tmp_a;
    }
}

cudaError_t launch_topk_tab(const PolishWin* tab, int nw, int k, unsigned long long* keys, cudaStream_t s) {
    if (nw <= 0) return cudaSuccess;
    if (k < 1 || k > kTopkTabMax) return cudaErrorInvalidValue;
    (void)cudaGetLastError();
    topk_tab_kernel<<<(unsigned)nw, kTopkThreads, 0, s>>>(tab, k, keys);
    return cudaGetLastError();
}

cudaError_t launch_topk_gather(const unsigned long long* keys, int k, const float* pb, const float* pbf, int ld,
                               int P, uint32_t logmask, double* theta_out, double* loss_out, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    (void)cudaGetLastError();
    topk_gather_kernel<<<(k + 127) / 128, 128, 0, s>>>(keys, k, pb, pbf, ld, P, logmask, theta_out, loss_out);
    return cudaGetLastError();
}

cudaError_t launch_reeval(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<float>* c32,
                          const PsoCoeffs<double>* c64, const void* pb, const void* pbf, int ld,
                          const unsigned long long* keys, int k, const int* gbest_idx, ResultDev* res,
                          cudaStream_t s) {
    const int block = ((k + 31) / 32) * 32;
    if (block < 32 || block > 1024) return cudaErrorInvalidValue;
    const size_t sm = smem_bytes_f64(w, m, block, false);
    cudaError_t e = set_smem(reeval_kernel, sm);
    if (e != cudaSuccess) return e;
    const uint32_t logmask = c64 ? c64->logmask : c32->logmask;
    (void)cudaGetLastError();
    reeval_kernel<<<1, block, sm, s>>>(w, m, o, logmask, c64 ? 1 : 0, pb, pbf, ld, keys, k, gbest_idx, res);
    return cudaGetLastError();
}

}  // namespace sird
