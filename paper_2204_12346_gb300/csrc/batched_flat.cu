// batched_flat.cu -- the flat form of a batch of windows.
//
// Every window's particle pairs are spread over one co-resident grid; the arithmetic and the
// Philox counters of each particle are those of the one-window-per-block form (batched.cu), so
// both forms give the same results.
#include <cmath>

#include "kernels.h"
#include "launch_util.cuh"

namespace sird {

namespace {

// ------------------------------------------------------------------ flat form
// Every window's swarm is spread over the whole grid: thread t owns items t, t + T, t + 2T, ...
// (T threads), an item being a pair of particles of one window (or a last single one), items
// listed window by window, longest windows first.  Per iteration a thread updates and
// integrates its items; lanes of a warp that share a window combine their minimum and their
// item count, one atomicMin and one atomicAdd per window and warp; the lane whose count
// completes the window copies the window's new global-best position to gpos (and, after the
// last iteration, its result to out).  One grid barrier per iteration (all blocks co-resident:
// cooperative launch) keeps the swarm synchronous.  Every particle sees the same Philox counters
// and arithmetic as in the one-window-per-block form, so results are identical.
constexpr unsigned kFlatSpinLimit = 1u << 22;  // polls of >= 32 ns: a few seconds at most

// Bounded grid barrier; returns false (and raises the abort flag) if a wait ran out or another
// block gave up.
__device__ __forceinline__ bool flat_grid_sync(const FlatScratch& fs, unsigned spin_limit, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned gen = __ldcg(fs.bar_gen);
        if (atomicAdd(fs.bar_count, 1u) == gridDim.x - 1) {
            *fs.bar_count = 0u;
            __threadfence();
            atomicAdd(fs.bar_gen, 1u);
        } else {
            ok = 0;
            for (unsigned spin = 0; spin < spin_limit; ++spin) {
                if (__ldcg(fs.bar_gen) != gen) {
                    ok = 1;
                    break;
                }
                if ((spin & 255) == 255 && __ldcg(fs.abort) != 0u) break;
                __nanosleep(32);
            }
            if (!ok) {
                atomicOr(fs.err, kErrTimeout);
                atomicExch(fs.abort, 1u);
            }
        }
        __threadfence();
        *s_ok = ok && __ldcg(fs.abort) == 0u;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <int SPD, int COST>
__global__ void __launch_bounds__(flat_launch_bound(COST)) pso_flat_f32(const BatchWindow* __restrict__ wins,
                                                    const int* __restrict__ n_items_w,
                                                    const int4* __restrict__ items, int n_items, ModelDev m,
                                                    PsoCoeffs<float> c, const float* __restrict__ yf_all,
                                                    const float* __restrict__ invy_all, float* __restrict__ swarm,
                                                    FlatScratch fs, BatchOut* __restrict__ out, int iters,
                                                    unsigned spin_limit) {
    extern __shared__ float smem[];
    __shared__ int s_ok;
    const int B = blockDim.x, B2 = 2 * B, tid = threadIdx.x, P = m.P;
    const int T = gridDim.x * B, t = blockIdx.x * B + tid;
    float* th_s = smem;  // [P][2B]
    float* lb_s = th_s + P * B2;
    float* ub_s = lb_s + kMaxParams;
    if (tid < P) {
        lb_s[tid] = c.zlb[tid];
        ub_s[tid] = c.zub[tid];
    }
    __syncthreads();
    for (int it = 0; it <= iters; ++it) {
        for (int i = t; i < n_items; i += T) {
            const int4 item = items[i];
            const int wi = item.x, j0 = item.y, j1 = item.z;
            const BatchWindow& bw = wins[wi];  // read through the cache as needed, not copied
            const int ld = bw.ld;
            float* X = swarm + bw.sw_off;
            float* V = X + (size_t)P * ld;
            float* PB = V + (size_t)P * ld;
            float* PBF = PB + (size_t)P * ld;
            const float* g = fs.gpos + (size_t)wi * kMaxParams;
            auto update = [&](int j, int col) {
                uint4 rnd = make_uint4(0, 0, 0, 0);
                for (int d = 0; d < P; ++d) {
                    if ((d & 1) == 0)
                        rnd = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)it, (uint32_t)(d >> 1), bw.stream_id),
                                            bw.key0, bw.key1);
                    const float ua = u01f((d & 1) ? rnd.z : rnd.x);
                    const float ub = u01f((d & 1) ? rnd.w : rnd.y);
                    const size_t off = (size_t)d * ld + j;
                    const float lo = lb_s[d], hi = ub_s[d];
                    float xn, vn;
                    if (it == 0) {
                        const float range = __fsub_rn(hi, lo);
                        xn = fminf(__fmaf_rn(range, ua, lo), hi);
                        vn = __fmul_rn(range, __fmaf_rn(2.f, ub, -1.f));
                    } else {
                        const float x = X[off], v = V[off], pbv = PB[off];
                        const float tt = __fmaf_rn(__fmul_rn(c.c1, ua), __fsub_rn(pbv, x), __fmul_rn(c.w, v));
                        vn = __fmaf_rn(__fmul_rn(c.c2, ub), __fsub_rn(__ldcg(g + d), x), tt);
                        xn = fminf(fmaxf(__fadd_rn(x, vn), lo), hi);
                    }
                    X[off] = xn;
                    V[off] = vn;
                    th_s[d * B2 + col] = ((c.logmask >> d) & 1u) ? expf(xn) : xn;
                }
            };
            unsigned long long key = ~0ull;
            auto settle = [&](int j, float f) {
                if (f != f) f = INFINITY;
                float best = f;
                if (it == 0 || f < PBF[j]) {
                    PBF[j] = f;
                    for (int d = 0; d < P; ++d) PB[(size_t)d * ld + j] = X[(size_t)d * ld + j];
                } else {
                    best = PBF[j];
                }
                const unsigned long long kj = argmin_key(best, (uint32_t)j);
                key = kj < key ? kj : key;
            };
            const float* ys = yf_all + bw.obs_off;
            const float* invys = invy_all + bw.obs_off;
            update(j0, tid);
            if (j1 >= 0) {
                update(j1, B + tid);
                float fa, fb;
                fitness_f32x2<SPD, COST>(bw.w, m, ys, invys, th_s + tid, th_s + B + tid, B2, fa, fb);
                settle(j0, fa);
                settle(j1, fb);
            } else {
                settle(j0, fitness_f32<SPD, COST>(bw.w, m, ys, invys, th_s + tid, B2));
            }
            // publish: lanes of this warp working on the same window combine first
            __threadfence();
            const unsigned act = __activemask();
            const unsigned grp = __match_any_sync(act, wi);
            const unsigned long long kmin = masked_min_key(grp, key);
            const int leader = __ffs(grp) - 1;
            if ((tid & 31) == leader) {
                atomicMin(fs.gkey + wi, kmin);
                const unsigned cnt = (unsigned)__popc(grp);
                if (atomicAdd(fs.done + wi, cnt) + cnt == (unsigned)n_items_w[wi]) {
                    // the window's last item of this iteration: its global best is final
                    __threadfence();
                    const unsigned long long gk = atomicExch(fs.gkey + wi, ~0ull);
                    fs.done[wi] = 0u;
                    const int gidx = (int)(gk & 0xFFFFFFFFu);
                    float* gp = fs.gpos + (size_t)wi * kMaxParams;
                    for (int d = 0; d < P; ++d) gp[d] = __ldcg(PB + (size_t)d * ld + gidx);
                    if (it == iters) {
                        out[wi].index = gidx;
                        out[wi].loss = from_ordered_bits((uint32_t)(gk >> 32));
                        for (int d = 0; d < P; ++d) out[wi].z[d] = gp[d];
                    }
                }
            }
        }
        if (it < iters && !flat_grid_sync(fs, spin_limit, &s_ok)) return;
    }
}

// FP64 re-evaluation of every window's global best (one thread per window).
}  // namespace

size_t flat_smem_bytes(const ModelDev& m, int block) {
    return ((size_t)m.P * 2 * block + 2 * kMaxParams) * sizeof(float);
}

int flat_blocks_per_sm(const ModelDev& m, int block) {
    const size_t sm = flat_smem_bytes(m, block);
    int per = 0;
    SIRD_DISPATCH_F32(m, { per = blocks_per_sm_of(pso_flat_f32<S_, C_>, block, sm); });
    (void)cudaGetLastError();
    return per;
}

cudaError_t launch_flat(const BatchWindow* wins, const int* n_items_w, const int4* items, int n_items, int W,
                        const ModelDev& m, const PsoCoeffs<float>& c, const float* yf_all, const float* invy_all,
                        float* swarm, const FlatScratch& fs, BatchOut* out, int iters, int block, int grid,
                        cudaStream_t s) {
    const size_t sm = flat_smem_bytes(m, block);
    (void)cudaGetLastError();
    // neutral reduction words, a fresh barrier, no error
    cudaError_t e = cudaMemsetAsync(fs.gkey, 0xFF, sizeof(unsigned long long) * W, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(fs.done, 0, sizeof(unsigned) * W, s);
    // bar_count, bar_gen, err, abort are four consecutive words
    if (e == cudaSuccess) e = cudaMemsetAsync(fs.bar_count, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    SIRD_DISPATCH_F32(m, {
        auto kern = pso_flat_f32<S_, C_>;
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3((unsigned)block);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, kern, wins, n_items_w, items, n_items, m, c, yf_all, invy_all, swarm, fs,
                                   out, iters, bounded_wait_limit(kFlatSpinLimit));
        }
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sird
