// pso_persistent.cu -- all PSO iterations of an FP32 swarm in one cooperative launch.
//
// For swarms whose blocks all fit on the GPU at once (e.g. 4096 particles = 32 blocks of
// 128), launching one kernel per iteration costs more than the iteration itself.  Here every
// block keeps its particles' position, velocity and personal best in shared memory for the
// whole run.  After each iteration a block publishes its best personal best (loss, index and
// position) in a global slot whose every 64-bit word carries the iteration number in its high
// half; a word is written and read whole, so a reader knows it is current without fences.
// Every block waits (bounded) until all words of all slots carry the current iteration, then
// takes the minimum -- the same global best in every block, as the synchronous PSO of
// Sec. 3.3 requires.  Slots are double-buffered by iteration parity, so a block that runs
// ahead never overwrites data a slower block is still reading.  The next iteration's Philox
// words are drawn while the exchange is in flight.
//
// The launch is cooperative (all blocks co-resident).  Every wait has an iteration cap: a
// block that gives up sets kErrTimeout and an abort flag that releases the others, and the
// kernel returns with the swarm written back.
#include <cmath>

#include <cooperative_groups.h>

#include "kernels.h"

namespace sird {

namespace {

constexpr unsigned kSpinLimit = 1u << 21;  // polls of about 1 us: about two seconds

__host__ __device__ __forceinline__ int pad4(int n) { return (n + 3) & ~3; }

// Philox words of one iteration for this thread's particle: pair j of dimensions at rnd[j*B].
__device__ __forceinline__ void draw_iteration(uint4* rnd, int npairs, int B, uint32_t p, uint32_t it,
                                               const PsoCoeffs<float>& c) {
#pragma unroll 4
    for (int j = 0; j < npairs; ++j) rnd[j * B] = philox4x32_10(make_uint4(p, it, (uint32_t)j, c.stream_id), c.key0, c.key1);
}

__device__ __forceinline__ unsigned long long tagged(unsigned tag, uint32_t v) {
    return ((unsigned long long)tag << 32) | v;
}

// CLUSTER: the grid is one thread-block cluster (at most 16 blocks) and the blocks exchange their
// best through distributed shared memory -- each block's (key, position) in its own shared
// memory, double-buffered by iteration parity, read by every block after one cluster barrier --
// instead of the global slots; no wait is spun (the hardware barrier needs every block to
// arrive, and every block runs the same iterations).
template <int SPD, int COST, bool CLUSTER>
__global__ void __launch_bounds__(1024) pso_f32_persistent(WindowDev w, ModelDev m, ObsDev o, PsoCoeffs<float> c,
                                                            SwarmDev<float> sw, ReduceScratch r,
                                                            ExchangeSlot* __restrict__ slots, int iter0, int n_iters,
                                                            unsigned spin_limit) {
    extern __shared__ float smem[];
    __shared__ unsigned long long wk[32];
    __shared__ int s_flag;
    __shared__ unsigned long long s_gkey;
    __shared__ unsigned long long ex_key[2];    // CLUSTER: this block's best of the iteration
    __shared__ float ex_pos[2][kMaxParams];     // and its position
    const int B = blockDim.x, tid = threadIdx.x, P = m.P, G = gridDim.x;
    const int npairs = (P + 1) >> 1;
    float* ys = smem;
    float* invys = (variant_cost(COST) == COST_MAPE) ? ys + obs_span_pad(w, m) : ys;
    float* th_s = smem + obs_span_pad(w, m) * (variant_cost(COST) == COST_MAPE ? 2 : 1);
    float* xs = th_s + P * B;
    float* vs = xs + P * B;
    float* pbs = vs + P * B;
    float* pbfs = pbs + P * B;
    float* g_s = pbfs + B;
    float* lb_s = g_s + kMaxParams;
    float* ub_s = lb_s + kMaxParams;
    float* slot_pos = ub_s + kMaxParams;                          // [G][P] positions read from the slots
    uint4* rnd = (uint4*)(slot_pos + pad4(G * P));                 // [npairs][B] Philox words

    for (int i = tid, span = obs_span(w, m); i < span; i += B) {
        ys[i] = o.yf[i];
        if (variant_cost(COST) == COST_MAPE) invys[i] = o.invyf[i];
    }
    const int base = blockIdx.x * B;
    for (int i = tid; i < P * B; i += B) {
        const int d = i / B, j = i - d * B, q = base + j;
        if (q < sw.M) {
            const size_t off = (size_t)d * sw.ld + q;
            xs[i] = sw.x[off];
            vs[i] = sw.v[off];
            pbs[i] = sw.pb[off];
        }
    }
    const int p = base + tid;
    const bool active = p < sw.M;
    pbfs[tid] = active ? sw.pbf[p] : INFINITY;
    if (tid < P) {
        g_s[tid] = sw.gbest[tid];
        lb_s[tid] = c.zlb[tid];
        ub_s[tid] = c.zub[tid];
    }
    if (active && n_iters > 0) draw_iteration(rnd + tid, npairs, B, (uint32_t)p, (uint32_t)(iter0 + 1), c);
    __syncthreads();

    bool aborted = false;
    unsigned long long gkey = ~0ull;
    for (int it = iter0 + 1; it <= iter0 + n_iters && !aborted; ++it) {
        unsigned long long key = ~0ull;
        if (active) {
            // velocity and position of every dimension (independent: unrolled for ILP), then decode
#pragma unroll 4
            for (int d = 0; d < P; ++d) {
                const uint4 rr = rnd[(d >> 1) * B + tid];
                const float ua = u01f((d & 1) ? rr.z : rr.x);
                const float ub = u01f((d & 1) ? rr.w : rr.y);
                const int i = d * B + tid;
                const float x = xs[i], v = vs[i], pbv = pbs[i];
                const float t = __fmaf_rn(__fmul_rn(c.c1, ua), __fsub_rn(pbv, x), __fmul_rn(c.w, v));
                const float vn = __fmaf_rn(__fmul_rn(c.c2, ub), __fsub_rn(g_s[d], x), t);
                xs[i] = fminf(fmaxf(__fadd_rn(x, vn), lb_s[d]), ub_s[d]);
                vs[i] = vn;
            }
#pragma unroll 4
            for (int d = 0; d < P; ++d) {
                const int i = d * B + tid;
                th_s[i] = ((c.logmask >> d) & 1u) ? expf(xs[i]) : xs[i];
            }
            float f = fitness_f32<SPD, COST>(w, m, ys, invys, th_s + tid, B);
            if (f != f) f = INFINITY;
            if (f < pbfs[tid]) {
                pbfs[tid] = f;
                for (int d = 0; d < P; ++d) pbs[d * B + tid] = xs[d * B + tid];
            }
            key = argmin_key(pbfs[tid], (uint32_t)p);
        }
        key = warp_min_key(key);
        if ((tid & 31) == 0) wk[tid >> 5] = key;
        __syncthreads();
        const unsigned tag = (unsigned)it;
        ExchangeSlot* row = slots + (size_t)(it & 1) * G;
        if (CLUSTER) {
            const int par = it & 1;
            if (tid < 32) {
                const unsigned long long bkey = warp_min_key((tid < (B + 31) / 32) ? wk[tid] : ~0ull);
                const int j = (int)(bkey & 0xFFFFFFFFu) - base;  // the block's best is one of its own particles
                if (tid < P) ex_pos[par][tid] = pbs[tid * B + j];
                if (tid == 0) ex_key[par] = bkey;
                if (B == 32 && it < iter0 + n_iters && active)  // a one-warp block draws its own
                    draw_iteration(rnd + tid, npairs, B, (uint32_t)p, (uint32_t)(it + 1), c);
            } else if (it < iter0 + n_iters) {  // the next iteration's random numbers meanwhile
                for (int i = tid - 32; i < npairs * B; i += B - 32) {
                    const int j = i / B, q = i - j * B;
                    if (base + q < sw.M)
                        rnd[i] = philox4x32_10(make_uint4((uint32_t)(base + q), (uint32_t)(it + 1), (uint32_t)j,
                                                          c.stream_id), c.key0, c.key1);
                }
            }
            cooperative_groups::this_cluster().sync();
            if (tid < 32) {
                auto cl = cooperative_groups::this_cluster();
                unsigned long long best = ~0ull;
                int bblk = 0;
                if (tid < G) {
                    best = *cl.map_shared_rank(&ex_key[par], (unsigned)tid);
                    bblk = tid;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long k2 = __shfl_xor_sync(0xFFFFFFFFu, best, off);
                    const int b2 = __shfl_xor_sync(0xFFFFFFFFu, bblk, off);
                    if (k2 < best) {
                        best = k2;
                        bblk = b2;
                    }
                }
                if (tid < P) g_s[tid] = *cl.map_shared_rank(&ex_pos[par][tid], (unsigned)bblk);
                if (tid == 0) s_gkey = best;
            }
            __syncthreads();
            gkey = s_gkey;
            continue;
        }
        if (tid < 32) {
            // block minimum, then publish it: every word carries the iteration number
            const unsigned long long bkey = warp_min_key((tid < (B + 31) / 32) ? wk[tid] : ~0ull);
            ExchangeSlot* mine = row + blockIdx.x;
            if (tid < P) {
                const int j = (int)(bkey & 0xFFFFFFFFu) - base;  // the block's best is one of its own particles
                __stcg(&mine->w_pos[tid], tagged(tag, __float_as_uint(pbs[tid * B + j])));
            }
            if (tid == 0) {
                __stcg(&mine->w_loss, tagged(tag, (uint32_t)(bkey >> 32)));
                __stcg(&mine->w_idx, tagged(tag, (uint32_t)bkey));
            }
        }
        // the next iteration's random numbers while the exchange is in flight: drawn by the
        // warps that do not poll (by warp 0 itself only when it is the block's one warp)
        if (it < iter0 + n_iters) {
            if (B == 32) {
                if (active) draw_iteration(rnd + tid, npairs, B, (uint32_t)p, (uint32_t)(it + 1), c);
            } else if (tid >= 32) {
                for (int i = tid - 32; i < npairs * B; i += B - 32) {
                    const int j = i / B, q = i - j * B;
                    if (base + q < sw.M)
                        rnd[i] = philox4x32_10(make_uint4((uint32_t)(base + q), (uint32_t)(it + 1), (uint32_t)j,
                                                          c.stream_id), c.key0, c.key1);
                }
            }
        }
        if (tid < 32) {
            unsigned long long best = ~0ull;
            int bblk = 0;
            bool ok = false;
            for (unsigned spin = 0; spin < spin_limit; ++spin) {
                bool ready = true;
                for (int b = tid; b < G; b += 32) {
                    const ExchangeSlot* sl = row + b;
                    const unsigned long long wl = __ldcg(&sl->w_loss), wi = __ldcg(&sl->w_idx);
                    bool rdy = (unsigned)(wl >> 32) == tag && (unsigned)(wi >> 32) == tag;
                    for (int d = 0; d < P; ++d) {
                        const unsigned long long wp = __ldcg(&sl->w_pos[d]);
                        rdy &= (unsigned)(wp >> 32) == tag;
                        slot_pos[b * P + d] = __uint_as_float((uint32_t)wp);
                    }
                    if (rdy) {
                        const unsigned long long kb = ((wl & 0xFFFFFFFFull) << 32) | (wi & 0xFFFFFFFFull);
                        if (kb < best) {
                            best = kb;
                            bblk = b;
                        }
                    }
                    ready &= rdy;
                }
                if (__all_sync(0xFFFFFFFFu, ready)) {
                    ok = true;
                    break;
                }
                best = ~0ull;
                if ((spin & 63) == 63 && __any_sync(0xFFFFFFFFu, tid == 0 && __ldcg(r.abort) != 0u)) break;
                __nanosleep(32);
            }
            if (ok) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long k2 = __shfl_xor_sync(0xFFFFFFFFu, best, off);
                    const int b2 = __shfl_xor_sync(0xFFFFFFFFu, bblk, off);
                    if (k2 < best) {
                        best = k2;
                        bblk = b2;
                    }
                }
                __syncwarp();
                if (tid < P) g_s[tid] = slot_pos[bblk * P + tid];
            } else if (tid == 0) {
                atomicOr(r.err, kErrTimeout);
                atomicExch(r.abort, 1u);
            }
            if (tid == 0) {
                s_flag = ok ? 1 : 0;
                s_gkey = best;
            }
        }
        __syncthreads();
        aborted = (s_flag == 0);
        gkey = s_gkey;
    }

    // no block leaves while another may still read its exchange words
    if (CLUSTER && n_iters > 0) cooperative_groups::this_cluster().sync();
    // write the swarm back
    for (int i = tid; i < P * B; i += B) {
        const int d = i / B, j = i - d * B, q = base + j;
        if (q < sw.M) {
            const size_t off = (size_t)d * sw.ld + q;
            sw.x[off] = xs[i];
            sw.v[off] = vs[i];
            sw.pb[off] = pbs[i];
        }
    }
    if (active) sw.pbf[p] = pbfs[tid];
    if (blockIdx.x == 0 && !aborted && n_iters > 0) {
        if (tid < P) sw.gbest[tid] = g_s[tid];
        if (tid == 0) {
            *r.gbest_idx = (int)(gkey & 0xFFFFFFFFu);
            *(float*)r.gbest_f = from_ordered_bits((uint32_t)(gkey >> 32));
        }
    }
}

}  // namespace

size_t smem_bytes_persistent(const WindowDev& w, const ModelDev& m, int block, int grid) {
    const size_t floats = (size_t)obs_span_pad(w, m) * (m.cost == COST_MAPE ? 2 : 1) + 4 * (size_t)m.P * block + block +
                          3 * kMaxParams + pad4(grid * m.P);
    return floats * sizeof(float) + (size_t)((m.P + 1) / 2) * block * sizeof(uint4);
}

// Largest grid of `block`-thread blocks that can be co-resident for this problem (0 if none).
// Whether the whole grid fits as one thread-block cluster (at most kMaxClusterBlocks blocks).
bool cluster_fits(const WindowDev& w, const ModelDev& m, int block, int grid) {
    if (grid < 1 || grid > kMaxClusterBlocks) return false;
    const size_t sm = smem_bytes_persistent(w, m, block, grid);
    const void* fn = (const void*)pso_f32_persistent<0, COST_MSE, true>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (sm > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)grid;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
    (void)cudaGetLastError();
    return e == cudaSuccess && n >= 1;
}

int persistent_capacity(const WindowDev& w, const ModelDev& m, int block, int grid) {
    const size_t sm = smem_bytes_persistent(w, m, block, grid);
    int dev = 0, nsm = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const void* fn = nullptr;
    switch (m.cost) {  // every instantiation has the same resources; use the MSE / runtime-spd one
        default: fn = (const void*)pso_f32_persistent<0, COST_MSE, false>; break;
    }
    if (sm > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, sm) != cudaSuccess) return 0;
    (void)cudaGetLastError();
    return per * nsm;
}

cudaError_t launch_pso_f32_persistent(const WindowDev& w, const ModelDev& m, const ObsDev& o,
                                      const PsoCoeffs<float>& c, const SwarmDev<float>& sw, const ReduceScratch& r,
                                      ExchangeSlot* slots, int iter0, int n_iters, int block, cudaStream_t s) {
    const unsigned grid = (unsigned)((sw.M + block - 1) / block);
    const size_t sm = smem_bytes_persistent(w, m, block, (int)grid);
    (void)cudaGetLastError();
    // tags of both parities back to 0 so no slot looks current before it is written
    cudaError_t e = cudaMemsetAsync(slots, 0, 2 * (size_t)grid * sizeof(ExchangeSlot), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.abort, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    SIRD_DISPATCH_F32(m, {
        auto kern = pso_f32_persistent<S_, C_, false>;
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(block);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, kern, w, m, o, c, sw, r, slots, iter0, n_iters,
                                   bounded_wait_limit(kSpinLimit));
        }
    });
    return e;
}

cudaError_t launch_pso_f32_cluster(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<float>& c,
                                   const SwarmDev<float>& sw, const ReduceScratch& r, int iter0, int n_iters, int block,
                                   cudaStream_t s) {
    const unsigned grid = (unsigned)((sw.M + block - 1) / block);
    if (grid > (unsigned)kMaxClusterBlocks) return cudaErrorInvalidValue;
    const size_t sm = smem_bytes_persistent(w, m, block, (int)grid);
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
    SIRD_DISPATCH_F32(m, {
        auto kern = pso_f32_persistent<S_, C_, true>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess && sm > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(block);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = grid;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, kern, w, m, o, c, sw, r, (ExchangeSlot*)nullptr, iter0, n_iters, 0u);
        }
    });
    return e;
}

}  // namespace sird
