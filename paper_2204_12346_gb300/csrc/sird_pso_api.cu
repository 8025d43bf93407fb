// sird_pso_api.cu -- the C ABI (include/sird_pso.h): validation, device memory, graphs.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sird_pso.h"
#include "kernels.h"
#include "trace.h"

using namespace sird;

namespace {

thread_local std::string g_create_error;

struct Split {
    float h, l;
};
Split split(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

constexpr uint32_t kStateMagic = 0x44524953u;  // "SIRD"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
    uint32_t magic, version;
    int32_t M, P, precision, iter, gbest_idx, reserved;
    uint64_t seed;
    uint32_t stream_id, reserved2;
};

}  // namespace

void sird::set_global_error(const char* msg) { g_create_error = msg; }

namespace {

int nparams_of(const sird_problem* pb) {
    return (pb->beta_form == SIRD_BETA_RAMP ? 6 : pb->K + 2) + (pb->fit_I0 ? 1 : 0);
}

}  // namespace

struct sird_pso {
    // problem
    WindowDev win{};
    ModelDev mdl{};
    double ss_tot = 0.0;  // sum (y - mean y)^2 of the observed deaths, for R^2
    // configuration
    int M = 0, ld = 0, P = 0, iters = 0, precision = 32, block = 128, reeval_k = 0;
    bool persistent = false;
    bool cluster = false;  // persistent in one thread-block cluster (exchange in shared memory)
    int cblock = 0;        // its threads per block
    void* d_slots = nullptr;  // abort flag + exchange slots of the persistent kernel
    ExchangeSlot* slots = nullptr;
    PsoCoeffs<float> c32{};
    PsoCoeffs<double> c64{};
    uint64_t seed = 0;
    uint32_t stream_id = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // library-owned stream the calibration graph is captured on
    int iter = -1;  // completed iterations; -1 before init
    // device memory
    void* d_mem = nullptr;   // swarm
    void* d_obs = nullptr;   // observations
    void* d_aux = nullptr;   // reduction scratch, top-k keys, result
    ObsDev obs{};
    void *x = nullptr, *v = nullptr, *pb = nullptr, *pbf = nullptr, *gbest = nullptr;
    ReduceScratch red{};
    unsigned long long *tk_a = nullptr, *tk_b = nullptr;
    ResultDev* d_res = nullptr;
    ResultDev* h_res = nullptr;  // pinned
    cudaGraphExec_t calib = nullptr;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // optional timing events (sird_pso_set_timing)
    double* h_stage = nullptr;                          // pinned staging for observation uploads
    void* d_ckpt = nullptr;                             // adjoint checkpoints (grown on demand)
    size_t ckpt_bytes = 0;
    int n_obs = 0;
    int shard_total = 0;  // > 0: the handle holds particles c32.p_off .. c32.p_off + M - 1 of a swarm this size
    // errors
    sird_status sticky = SIRD_OK;
    std::string msg;

    sird_status fail(sird_status s, const std::string& m) {
        if (sticky == SIRD_OK) {
            sticky = s;
            msg = m;
        }
        return s;
    }
    sird_status cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return SIRD_OK;
        (void)cudaGetLastError();  // the status now lives in the handle; do not leak it into later launches
        return fail(SIRD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }

    SwarmDev<float> sw32() const {
        return {(float*)x, (float*)v, (float*)pb, (float*)pbf, (float*)gbest, M, ld};
    }
    SwarmDev<double> sw64() const {
        return {(double*)x, (double*)v, (double*)pb, (double*)pbf, (double*)gbest, M, ld};
    }

    cudaError_t enqueue_iter(int t, cudaStream_t s) {
        if (precision == 32) return launch_pso_f32(win, mdl, obs, c32, sw32(), red, t, block, s);
        return launch_pso_f64(win, mdl, obs, c64, sw64(), red, t, block, s);
    }
    // iterations iter0+1 .. iter0+n
    cudaError_t enqueue_iters(int iter0, int n, cudaStream_t s) {
        if (n <= 0) return cudaSuccess;
        if (cluster) return launch_pso_f32_cluster(win, mdl, obs, c32, sw32(), red, iter0, n, cblock, s);
        if (persistent) return launch_pso_f32_persistent(win, mdl, obs, c32, sw32(), red, slots, iter0, n, block, s);
        for (int t = iter0 + 1; t <= iter0 + n; ++t) {
            cudaError_t e = enqueue_iter(t, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t enqueue_result(cudaStream_t s) {
        // a shard's global-best index is global and may lie in another shard: it re-evaluates
        // the best of its own particles, found by the top-k selection (local indices)
        const int k = (precision == 32 && shard_total > 0 && reeval_k == 0) ? 1 : reeval_k;
        if (precision == 32 && k > 0) {
            unsigned long long* keys = nullptr;
            cudaError_t e = launch_topk_f32((const float*)pbf, M, k, tk_a, tk_b, &keys, s);
            if (e != cudaSuccess) return e;
            e = launch_reeval(win, mdl, obs, &c32, nullptr, pb, pbf, ld, keys, k, nullptr, d_res, s);
            if (e != cudaSuccess) return e;
        } else {
            cudaError_t e = launch_reeval(win, mdl, obs, precision == 32 ? &c32 : nullptr,
                                          precision == 64 ? &c64 : nullptr, pb, pbf, ld, nullptr, 1, red.gbest_idx,
                                          d_res, s);
            if (e != cudaSuccess) return e;
        }
        return cudaMemcpyAsync(h_res, d_res, sizeof(ResultDev), cudaMemcpyDeviceToHost, s);
    }
    void fill_result(sird_result* out) const {
        std::memset(out, 0, sizeof(*out));
        out->n_params = P;
        for (int d = 0; d < P; ++d) out->theta[d] = h_res->theta[d];
        out->loss = h_res->loss;
        out->loss_search = h_res->loss_search;
        out->r2_D = ss_tot > 0 ? 1.0 - h_res->sse / ss_tot : NAN;
        out->index = h_res->index + (int)c32.p_off;  // global particle index (a shard's offset added)
        out->iters_done = iter;
    }
};

unsigned sird::bounded_wait_limit(unsigned dflt) {
    const char* v = std::getenv("SIRD_WAIT_LIMIT");
    if (!v || !*v) return dflt;
    const long long x = std::atoll(v);
    return x > 0 && x < (1LL << 31) ? (unsigned)x : dflt;
}

// ---------------------------------------------------------------- validation

sird_status sird_check_problem(const sird_problem* pb, std::string& why) {
    if (!pb) return why = "problem is NULL", SIRD_ERR_ARG;
    if (pb->n_obs < 2 || pb->n_obs > SIRD_MAX_OBS) return why = "n_obs out of range [2, SIRD_MAX_OBS]", SIRD_ERR_ARG;
    if (!pb->y_D) return why = "y_D is NULL", SIRD_ERR_ARG;
    for (int i = 0; i < pb->n_obs; ++i)
        if (!std::isfinite(pb->y_D[i])) return why = "non-finite observation in y_D", SIRD_ERR_ARG;
    if (!(pb->N > 0) || !std::isfinite(pb->N)) return why = "N must be finite and positive", SIRD_ERR_ARG;
    if (!std::isfinite(pb->R0) || !std::isfinite(pb->I0)) return why = "I0/R0 must be finite", SIRD_ERR_ARG;
    if (pb->steps_per_day < 1 || pb->steps_per_day > 1000) return why = "steps_per_day out of range [1, 1000]", SIRD_ERR_ARG;
    if ((long long)(pb->n_obs - 1) * pb->steps_per_day > (1LL << 30)) return why = "too many Euler steps", SIRD_ERR_ARG;
    if (pb->beta_form != SIRD_BETA_PWC && pb->beta_form != SIRD_BETA_RAMP) return why = "unknown beta_form", SIRD_ERR_ARG;
    if (pb->beta_form == SIRD_BETA_PWC && (pb->K < 1 || pb->K > SIRD_MAX_PARAMS - 3))
        return why = "K out of range [1, SIRD_MAX_PARAMS-3]", SIRD_ERR_ARG;
    if (pb->cost < SIRD_COST_MSE || pb->cost > SIRD_COST_MAPE) return why = "unknown cost", SIRD_ERR_ARG;
    if (pb->fit_I0 != 0 && pb->fit_I0 != 1) return why = "fit_I0 must be 0 or 1", SIRD_ERR_ARG;
    if (pb->objective != SIRD_FIT_D && pb->objective != SIRD_FIT_IRD) return why = "unknown objective", SIRD_ERR_ARG;
    if (pb->objective == SIRD_FIT_IRD) {
        if (!pb->y_I || !pb->y_R) return why = "F_IRD needs y_I and y_R", SIRD_ERR_ARG;
        for (int i = 0; i < pb->n_obs; ++i)
            if (!std::isfinite(pb->y_I[i]) || !std::isfinite(pb->y_R[i]))
                return why = "non-finite observation in y_I / y_R", SIRD_ERR_ARG;
    }
    return SIRD_OK;
}

void sird_fill_window(const sird_problem* pb, WindowDev& w, ModelDev& m) {
    const int n = pb->n_obs;
    w.n_obs = n;
    w.n_kept = 0;
    for (int i = 0; i < n; ++i) w.n_kept += (pb->y_D[i] != 0.0);
    w.N = pb->N;
    w.I0 = pb->I0;
    w.R0 = pb->R0;
    w.D0 = pb->y_D[0];
    w.dt = 1.0 / (double)pb->steps_per_day;
    Split s = split(pb->N);
    w.Nh = s.h;
    w.Nl = s.l;
    s = split(pb->R0 + pb->y_D[0]);
    w.RD0h = s.h;
    w.RD0l = s.l;
    s = split(pb->I0);
    w.I0f = s.h;
    w.I0l = s.l;
    s = split(w.dt / pb->N);
    w.cbn_h = s.h;
    w.cbn_l = s.l;
    s = split(w.dt);
    w.dt_h = s.h;
    w.dt_l = s.l;
    s = split(pb->R0);
    w.R0h = s.h;
    w.R0l = s.l;
    s = split(pb->N - pb->R0 - pb->y_D[0]);  // S0 + I0, whatever I0
    w.Q0h = s.h;
    w.Q0l = s.l;
    // F_IRD: ranges of the reported series for the min-max normalisation (a flat series: 1)
    auto range = [n](const double* y) {
        double lo = y[0], hi = y[0];
        for (int i = 1; i < n; ++i) {
            lo = y[i] < lo ? y[i] : lo;
            hi = y[i] > hi ? y[i] : hi;
        }
        return hi > lo ? hi - lo : 1.0;
    };
    const bool ird = pb->objective == SIRD_FIT_IRD;
    w.rng_D = ird ? range(pb->y_D) : 1.0;
    w.rng_I = ird ? range(pb->y_I) : 1.0;
    w.rng_R = ird ? range(pb->y_R) : 1.0;
    w.inv_rng_D = (float)(1.0 / w.rng_D);
    w.inv_rng_I = (float)(1.0 / w.rng_I);
    w.inv_rng_R = (float)(1.0 / w.rng_R);
    w.eR0 = ird ? (float)(pb->y_R[0] - pb->R0) : 0.f;
    w.n_kept_I = w.n_kept_R = 0;
    if (ird)
        for (int i = 0; i < n; ++i) {
            w.n_kept_I += (pb->y_I[i] != 0.0);
            w.n_kept_R += (pb->y_R[i] != 0.0);
        }
    m.ird = ird ? 1 : 0;
    m.P = nparams_of(pb);
    m.K = pb->beta_form == SIRD_BETA_PWC ? pb->K : 1;
    m.spd = pb->steps_per_day;
    m.beta_form = pb->beta_form;
    m.fit_I0 = pb->fit_I0;
    m.cost = pb->cost;
}

// Observations to the device: float copy, float reciprocals (0 where y == 0), double copy, each
// holding the series stacked D | I | R (I, R for F_IRD only) with stride obs_stride(n).
static cudaError_t upload_obs(const sird_problem* pb, void** mem, ObsDev& o, cudaStream_t s) {
    const int n = pb->n_obs;
    const int nser = pb->objective == SIRD_FIT_IRD ? 3 : 1;
    const size_t ps = (size_t)obs_stride(n), nf = ps * nser;
    const size_t bytes = nf * 2 * sizeof(float) + nf * sizeof(double);
    cudaError_t e = cudaMalloc(mem, bytes);
    if (e != cudaSuccess) return e;
    std::vector<unsigned char> host(bytes, 0);
    float* yf = (float*)host.data();
    float* inv = yf + nf;
    double* yd = (double*)(inv + nf);
    const double* series[3] = {pb->y_D, pb->y_I, pb->y_R};
    for (int k = 0; k < nser; ++k)
        for (int i = 0; i < n; ++i) {
            const double y = series[k][i];
            yf[k * ps + i] = obs_f32(series[k], i, k != 1);
            inv[k * ps + i] = y != 0.0 ? (float)(1.0 / y) : 0.f;
            yd[k * ps + i] = y;
        }
    e = cudaMemcpyAsync(*mem, host.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    o.yf = (const float*)*mem;
    o.invyf = o.yf + nf;
    o.yd = (const double*)(o.invyf + nf);
    return e;
}

// ---------------------------------------------------------------- lifetime

extern "C" sird_status sird_pso_create(const sird_problem* pb, const sird_pso_config* cfg, void* cuda_stream,
                                       sird_pso_t* out) {
    if (!out) return g_create_error = "out is NULL", SIRD_ERR_ARG;
    *out = nullptr;
    std::string why;
    sird_status st = sird_check_problem(pb, why);
    if (st != SIRD_OK) return g_create_error = why, st;
    if (!cfg) return g_create_error = "config is NULL", SIRD_ERR_ARG;
    const int P = nparams_of(pb);
    if (P > SIRD_MAX_PARAMS) return g_create_error = "too many parameters", SIRD_ERR_ARG;
    if (cfg->particles < 1 || cfg->particles > SIRD_MAX_PARTICLES) return g_create_error = "particles out of range", SIRD_ERR_ARG;
    if (cfg->iters < 0) return g_create_error = "iters < 0", SIRD_ERR_ARG;
    if (cfg->precision != 32 && cfg->precision != 64) return g_create_error = "precision must be 32 or 64", SIRD_ERR_ARG;
    if (!cfg->lb || !cfg->ub) return g_create_error = "lb/ub is NULL", SIRD_ERR_ARG;
    if (cfg->block_size != 0 && (cfg->block_size < 32 || cfg->block_size > 1024 || cfg->block_size % 32))
        return g_create_error = "block_size must be 0 or a multiple of 32 in [32, 1024]", SIRD_ERR_ARG;
    if (cfg->precision == 64 && cfg->block_size > 256) return g_create_error = "FP64 block_size must be <= 256", SIRD_ERR_ARG;
    if (cfg->launch_mode < SIRD_LAUNCH_AUTO ||
        (cfg->launch_mode > SIRD_LAUNCH_PERSISTENT && cfg->launch_mode != SIRD_LAUNCH_CLUSTER))
        return g_create_error = "unknown launch_mode", SIRD_ERR_ARG;
    if ((cfg->launch_mode == SIRD_LAUNCH_PERSISTENT || cfg->launch_mode == SIRD_LAUNCH_CLUSTER) && cfg->precision != 32)
        return g_create_error = "the persistent and cluster launches are FP32 only", SIRD_ERR_UNSUPPORTED;
    if (cfg->reeval_topk < 0 || cfg->reeval_topk > 1024 || cfg->reeval_topk > cfg->particles)
        return g_create_error = "reeval_topk out of range [0, min(particles, 1024)]", SIRD_ERR_ARG;
    for (int d = 0; d < P; ++d) {
        const bool lg = cfg->log_scale && cfg->log_scale[d];
        if (!std::isfinite(cfg->lb[d]) || !std::isfinite(cfg->ub[d]) || cfg->lb[d] > cfg->ub[d])
            return g_create_error = "bounds must be finite with lb <= ub", SIRD_ERR_ARG;
        if (lg && !(cfg->lb[d] > 0)) return g_create_error = "log_scale needs lb > 0", SIRD_ERR_ARG;
    }

    sird_pso* h = new (std::nothrow) sird_pso();
    if (!h) return g_create_error = "host allocation failed", SIRD_ERR_NOMEM;
    h->stream = (cudaStream_t)cuda_stream;
    h->n_obs = pb->n_obs;
    sird_fill_window(pb, h->win, h->mdl);
    {
        double mean = 0;
        for (int i = 0; i < pb->n_obs; ++i) mean += pb->y_D[i];
        mean /= pb->n_obs;
        for (int i = 0; i < pb->n_obs; ++i) h->ss_tot += (pb->y_D[i] - mean) * (pb->y_D[i] - mean);
    }
    h->M = cfg->particles;
    h->ld = (cfg->particles + 31) & ~31;
    h->P = P;
    h->iters = cfg->iters;
    h->precision = cfg->precision;
    h->block = cfg->block_size ? cfg->block_size : (cfg->precision == 32 ? 128 : 64);
    h->reeval_k = cfg->precision == 32 ? cfg->reeval_topk : 0;
    h->seed = cfg->seed;
    h->stream_id = cfg->stream_id;
    uint32_t logmask = 0;
    for (int d = 0; d < P; ++d) {
        const bool lg = cfg->log_scale && cfg->log_scale[d];
        if (lg) logmask |= 1u << d;
        const double zl = lg ? std::log(cfg->lb[d]) : cfg->lb[d];
        const double zu = lg ? std::log(cfg->ub[d]) : cfg->ub[d];
        h->c64.zlb[d] = zl;
        h->c64.zub[d] = zu;
        h->c32.zlb[d] = (float)zl;
        h->c32.zub[d] = (float)zu;
    }
    h->c64.w = cfg->w;
    h->c64.c1 = cfg->c1;
    h->c64.c2 = cfg->c2;
    h->c32.w = (float)cfg->w;
    h->c32.c1 = (float)cfg->c1;
    h->c32.c2 = (float)cfg->c2;
    h->c32.logmask = h->c64.logmask = logmask;
    h->c32.key0 = h->c64.key0 = (uint32_t)cfg->seed;
    h->c32.key1 = h->c64.key1 = (uint32_t)(cfg->seed >> 32);
    h->c32.stream_id = h->c64.stream_id = cfg->stream_id;

    if (h->precision == 32 && smem_bytes_f32(h->win, h->mdl, h->block, true) > 227 * 1024) {
        g_create_error = "block_size too large for this many parameters (shared memory)";
        sird_pso_destroy(h);
        return SIRD_ERR_ARG;
    }
    auto bail = [&](cudaError_t e, const char* what) {
        g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
        sird_pso_destroy(h);
        return e == cudaErrorMemoryAllocation ? SIRD_ERR_NOMEM : SIRD_ERR_CUDA;
    };
    cudaError_t e = upload_obs(pb, &h->d_obs, h->obs, h->stream);
    if (e != cudaSuccess) return bail(e, "uploading observations");

    const size_t tsz = h->precision == 32 ? sizeof(float) : sizeof(double);
    const size_t plane = (size_t)P * h->ld * tsz;
    const size_t swarm_bytes = 3 * plane + (size_t)h->ld * tsz + SIRD_MAX_PARAMS * tsz;
    e = cudaMalloc(&h->d_mem, swarm_bytes);
    if (e != cudaSuccess) return bail(e, "allocating the swarm");
    unsigned char* base = (unsigned char*)h->d_mem;
    h->x = base;
    h->v = base + plane;
    h->pb = base + 2 * plane;
    h->pbf = base + 3 * plane;
    h->gbest = base + 3 * plane + (size_t)h->ld * tsz;

    const size_t grid = (size_t)((h->M + h->block - 1) / h->block);
    // top-k keys for the FP32 re-evaluation (at least the best one: a shard's result uses them)
    const int tk_k = h->precision == 32 ? (h->reeval_k > 1 ? h->reeval_k : 1) : h->reeval_k;
    const size_t tk = tk_k > 0 ? topk_scratch_keys(h->M, tk_k) : 0;
    const size_t aux_bytes = 256 + grid * sizeof(MinPair64) + 2 * tk * sizeof(unsigned long long) + sizeof(ResultDev);
    e = cudaMalloc(&h->d_aux, aux_bytes);
    if (e != cudaSuccess) return bail(e, "allocating scratch");
    unsigned char* a = (unsigned char*)h->d_aux;
    h->red.gkey = (unsigned long long*)a;
    h->red.counter = (unsigned int*)(a + 8);
    h->red.gbest_idx = (int*)(a + 16);
    h->red.gbest_f = a + 24;
    h->red.err = (unsigned*)(a + 32);
    h->red.partial = (MinPair64*)(a + 256);
    h->tk_a = (unsigned long long*)(a + 256 + grid * sizeof(MinPair64));
    h->tk_b = h->tk_a + tk;
    h->d_res = (ResultDev*)(h->tk_b + tk);
    e = cudaMemsetAsync(h->d_aux, 0, 256, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->red.gkey, 0xFF, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(e, "initialising scratch");
    e = cudaMallocHost((void**)&h->h_res, sizeof(ResultDev));
    if (e != cudaSuccess) return bail(e, "allocating pinned result");
    if (h->precision == 32 && (cfg->launch_mode == SIRD_LAUNCH_AUTO || cfg->launch_mode == SIRD_LAUNCH_CLUSTER)) {
        // one cluster of the handle's blocks (one warp per scheduler at the default 128 threads:
        // swarms of up to 2048 particles); an explicit cluster request without a block size
        // splits the swarm over 16 blocks
        int cb = h->block;
        if (cfg->launch_mode == SIRD_LAUNCH_CLUSTER && !cfg->block_size)
            cb = std::min(1024, std::max(32, ((h->M + kMaxClusterBlocks - 1) / kMaxClusterBlocks + 31) / 32 * 32));
        const int cgrid = (h->M + cb - 1) / cb;
        // AUTO takes it from 4 blocks on: measured 1.5-4% faster than the global exchange at
        // 1024-2048 particles, equal at 512, slower for a single block
        const bool want = cfg->launch_mode == SIRD_LAUNCH_CLUSTER || cgrid >= 4;
        if (want && cgrid <= kMaxClusterBlocks && cluster_fits(h->win, h->mdl, cb, cgrid)) {
            h->cluster = h->persistent = true;
            h->cblock = cb;
        } else if (cfg->launch_mode == SIRD_LAUNCH_CLUSTER) {
            g_create_error = "cluster launch requested but the swarm does not fit one cluster of <= 16 blocks";
            sird_pso_destroy(h);
            return SIRD_ERR_UNSUPPORTED;
        }
    }
    if (h->precision == 32 && !h->cluster && cfg->launch_mode != SIRD_LAUNCH_PER_ITER) {
        const int cap = persistent_capacity(h->win, h->mdl, h->block, (int)grid);
        const bool fits = grid <= (size_t)cap && grid <= (size_t)kMaxPersistentBlocks;
        if (!fits && cfg->launch_mode == SIRD_LAUNCH_PERSISTENT) {
            g_create_error = "persistent launch requested but the blocks cannot all be co-resident";
            sird_pso_destroy(h);
            return SIRD_ERR_UNSUPPORTED;
        }
        if (fits) {
            e = cudaMalloc(&h->d_slots, 256 + 2 * grid * sizeof(ExchangeSlot));
            if (e != cudaSuccess) return bail(e, "allocating exchange slots");
            h->red.abort = (unsigned*)h->d_slots;
            h->slots = (ExchangeSlot*)((unsigned char*)h->d_slots + 256);
            h->persistent = true;
        }
    }
    *out = h;
    return SIRD_OK;
}

extern "C" void sird_pso_destroy(sird_pso_t h) {
    if (!h) return;
    if (h->stream || h->d_mem) cudaStreamSynchronize(h->stream);
    if (h->calib) cudaGraphExecDestroy(h->calib);
    if (h->cap) cudaStreamDestroy(h->cap);
    cudaFree(h->d_mem);
    cudaFree(h->d_obs);
    cudaFree(h->d_aux);
    cudaFree(h->d_slots);
    cudaFree(h->d_ckpt);
    if (h->h_res) cudaFreeHost(h->h_res);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    delete h;
}

extern "C" const char* sird_last_error(sird_pso_t h) {
    if (!h) return g_create_error.c_str();
    return h->msg.c_str();
}

extern "C" sird_status sird_pso_clear_error(sird_pso_t h) {
    if (!h) return SIRD_ERR_ARG;
    h->sticky = SIRD_OK;
    h->msg.clear();
    return SIRD_OK;
}

extern "C" sird_status sird_pso_set_stream(sird_pso_t h, void* cuda_stream) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if ((cudaStream_t)cuda_stream != h->stream) {
        sird_status s = h->cuda(cudaStreamSynchronize(h->stream), "synchronising the old stream");
        if (s) return s;
        h->stream = (cudaStream_t)cuda_stream;
        if (h->calib) {
            cudaGraphExecDestroy(h->calib);
            h->calib = nullptr;
        }
    }
    return SIRD_OK;
}

extern "C" int sird_pso_num_params(sird_pso_t h) { return h ? h->P : 0; }

extern "C" int sird_pso_launch_mode(sird_pso_t h) {
    if (!h) return 0;
    return h->cluster ? SIRD_LAUNCH_CLUSTER : (h->persistent ? SIRD_LAUNCH_PERSISTENT : SIRD_LAUNCH_PER_ITER);
}

// ---------------------------------------------------------------- fitness

extern "C" sird_status sird_pso_eval(sird_pso_t h, const void* d_theta, int M, int ld, void* d_loss, int precision) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (M < 0 || ld < M || (M > 0 && (!d_theta || !d_loss))) return h->fail(SIRD_ERR_ARG, "eval: bad M/ld/pointers");
    if (precision != 32 && precision != 64) return h->fail(SIRD_ERR_ARG, "eval: precision must be 32 or 64");
    if (M == 0) return SIRD_OK;
    const int block = precision == 32 ? 128 : 64;
    cudaError_t e = precision == 32
                        ? launch_eval_f32(h->win, h->mdl, h->obs, (const float*)d_theta, ld, M, (float*)d_loss, block,
                                          h->red.err, h->stream)
                        : launch_eval_f64(h->win, h->mdl, h->obs, (const double*)d_theta, ld, M, (double*)d_loss,
                                          block, h->red.err, h->stream);
    return h->cuda(e, "eval launch");
}

// ---------------------------------------------------------------- swarm

extern "C" sird_status sird_pso_init(sird_pso_t h) {
    TraceRange trace("sird_pso_init");
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    sird_status s = h->cuda(h->enqueue_iter(0, h->stream), "init launch");
    if (s) return s;
    h->iter = 0;
    return SIRD_OK;
}

extern "C" sird_status sird_pso_step(sird_pso_t h, int n_iters) {
    TraceRange trace("sird_pso_step");
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (n_iters < 0) return h->fail(SIRD_ERR_ARG, "step: n_iters < 0");
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "step before init/set_state");
    sird_status s = h->cuda(h->enqueue_iters(h->iter, n_iters, h->stream), "step launch");
    if (s) return s;
    h->iter += n_iters;
    return SIRD_OK;
}

extern "C" sird_status sird_pso_sync(sird_pso_t h) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    sird_status s = h->cuda(cudaStreamSynchronize(h->stream), "sync");
    if (s) return s;
    unsigned err = 0;
    s = h->cuda(cudaMemcpy(&err, h->red.err, sizeof(err), cudaMemcpyDeviceToHost), "reading the error word");
    if (s) return s;
    if (err & kErrTimeout) return h->fail(SIRD_ERR_TIMEOUT, "a device-side wait ran out");
    if (err & kErrBounds) return h->fail(SIRD_ERR_ARG, "a device-side index check failed");
    return SIRD_OK;
}

extern "C" sird_status sird_pso_set_observations(sird_pso_t h, const double* y_D, int n_obs) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (!y_D || n_obs != h->n_obs) return h->fail(SIRD_ERR_ARG, "set_observations: y_D NULL or n_obs differs");
    if (h->mdl.ird) return h->fail(SIRD_ERR_UNSUPPORTED, "set_observations: F_D handles only");
    for (int i = 0; i < n_obs; ++i)
        if (!std::isfinite(y_D[i])) return h->fail(SIRD_ERR_ARG, "set_observations: non-finite observation");
    if (y_D[0] != h->win.D0) return h->fail(SIRD_ERR_ARG, "set_observations: y_D[0] (D0) must not change");
    const size_t nf = (size_t)((n_obs + 3) & ~3);
    const size_t bytes = nf * 2 * sizeof(float) + (size_t)n_obs * sizeof(double);
    sird_status s = SIRD_OK;
    if (!h->h_stage) s = h->cuda(cudaMallocHost((void**)&h->h_stage, bytes), "allocating pinned staging");
    if (s) return s;
    s = h->cuda(cudaStreamSynchronize(h->stream), "sync");  // the previous upload may still read the stage
    if (s) return s;
    float* yf = (float*)h->h_stage;
    float* inv = yf + nf;
    double* yd = (double*)(inv + nf);
    std::memset(h->h_stage, 0, bytes);
    int kept = 0;
    double mean = 0.0, ss = 0.0;
    for (int i = 0; i < n_obs; ++i) {
        yf[i] = obs_f32(y_D, i, true);
        inv[i] = y_D[i] != 0.0 ? (float)(1.0 / y_D[i]) : 0.f;
        yd[i] = y_D[i];
        kept += (y_D[i] != 0.0);
        mean += y_D[i];
    }
    mean /= n_obs;
    for (int i = 0; i < n_obs; ++i) ss += (y_D[i] - mean) * (y_D[i] - mean);
    if (kept != h->win.n_kept) return h->fail(SIRD_ERR_ARG, "set_observations: the count of zero observations must not change");
    h->ss_tot = ss;
    return h->cuda(cudaMemcpyAsync((void*)h->obs.yf, h->h_stage, bytes, cudaMemcpyHostToDevice, h->stream),
                   "uploading observations");
}

extern "C" sird_status sird_pso_set_timing(sird_pso_t h, void* event_iter_begin, void* event_iter_end) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    h->ev_begin = (cudaEvent_t)event_iter_begin;
    h->ev_end = (cudaEvent_t)event_iter_end;
    if (h->calib) {
        cudaGraphExecDestroy(h->calib);
        h->calib = nullptr;
    }
    return SIRD_OK;
}

extern "C" sird_status sird_pso_result(sird_pso_t h, sird_result* out) {
    if (!h || !out) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "result before init");
    sird_status s = h->cuda(h->enqueue_result(h->stream), "result launch");
    if (s) return s;
    s = sird_pso_sync(h);
    if (s) return s;
    h->fill_result(out);
    return SIRD_OK;
}

extern "C" sird_status sird_pso_calibrate(sird_pso_t h, sird_result* out) {
    TraceRange trace("sird_pso_calibrate");
    if (!h || !out) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->shard_total > 0)
        return h->fail(SIRD_ERR_STATE, "calibrate: a shard steps with sird_pso_step, its global best set between steps");
    if (!h->calib) {
        // captured once on a private stream (the caller's may be the legacy default stream,
        // which cannot be captured), then launched on the caller's stream
        if (!h->cap) {
            sird_status s = h->cuda(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "capture stream");
            if (s) return s;
        }
        cudaGraph_t g = nullptr;
        sird_status s = h->cuda(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (s) return s;
        cudaError_t e = h->enqueue_iter(0, h->cap);
        if (e == cudaSuccess && h->ev_begin) e = cudaEventRecordWithFlags(h->ev_begin, h->cap, cudaEventRecordExternal);
        if (e == cudaSuccess) e = h->enqueue_iters(0, h->iters, h->cap);
        if (e == cudaSuccess && h->ev_end) e = cudaEventRecordWithFlags(h->ev_end, h->cap, cudaEventRecordExternal);
        if (e == cudaSuccess) e = h->enqueue_result(h->cap);
        cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->calib, g, 0);
        if (g) cudaGraphDestroy(g);
        s = h->cuda(e, "capturing the calibration graph");
        if (s) return s;
    }
    sird_status s = h->cuda(cudaGraphLaunch(h->calib, h->stream), "graph launch");
    if (s) return s;
    h->iter = h->iters;
    s = sird_pso_sync(h);
    if (s) return s;
    h->fill_result(out);
    return SIRD_OK;
}

// ---------------------------------------------------------------- state

extern "C" sird_status sird_pso_get_state(sird_pso_t h, void* buf, size_t* size) {
    if (!h || !size) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->shard_total > 0) return h->fail(SIRD_ERR_UNSUPPORTED, "get_state: not for a shard of a swarm");
    const size_t tsz = h->precision == 32 ? 4 : 8;
    const size_t need = sizeof(StateHeader) + (3 * (size_t)h->P + 1) * h->M * tsz;
    if (!buf) {
        *size = need;
        return SIRD_OK;
    }
    if (*size < need) return h->fail(SIRD_ERR_ARG, "get_state: buffer too small");
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "get_state before init");
    sird_status s = h->cuda(cudaStreamSynchronize(h->stream), "sync");
    if (s) return s;
    StateHeader hd{kStateMagic, kStateVersion, h->M, h->P, h->precision, h->iter, 0, 0, h->seed, h->stream_id, 0};
    s = h->cuda(cudaMemcpy(&hd.gbest_idx, h->red.gbest_idx, sizeof(int), cudaMemcpyDeviceToHost), "get_state");
    if (s) return s;
    unsigned char* p = (unsigned char*)buf;
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const size_t row = (size_t)h->M * tsz, pitch = (size_t)h->ld * tsz;
    for (void* src : {h->x, h->v, h->pb}) {
        s = h->cuda(cudaMemcpy2D(p, row, src, pitch, row, h->P, cudaMemcpyDeviceToHost), "get_state copy");
        if (s) return s;
        p += row * h->P;
    }
    s = h->cuda(cudaMemcpy(p, h->pbf, row, cudaMemcpyDeviceToHost), "get_state copy");
    if (s) return s;
    *size = need;
    return SIRD_OK;
}

extern "C" sird_status sird_pso_set_state(sird_pso_t h, const void* buf, size_t size) {
    if (!h || !buf) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->shard_total > 0) return h->fail(SIRD_ERR_UNSUPPORTED, "set_state: not for a shard of a swarm");
    const size_t tsz = h->precision == 32 ? 4 : 8;
    const size_t need = sizeof(StateHeader) + (3 * (size_t)h->P + 1) * h->M * tsz;
    StateHeader hd;
    if (size < sizeof(hd)) return h->fail(SIRD_ERR_STATE, "set_state: blob too small");
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.M != h->M || hd.P != h->P ||
        hd.precision != h->precision || size < need || hd.iter < 0 || hd.gbest_idx < 0 || hd.gbest_idx >= h->M)
        return h->fail(SIRD_ERR_STATE, "set_state: blob does not match this handle");
    sird_status s = h->cuda(cudaStreamSynchronize(h->stream), "sync");
    if (s) return s;
    const unsigned char* p = (const unsigned char*)buf + sizeof(hd);
    const size_t row = (size_t)h->M * tsz, pitch = (size_t)h->ld * tsz;
    for (void* dst : {h->x, h->v, h->pb}) {
        s = h->cuda(cudaMemcpy2D(dst, pitch, p, row, row, h->P, cudaMemcpyHostToDevice), "set_state copy");
        if (s) return s;
        p += row * h->P;
    }
    s = h->cuda(cudaMemcpy(h->pbf, p, row, cudaMemcpyHostToDevice), "set_state copy");
    if (s) return s;
    // global best = personal best of the recorded index
    std::vector<unsigned char> g(tsz * h->P), gf(tsz);
    const unsigned char* pbh = (const unsigned char*)buf + sizeof(hd) + 2 * row * h->P;
    for (int d = 0; d < h->P; ++d) std::memcpy(&g[d * tsz], pbh + d * row + (size_t)hd.gbest_idx * tsz, tsz);
    std::memcpy(gf.data(), p + (size_t)hd.gbest_idx * tsz, tsz);
    s = h->cuda(cudaMemcpy(h->gbest, g.data(), g.size(), cudaMemcpyHostToDevice), "set_state gbest");
    if (!s) s = h->cuda(cudaMemcpy(h->red.gbest_idx, &hd.gbest_idx, sizeof(int), cudaMemcpyHostToDevice), "set_state");
    if (!s) s = h->cuda(cudaMemcpy(h->red.gbest_f, gf.data(), tsz, cudaMemcpyHostToDevice), "set_state");
    if (s) return s;
    h->iter = hd.iter;
    return SIRD_OK;
}

// ---------------------------------------------------------------- gradient

extern "C" sird_status sird_loss_grad(sird_pso_t h, const void* d_theta, int M, int ld, void* d_loss, void* d_grad,
                                      int ld_grad, void* d_grad_u0, int precision, int ckpt_every) {
    TraceRange trace("sird_loss_grad");
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (M < 0 || ld < M || ld_grad < M || (M > 0 && (!d_theta || !d_loss || !d_grad)))
        return h->fail(SIRD_ERR_ARG, "loss_grad: bad M/ld/pointers");
    if (ckpt_every < 1 || ckpt_every > 64) return h->fail(SIRD_ERR_ARG, "loss_grad: ckpt_every out of range [1, 64]");
    if (precision != 32 && precision != 64) return h->fail(SIRD_ERR_ARG, "loss_grad: precision must be 32 or 64");
    if (precision == 32 && h->mdl.spd != 10 && h->mdl.spd != 20 && h->mdl.spd > 64)
        return h->fail(SIRD_ERR_UNSUPPORTED, "loss_grad: FP32 needs steps_per_day <= 64");
    if (M == 0) return SIRD_OK;
    const size_t need = precision == 64 ? adjoint_ckpt_bytes(h->win, h->mdl, M, ckpt_every)
                                        : adjoint_ckpt_bytes_f32(h->win, h->mdl, M);
    if (need > h->ckpt_bytes) {
        sird_status s = h->cuda(cudaStreamSynchronize(h->stream), "sync");
        if (s) return s;
        cudaFree(h->d_ckpt);
        h->d_ckpt = nullptr;
        h->ckpt_bytes = 0;
        s = h->cuda(cudaMalloc(&h->d_ckpt, need), "allocating adjoint checkpoints");
        if (s) return s;
        h->ckpt_bytes = need;
    }
    if (precision == 32)
        return h->cuda(launch_loss_grad_f32(h->win, h->mdl, h->obs, (const float*)d_theta, ld, M, (float*)d_loss,
                                            (float*)d_grad, ld_grad, (float*)d_grad_u0, (float*)h->d_ckpt, h->stream),
                       "loss_grad launch");
    return h->cuda(launch_loss_grad_f64(h->win, h->mdl, h->obs, (const double*)d_theta, ld, M, (double*)d_loss,
                                        (double*)d_grad, ld_grad, (double*)d_grad_u0, (double*)h->d_ckpt,
                                        ckpt_every, h->stream),
                   "loss_grad launch");
}

extern "C" sird_status sird_pso_polish(sird_pso_t h, int k, int iters, double first_step, int ckpt_every,
                                       int precision, sird_result* out) {
    TraceRange trace("sird_pso_polish");
    if (!h || !out) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->shard_total > 0) return h->fail(SIRD_ERR_STATE, "polish: not for a shard of a swarm");
    if (h->precision != 32) return h->fail(SIRD_ERR_UNSUPPORTED, "polish: FP32 swarms only");
    if (k < 1 || k > 1024 || k > h->M || iters < 0 || !(first_step > 0) || ckpt_every < 1 || ckpt_every > 64 ||
        (precision != 32 && precision != 64))
        return h->fail(SIRD_ERR_ARG, "polish: bad k/iters/first_step/ckpt_every/precision");
    if (precision == 32 && h->mdl.spd != 10 && h->mdl.spd != 20 && h->mdl.spd > 64)
        return h->fail(SIRD_ERR_UNSUPPORTED, "polish: FP32 needs steps_per_day <= 64");
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "polish before init");
    const size_t nk = topk_scratch_keys(h->M, k);
    const size_t ck = precision == 32 ? polish_ckpt_floats(h->win.n_obs, k, h->mdl) * sizeof(float)
                                      : adjoint_ckpt_bytes(h->win, h->mdl, k, ckpt_every);
    // device: the window's table entry | top-k keys (two buffers) | polish state | checkpoints
    const size_t tab_bytes = (sizeof(PolishWin) + 255) & ~(size_t)255;
    const size_t bytes =
        tab_bytes + 2 * nk * sizeof(unsigned long long) + polish_scratch_doubles(h->P, k) * sizeof(double) + ck;
    void* dmem = nullptr;
    sird_status st = h->cuda(cudaMalloc(&dmem, bytes), "polish scratch");
    if (st) return st;
    PolishWin* tab = (PolishWin*)dmem;
    unsigned long long* a = (unsigned long long*)((unsigned char*)dmem + tab_bytes);
    unsigned long long* b = a + nk;
    double* scratch = (double*)(b + nk);
    void* ckpt = scratch + polish_scratch_doubles(h->P, k);
    PolishWin hw{};
    hw.w = h->win;
    hw.o = h->obs;
    hw.pb = (const float*)h->pb;
    hw.pbf = (const float*)h->pbf;
    hw.ld = h->ld;
    hw.M = h->M;
    unsigned long long* keys = nullptr;
    cudaError_t e = cudaMemcpyAsync(tab, &hw, sizeof(PolishWin), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_topk_f32((const float*)h->pbf, h->M, k, a, b, &keys, h->stream);
    if (e == cudaSuccess)
        e = launch_polish(tab, 1, h->win.n_obs, h->win, h->obs, h->mdl, h->c64, keys, k, iters, first_step, precision,
                          scratch, ckpt, ckpt_every, h->d_res, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_res, h->d_res, sizeof(ResultDev), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dmem);
    st = h->cuda(e, "polish");
    if (st) return st;
    h->fill_result(out);
    return SIRD_OK;
}

static sird_status forecast_impl(const sird_problem* pb, const double* theta, int k, int horizon, double* out_D,
                                 int precision, void* cuda_stream) {
    std::string why;
    sird_status st = sird_check_problem(pb, why);
    if (st != SIRD_OK) return g_create_error = why, st;
    if (!theta || !out_D || k < 1 || k > SIRD_MAX_PARTICLES || horizon < 1 || horizon > 100000)
        return g_create_error = "forecast: bad theta/out_D/k/horizon", SIRD_ERR_ARG;
    if (precision != 32 && precision != 64) return g_create_error = "forecast: precision must be 32 or 64", SIRD_ERR_ARG;
    WindowDev w{};
    ModelDev m{};
    sird_fill_window(pb, w, m);
    const int P = m.P;
    const size_t tsz = precision == 32 ? 4 : 8;
    const size_t th_bytes = (size_t)P * k * tsz, out_bytes = (size_t)k * horizon * tsz;
    const size_t y_bytes = precision == 32 ? (size_t)pb->n_obs * sizeof(float) : 0;
    std::vector<unsigned char> hth(th_bytes + y_bytes), hout(out_bytes);
    for (size_t i = 0; i < y_bytes / sizeof(float); ++i)  // the FP32 trajectory follows y_D's float values
        ((float*)(hth.data() + th_bytes))[i] = (float)pb->y_D[i];
    for (int j = 0; j < k; ++j)
        for (int d = 0; d < P; ++d) {
            const double v = theta[(size_t)j * P + d];
            if (precision == 32) ((float*)hth.data())[(size_t)d * k + j] = (float)v;
            else ((double*)hth.data())[(size_t)d * k + j] = v;
        }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void* dmem = nullptr;
    // device: theta | observations (FP32) | forecast
    cudaError_t e = cudaMalloc(&dmem, th_bytes + y_bytes + out_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmem, hth.data(), th_bytes + y_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_forecast(w, m, dmem, k, k, horizon, (const float*)((unsigned char*)dmem + th_bytes),
                            (unsigned char*)dmem + th_bytes + y_bytes, precision, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout.data(), (unsigned char*)dmem + th_bytes + y_bytes, out_bytes,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dmem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        g_create_error = std::string("forecast: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SIRD_ERR_NOMEM : SIRD_ERR_CUDA;
    }
    for (size_t i = 0; i < (size_t)k * horizon; ++i)
        out_D[i] = precision == 32 ? (double)((float*)hout.data())[i] : ((double*)hout.data())[i];
    return SIRD_OK;
}

extern "C" sird_status sird_forecast(const sird_problem* pb, const double* theta, int k, int horizon, double* out_D,
                                     int precision, void* cuda_stream) {
    TraceRange trace("sird_forecast");
    try {  // the host copies scale with k and horizon: a failed allocation is reported, not thrown
        return forecast_impl(pb, theta, k, horizon, out_D, precision, cuda_stream);
    } catch (const std::bad_alloc&) {
        return g_create_error = "forecast: host allocation failed", SIRD_ERR_NOMEM;
    }
}

// Values left out at each end of k sorted ones by the central band holding each fraction:
// floor(k (1 - f) / 2) (the small offset keeps e.g. k = 1000, f = 0.9 at exactly 50).  False on a
// fraction outside (0, 1].
static bool band_drops(int k, const double* fractions, int n_bands, std::vector<int>& drop) {
    drop.assign(n_bands > 0 ? n_bands : 1, 0);
    for (int b = 0; b < n_bands; ++b) {
        const double f = fractions[b];
        if (!(f > 0.0 && f <= 1.0)) return false;
        drop[b] = (int)std::floor((double)k * (1.0 - f) / 2.0 + 1e-9);
    }
    return true;
}

static sird_status ensemble_bands_impl(const sird_problem* pb, const double* theta, int k, int horizon,
                                       const double* fractions, int n_bands, double* out, void* cuda_stream) {
    std::string why;
    sird_status st = sird_check_problem(pb, why);
    if (st != SIRD_OK) return g_create_error = why, st;
    if (!theta || !out || k < 1 || k > kMaxEnsemble || horizon < 0 || horizon > 100000 || n_bands < 0 ||
        n_bands > 16 || (n_bands > 0 && !fractions))
        return g_create_error = "ensemble_bands: bad theta/out/k/horizon/bands", SIRD_ERR_ARG;
    std::vector<int> drop;
    if (!band_drops(k, fractions, n_bands, drop))
        return g_create_error = "ensemble_bands: fractions must be in (0, 1]", SIRD_ERR_ARG;
    WindowDev w{};
    ModelDev m{};
    sird_fill_window(pb, w, m);
    const int P = m.P, n_days = pb->n_obs + horizon, nq = 1 + 2 * n_bands;
    for (size_t i = 0; i < (size_t)k * P; ++i)
        if (!std::isfinite(theta[i])) return g_create_error = "ensemble_bands: non-finite theta", SIRD_ERR_ARG;
    const size_t th_bytes = (size_t)P * k * sizeof(double), drop_bytes = 256;
    const size_t traj_bytes = ensemble_traj_bytes(k, n_days);
    const size_t out_count = (size_t)kBandQuantities * n_days * nq;
    std::vector<double> hth((size_t)P * k);
    for (int j = 0; j < k; ++j)
        for (int d = 0; d < P; ++d) hth[(size_t)d * k + j] = theta[(size_t)j * P + d];
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* dmem = nullptr;
    cudaError_t e = cudaMalloc((void**)&dmem, th_bytes + drop_bytes + traj_bytes + out_count * sizeof(double));
    double* dth = (double*)dmem;
    int* ddrop = (int*)(dmem + th_bytes);
    double* dtraj = (double*)(dmem + th_bytes + drop_bytes);
    double* dout = (double*)(dmem + th_bytes + drop_bytes + traj_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dth, hth.data(), th_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ddrop, drop.data(), sizeof(int) * drop.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_ensemble_bands(w, m, dth, k, n_days, ddrop, n_bands, dtraj, dout, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, out_count * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dmem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        g_create_error = std::string("ensemble_bands: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SIRD_ERR_NOMEM : SIRD_ERR_CUDA;
    }
    return SIRD_OK;
}

extern "C" sird_status sird_ensemble_bands(const sird_problem* pb, const double* theta, int k, int horizon,
                                           const double* fractions, int n_bands, double* out, void* cuda_stream) {
    TraceRange trace("sird_ensemble_bands");
    try {
        return ensemble_bands_impl(pb, theta, k, horizon, fractions, n_bands, out, cuda_stream);
    } catch (const std::bad_alloc&) {
        return g_create_error = "ensemble_bands: host allocation failed", SIRD_ERR_NOMEM;
    }
}

static sird_status parameter_bands_impl(const sird_problem* pb, const double* theta, int k, const double* fractions,
                                        int n_bands, double* out, void* cuda_stream) {
    std::string why;
    sird_status st = sird_check_problem(pb, why);
    if (st != SIRD_OK) return g_create_error = why, st;
    if (!theta || !out || k < 1 || k > kMaxEnsemble || n_bands < 0 || n_bands > 16 || (n_bands > 0 && !fractions))
        return g_create_error = "parameter_bands: bad theta/out/k/bands", SIRD_ERR_ARG;
    std::vector<int> drop;
    if (!band_drops(k, fractions, n_bands, drop))
        return g_create_error = "parameter_bands: fractions must be in (0, 1]", SIRD_ERR_ARG;
    WindowDev w{};
    ModelDev m{};
    sird_fill_window(pb, w, m);
    const int P = m.P, nq = 1 + 2 * n_bands;
    for (size_t i = 0; i < (size_t)k * P; ++i)
        if (!std::isfinite(theta[i])) return g_create_error = "parameter_bands: non-finite theta", SIRD_ERR_ARG;
    const size_t th_bytes = ((size_t)P * k * sizeof(double) + 255) & ~(size_t)255, drop_bytes = 256;
    const size_t out_count = (size_t)P * nq;
    std::vector<double> hth((size_t)P * k);
    for (int j = 0; j < k; ++j)
        for (int d = 0; d < P; ++d) hth[(size_t)d * k + j] = theta[(size_t)j * P + d];
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* dmem = nullptr;
    cudaError_t e = cudaMalloc((void**)&dmem, th_bytes + drop_bytes + out_count * sizeof(double));
    double* dth = (double*)dmem;
    int* ddrop = (int*)(dmem + th_bytes);
    double* dout = (double*)(dmem + th_bytes + drop_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dth, hth.data(), (size_t)P * k * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ddrop, drop.data(), sizeof(int) * drop.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_parameter_bands(m, dth, k, ddrop, n_bands, dout, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, out_count * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dmem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        g_create_error = std::string("parameter_bands: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SIRD_ERR_NOMEM : SIRD_ERR_CUDA;
    }
    return SIRD_OK;
}

extern "C" sird_status sird_parameter_bands(const sird_problem* pb, const double* theta, int k,
                                            const double* fractions, int n_bands, double* out, void* cuda_stream) {
    TraceRange trace("sird_parameter_bands");
    try {
        return parameter_bands_impl(pb, theta, k, fractions, n_bands, out, cuda_stream);
    } catch (const std::bad_alloc&) {
        return g_create_error = "parameter_bands: host allocation failed", SIRD_ERR_NOMEM;
    }
}

static sird_status topk_impl(sird_pso_t h, int k, double* theta_out, double* loss_out, int* index_out);

extern "C" sird_status sird_pso_topk(sird_pso_t h, int k, double* theta_out, double* loss_out) {
    return topk_impl(h, k, theta_out, loss_out, nullptr);
}

extern "C" sird_status sird_pso_topk_indexed(sird_pso_t h, int k, double* theta_out, double* loss_out,
                                             int* index_out) {
    if (h && !h->sticky && !index_out) return h->fail(SIRD_ERR_ARG, "topk_indexed: index_out is NULL");
    return topk_impl(h, k, theta_out, loss_out, index_out);
}

static sird_status topk_impl(sird_pso_t h, int k, double* theta_out, double* loss_out, int* index_out) {
    TraceRange trace("sird_pso_topk");
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->precision != 32) return h->fail(SIRD_ERR_UNSUPPORTED, "topk: FP32 swarms only");
    if (k < 1 || k > 2048 || k > h->M || !theta_out || !loss_out) return h->fail(SIRD_ERR_ARG, "topk: bad k or outputs");
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "topk before init");
    const size_t nk = topk_scratch_keys(h->M, k);
    const size_t bytes = 2 * nk * sizeof(unsigned long long) + (size_t)k * (h->P + 1) * sizeof(double);
    void* dmem = nullptr;
    sird_status st = h->cuda(cudaMalloc(&dmem, bytes), "topk scratch");
    if (st) return st;
    unsigned long long* a = (unsigned long long*)dmem;
    unsigned long long* b = a + nk;
    double* dth = (double*)(b + nk);
    double* dloss = dth + (size_t)k * h->P;
    unsigned long long* keys = nullptr;
    cudaError_t e = launch_topk_f32((const float*)h->pbf, h->M, k, a, b, &keys, h->stream);
    if (e == cudaSuccess)
        e = launch_topk_gather(keys, k, (const float*)h->pb, (const float*)h->pbf, h->ld, h->P, h->c32.logmask, dth,
                               dloss, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(theta_out, dth, (size_t)k * h->P * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss_out, dloss, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    std::vector<unsigned long long> hk(index_out ? (size_t)k : 0);
    if (e == cudaSuccess && index_out)
        e = cudaMemcpyAsync(hk.data(), keys, (size_t)k * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dmem);
    if (e == cudaSuccess && index_out)
        for (int j = 0; j < k; ++j) index_out[j] = (int)((hk[j] & 0xFFFFFFFFu) + h->c32.p_off);
    return h->cuda(e, "topk");
}

// ---------------------------------------------------------------- sharded swarm

extern "C" sird_status sird_pso_set_shard(sird_pso_t h, int offset, int total) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (h->precision != 32) return h->fail(SIRD_ERR_UNSUPPORTED, "set_shard: FP32 swarms only");
    if (h->iter >= 0) return h->fail(SIRD_ERR_STATE, "set_shard: before init");
    if (offset < 0 || total < 1 || total > SIRD_MAX_PARTICLES || (long long)offset + h->M > (long long)total)
        return h->fail(SIRD_ERR_ARG, "set_shard: particles offset .. offset + M - 1 must lie in 0 .. total - 1");
    h->c32.p_off = (uint32_t)offset;
    h->shard_total = total;
    h->persistent = h->cluster = false;  // one launch per iteration: the global best is exchanged between them
    return SIRD_OK;
}

extern "C" sird_status sird_pso_shard_best(sird_pso_t h, float* loss, int* index, float* z) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (!loss || !index || !z) return h->fail(SIRD_ERR_ARG, "shard_best: NULL output");
    if (h->precision != 32) return h->fail(SIRD_ERR_UNSUPPORTED, "shard_best: FP32 swarms only");
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "shard_best before init");
    cudaError_t e = cudaMemcpyAsync(loss, h->red.gbest_f, sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(index, h->red.gbest_idx, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, h->gbest, (size_t)h->P * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return h->cuda(e, "shard_best");
}

extern "C" sird_status sird_pso_set_gbest(sird_pso_t h, const float* z, float loss, int index) {
    if (!h) return SIRD_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (!z) return h->fail(SIRD_ERR_ARG, "set_gbest: z is NULL");
    if (h->precision != 32) return h->fail(SIRD_ERR_UNSUPPORTED, "set_gbest: FP32 swarms only");
    if (h->iter < 0) return h->fail(SIRD_ERR_STATE, "set_gbest before init");
    const int total = h->shard_total > 0 ? h->shard_total : h->M;
    if (index < 0 || index >= total) return h->fail(SIRD_ERR_ARG, "set_gbest: index out of range");
    for (int d = 0; d < h->P; ++d)
        if (!(z[d] >= h->c32.zlb[d] && z[d] <= h->c32.zub[d]))
            return h->fail(SIRD_ERR_ARG, "set_gbest: position outside the search box");
    // host copies first, then the device; the stream orders them before the next iteration
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h->gbest, z, (size_t)h->P * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->red.gbest_f, &loss, sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->red.gbest_idx, &index, sizeof(int), cudaMemcpyHostToDevice);
    return h->cuda(e, "set_gbest");
}

