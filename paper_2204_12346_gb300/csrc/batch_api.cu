// batch_api.cu -- C ABI of the batched calibration (many rolling windows, one launch).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/sird_pso.h"
#include "kernels.h"
#include "trace.h"

using namespace sird;

sird_status sird_check_problem(const sird_problem* pb, std::string& why);
void sird_fill_window(const sird_problem* pb, WindowDev& w, ModelDev& m);

struct sird_batch {
    int W = 0, P = 0, iters = 0, n_max = 0, block = 0, grid = 0, per_sm = 0;  // per_sm 0 = occupancy maximum
    int flat = 0;  // 1: the flat form (every swarm spread over the grid, one grid barrier per iteration)
    int n_items = 0;
    int4* items = nullptr;   // flat form: (window, particle, partner or -1), windows longest first
    int* n_items_w = nullptr;
    FlatScratch fs{};
    ModelDev mdl{};
    PsoCoeffs<float> c{};
    cudaStream_t stream = nullptr, cap = nullptr;
    void* d_mem = nullptr;
    BatchWindow* wins = nullptr;
    int* order = nullptr;
    float *yf = nullptr, *invy = nullptr, *swarm = nullptr;
    double* yd = nullptr;
    unsigned* queue = nullptr;
    BatchOut* out = nullptr;
    BatchOut* h_out = nullptr;  // pinned
    std::vector<double> ss_tot;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // optional timing events around the batch kernel
    std::string msg;
    // for sird_batch_set_observations: the windows' settings, their device images and a pinned
    // staging copy of [windows | observations] laid out like the device memory
    std::vector<sird_problem> probs;
    std::vector<BatchWindow> h_wins;
    std::vector<int> obs_off;
    size_t nobs = 0, wins_bytes = 0, obs_bytes = 0;
    unsigned char* h_stage = nullptr;
    cudaEvent_t ev_upload = nullptr;
    // polish (sird_batch_polish): the FP64 box, a calibration done, the device scratch (window
    // table | keys | polish state | checkpoints | results) and the pinned results
    PsoCoeffs<double> c64{};
    bool calibrated = false;
    void* pmem = nullptr;
    size_t pmem_bytes = 0;
    ResultDev* h_pres = nullptr;
};

namespace {

thread_local std::string g_batch_error;

sird_status berr(sird_status s, const std::string& m) {
    g_batch_error = m;
    set_global_error(m.c_str());
    return s;
}

// Optional on-disk cache of tuned block sizes: file named by SIRD_TUNE_CACHE, lines "key block".
std::string tune_key(const sird_batch* b, long long work) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|W%d|P%d|spd%d|K%d|cost%d|iters%d|work%lld|n%d", prop.name, b->W, b->P,
                  b->mdl.spd, b->mdl.K, b->mdl.cost, b->iters, work, b->n_max);
    std::string k(buf);
    for (char& ch : k)
        if (ch == ' ') ch = '_';
    return k;
}

int tune_cache_get(const std::string& key) {
    const char* path = std::getenv("SIRD_TUNE_CACHE");
    if (!path) return 0;
    FILE* f = std::fopen(path, "r");
    if (!f) return 0;
    char k[512];
    int v = 0, found = 0;
    while (std::fscanf(f, "%511s %d", k, &v) == 2)
        if (key == k) found = v;
    std::fclose(f);
    return found;
}

void tune_cache_put(const std::string& key, int block) {
    const char* path = std::getenv("SIRD_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), block);
    std::fclose(f);
}

cudaError_t run(sird_batch* b, int iters, int block, int per_sm, int flat, cudaStream_t s, bool reeval,
                bool timed = false) {
    int per = flat ? flat_blocks_per_sm(b->mdl, block) : batch_blocks_per_sm(b->mdl, block, b->n_max);
    if (per <= 0) return cudaErrorInvalidConfiguration;
    if (per_sm > 0 && per_sm < per) per = per_sm;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // the flat form needs every block resident at once (it waits at a grid barrier)
    const int grid = flat ? per * nsm : std::min(b->W, per * nsm);
    b->grid = grid;
    cudaError_t e = cudaSuccess;
    if (timed && b->ev_begin) e = cudaEventRecordWithFlags(b->ev_begin, s, cudaEventRecordExternal);
    if (e == cudaSuccess) {
        if (flat)
            e = launch_flat(b->wins, b->n_items_w, b->items, b->n_items, b->W, b->mdl, b->c, b->yf, b->invy,
                            b->swarm, b->fs, b->out, iters, block, grid, s);
        else
            e = launch_batch(b->wins, b->order, b->W, b->mdl, b->c, b->yf, b->invy, b->yd, b->swarm, b->queue,
                             b->out, iters, b->n_max, block, grid, false, s);
    }
    if (e == cudaSuccess && timed && b->ev_end) e = cudaEventRecordWithFlags(b->ev_end, s, cudaEventRecordExternal);
    if (e == cudaSuccess && reeval)
        e = launch_batch_reeval(b->wins, b->W, b->mdl, b->c.logmask, b->yd, b->out, s);
    return e;
}

// Times short trial runs (up to 8 iterations) of each candidate (form, threads per block, blocks
// per SM) and keeps the fastest.  One block per SM gives a long window a whole SM; more blocks per SM
// hide latency better when windows are short.
cudaError_t autotune(sird_batch* b, long long work) {
    const std::string key = tune_key(b, work);
    const int cached = tune_cache_get(key);
    if (cached) {
        b->block = cached & 0xFFFF;
        b->per_sm = (cached >> 16) & 0xFF;
        b->flat = (cached >> 24) & 1;
        return cudaSuccess;
    }
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    int best_block = 128, best_per = 0, best_flat = 0;
    // long enough that the balance of windows over blocks and the per-iteration costs weigh as
    // in the full run (two iterations favoured shapes that lose over a hundred)
    const int trial_iters = std::min(b->iters, 8);
    const char* vv = std::getenv("SIRD_TUNE_VERBOSE");  // candidate timings to stderr when set
    const bool verbose = vv && *vv && *vv != '0';
    for (int flat = 0; flat < 2 && e == cudaSuccess; ++flat) {
        for (int block : {128, 256, 384, 512, 640, 768, 1024}) {
            const int maxper = flat ? flat_blocks_per_sm(b->mdl, block) : batch_blocks_per_sm(b->mdl, block, b->n_max);
            for (int ci = 0; ci < 3; ++ci) {
                // each distinct (block, blocks per SM) that fits, once: 1, 2 and the maximum
                const int per = ci == 0 ? 1 : (ci == 1 ? 2 : maxper);
                if (maxper <= 0 || per > maxper || (ci == 2 && maxper <= 2)) continue;
                float ms = 0.f;
                for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms up
                    e = cudaEventRecord(e0, b->stream);
                    if (e == cudaSuccess) e = run(b, trial_iters, block, per, flat, b->stream, false);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                }
                if (e != cudaSuccess) break;
                if (verbose)
                    std::fprintf(stderr, "sird batch autotune: %s, %d threads x %d per SM: %.3f ms\n",
                                 flat ? "flat" : "one window per block", block, per, ms);
                if (ms < best) {
                    best = ms;
                    best_block = block;
                    best_per = per;
                    best_flat = flat;
                }
            }
            if (e != cudaSuccess) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    b->block = best_block;
    b->per_sm = best_per;
    b->flat = best_flat;
    tune_cache_put(key, best_block | (best_per << 16) | (best_flat << 24));
    return cudaSuccess;
}

}  // namespace

namespace {

sird_status batch_create(int W, const sird_problem* problems, const sird_pso_config* configs, void* cuda_stream,
                         sird_batch_t* out) {
    if (!out) return berr(SIRD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (W < 1 || W > (1 << 20) || !problems || !configs) return berr(SIRD_ERR_ARG, "bad W or NULL arrays");
    const sird_problem& p0 = problems[0];
    const sird_pso_config& c0 = configs[0];
    std::string why;
    long long all_particles = 0;
    for (int i = 0; i < W; ++i) {
        const sird_problem& p = problems[i];
        const sird_pso_config& c = configs[i];
        sird_status st = sird_check_problem(&p, why);
        if (st != SIRD_OK) return berr(st, "window " + std::to_string(i) + ": " + why);
        if (p.beta_form != p0.beta_form || p.K != p0.K || p.steps_per_day != p0.steps_per_day || p.cost != p0.cost ||
            p.objective != p0.objective || p.fit_I0 != p0.fit_I0)
            return berr(SIRD_ERR_ARG, "window " + std::to_string(i) + ": model settings differ from window 0");
        if (c.precision != 32) return berr(SIRD_ERR_UNSUPPORTED, "batched calibration is FP32 only");
        if (c.particles < 1 || c.particles > (1 << 20))
            return berr(SIRD_ERR_ARG, "particles per window out of range [1, 2^20]");
        all_particles += c.particles;
        if (c.iters != c0.iters || c.w != c0.w || c.c1 != c0.c1 || c.c2 != c0.c2 || c.iters < 0)
            return berr(SIRD_ERR_ARG, "window " + std::to_string(i) + ": PSO coefficients or iterations differ");
        if (!c.lb || !c.ub) return berr(SIRD_ERR_ARG, "lb/ub is NULL");
    }
    if (all_particles > SIRD_MAX_PARTICLES)
        return berr(SIRD_ERR_ARG, "more than SIRD_MAX_PARTICLES particles over all windows");
    const int P = (p0.beta_form == SIRD_BETA_RAMP ? 6 : p0.K + 2) + (p0.fit_I0 ? 1 : 0);
    for (int i = 0; i < W; ++i)
        for (int d = 0; d < P; ++d) {
            const bool lg = configs[i].log_scale && configs[i].log_scale[d];
            const bool lg0 = c0.log_scale && c0.log_scale[d];
            if (configs[i].lb[d] != c0.lb[d] || configs[i].ub[d] != c0.ub[d] || lg != lg0)
                return berr(SIRD_ERR_ARG, "window " + std::to_string(i) + ": bounds differ from window 0");
        }
    if (c0.block_size != 0 && (c0.block_size < 32 || c0.block_size > 1024 || c0.block_size % 32))
        return berr(SIRD_ERR_ARG, "block_size must be 0 (autotune) or a multiple of 32 in [32, 1024]");

    // owned by the guard until the batch is complete: every early return (and a failed host
    // allocation, thrown as std::bad_alloc) releases what was allocated
    std::unique_ptr<sird_batch, void (*)(sird_batch*)> guard(new (std::nothrow) sird_batch(), sird_batch_destroy);
    sird_batch* b = guard.get();
    if (!b) return berr(SIRD_ERR_NOMEM, "host allocation failed");
    b->W = W;
    b->P = P;
    b->iters = c0.iters;
    b->stream = (cudaStream_t)cuda_stream;
    std::vector<BatchWindow> wins(W);
    std::vector<int> obs_off(W + 1, 0);
    long long sw_total = 0, work = 0;
    for (int i = 0; i < W; ++i) {
        ModelDev m{};
        sird_fill_window(&problems[i], wins[i].w, m);
        if (i == 0) b->mdl = m;
        // the window's series stacked D | I | R (F_IRD) with stride obs_stride(n_obs)
        obs_off[i + 1] = obs_off[i] + (p0.objective == SIRD_FIT_IRD ? 3 : 1) * obs_stride(problems[i].n_obs);
        wins[i].obs_off = obs_off[i];
        wins[i].M = configs[i].particles;
        wins[i].ld = (configs[i].particles + 31) & ~31;
        wins[i].sw_off = sw_total;
        wins[i].key0 = (uint32_t)configs[i].seed;
        wins[i].key1 = (uint32_t)(configs[i].seed >> 32);
        wins[i].stream_id = configs[i].stream_id;
        sw_total += (long long)(3 * P + 1) * wins[i].ld;
        b->n_max = std::max(b->n_max, problems[i].n_obs);
        work += (long long)configs[i].particles * (problems[i].n_obs - 1);
    }
    // longest first, so the last windows taken from the queue are short
    std::vector<int> order(W);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)wins[a].M * (wins[a].w.n_obs - 1) > (long long)wins[c].M * (wins[c].w.n_obs - 1);
    });
    for (int d = 0; d < P; ++d) {
        const bool lg = c0.log_scale && c0.log_scale[d];
        if (lg && !(c0.lb[d] > 0)) return berr(SIRD_ERR_ARG, "log_scale needs lb > 0");
        if (lg) b->c.logmask |= 1u << d;
        const double zl = lg ? std::log(c0.lb[d]) : c0.lb[d];
        const double zu = lg ? std::log(c0.ub[d]) : c0.ub[d];
        b->c.zlb[d] = (float)zl;
        b->c.zub[d] = (float)zu;
        b->c64.zlb[d] = zl;
        b->c64.zub[d] = zu;
    }
    b->c64.logmask = b->c.logmask;
    b->c64.w = c0.w;
    b->c64.c1 = c0.c1;
    b->c64.c2 = c0.c2;
    b->c.w = (float)c0.w;
    b->c.c1 = (float)c0.c1;
    b->c.c2 = (float)c0.c2;
    b->ss_tot.resize(W);
    const size_t nobs = (size_t)obs_off[W];
    std::vector<float> yf(nobs, 0.f), invy(nobs, 0.f);
    std::vector<double> yd(nobs, 0.0);
    for (int i = 0; i < W; ++i) {
        const sird_problem& p = problems[i];
        double mean = 0.0;
        for (int j = 0; j < p.n_obs; ++j) {
            yf[obs_off[i] + j] = obs_f32(p.y_D, j, true);
            invy[obs_off[i] + j] = p.y_D[j] != 0.0 ? (float)(1.0 / p.y_D[j]) : 0.f;
            yd[obs_off[i] + j] = p.y_D[j];
            if (p.objective == SIRD_FIT_IRD) {
                const int ps = obs_stride(p.n_obs);
                const double* ir[2] = {p.y_I, p.y_R};
                for (int k = 0; k < 2; ++k) {
                    const int o = obs_off[i] + (k + 1) * ps + j;
                    yf[o] = obs_f32(ir[k], j, k == 1);
                    invy[o] = ir[k][j] != 0.0 ? (float)(1.0 / ir[k][j]) : 0.f;
                    yd[o] = ir[k][j];
                }
            }
            mean += p.y_D[j];
        }
        mean /= p.n_obs;
        double ss = 0.0;
        for (int j = 0; j < p.n_obs; ++j) ss += (p.y_D[j] - mean) * (p.y_D[j] - mean);
        b->ss_tot[i] = ss;
    }
    // flat form: particle pairs of every window, windows longest first (the items a thread owns,
    // i, i + T, ..., then fall on windows of similar length), pairs (2q, 2q + 1), a last single
    std::vector<int> by_len(W);
    std::iota(by_len.begin(), by_len.end(), 0);
    std::stable_sort(by_len.begin(), by_len.end(), [&](int a, int c) { return wins[a].w.n_obs > wins[c].w.n_obs; });
    std::vector<int4> items;
    std::vector<int> n_items_w(W, 0);
    for (int wi : by_len) {
        const int M = wins[wi].M;
        for (int q = 0; 2 * q < M; ++q) items.push_back(make_int4(wi, 2 * q, 2 * q + 1 < M ? 2 * q + 1 : -1, 0));
        n_items_w[wi] = (M + 1) / 2;
    }
    b->n_items = (int)items.size();
    auto r256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t bytes = r256(sizeof(BatchWindow) * W) + r256(sizeof(int) * W) + 2 * r256(nobs * sizeof(float)) +
                         r256(nobs * sizeof(double)) + r256(256) + r256(sizeof(BatchOut) * W) +
                         r256((size_t)sw_total * sizeof(float)) + r256(sizeof(int4) * items.size()) +
                         r256(sizeof(int) * W) + r256(sizeof(unsigned long long) * W) + r256(sizeof(unsigned) * W) +
                         r256(sizeof(float) * kMaxParams * W) + r256(256);
    cudaError_t e = cudaMalloc(&b->d_mem, bytes);
    auto bail = [&](cudaError_t err, const char* what) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(err);
        (void)cudaGetLastError();
        guard.reset();
        return berr(err == cudaErrorMemoryAllocation ? SIRD_ERR_NOMEM : SIRD_ERR_CUDA, m);
    };
    if (e != cudaSuccess) return bail(e, "allocating the batch");
    unsigned char* q = (unsigned char*)b->d_mem;
    auto take = [&](size_t n) {
        unsigned char* r = q;
        q += (n + 255) & ~(size_t)255;
        return r;
    };
    b->wins = (BatchWindow*)take(sizeof(BatchWindow) * W);
    b->order = (int*)take(sizeof(int) * W);
    b->yf = (float*)take(nobs * sizeof(float));
    b->invy = (float*)take(nobs * sizeof(float));
    b->yd = (double*)take(nobs * sizeof(double));
    b->queue = (unsigned*)take(256);
    b->out = (BatchOut*)take(sizeof(BatchOut) * W);
    b->swarm = (float*)take((size_t)sw_total * sizeof(float));
    b->items = (int4*)take(sizeof(int4) * items.size());
    b->n_items_w = (int*)take(sizeof(int) * W);
    b->fs.gkey = (unsigned long long*)take(sizeof(unsigned long long) * W);
    b->fs.done = (unsigned*)take(sizeof(unsigned) * W);
    b->fs.gpos = (float*)take(sizeof(float) * kMaxParams * W);
    unsigned* words = (unsigned*)take(256);
    b->fs.bar_count = words;
    b->fs.bar_gen = words + 1;
    b->fs.err = words + 2;
    b->fs.abort = words + 3;
    if ((size_t)(q - (unsigned char*)b->d_mem) > bytes) return bail(cudaErrorInvalidValue, "batch layout");
    e = cudaMemcpyAsync(b->wins, wins.data(), sizeof(BatchWindow) * W, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->order, order.data(), sizeof(int) * W, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->yf, yf.data(), nobs * sizeof(float), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->invy, invy.data(), nobs * sizeof(float), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->yd, yd.data(), nobs * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->n_items_w, n_items_w.data(), sizeof(int) * W, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, 256, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bail(e, "uploading the batch");
    e = cudaMallocHost((void**)&b->h_out, sizeof(BatchOut) * W);
    if (e != cudaSuccess) return bail(e, "allocating pinned results");
    b->probs.assign(problems, problems + W);
    for (auto& pr : b->probs) pr.y_D = nullptr;
    b->h_wins = wins;
    b->obs_off = obs_off;
    b->nobs = nobs;
    b->wins_bytes = sizeof(BatchWindow) * W;
    b->obs_bytes = (size_t)((unsigned char*)(b->yd + nobs) - (unsigned char*)b->yf);
    if (c0.block_size) {
        b->block = c0.block_size;
        b->flat = c0.launch_mode == SIRD_LAUNCH_FLAT ? 1 : 0;
        if (b->flat && flat_blocks_per_sm(b->mdl, b->block) <= 0)
            return berr(SIRD_ERR_ARG, "block_size does not fit the flat form");
        if (!b->flat && batch_blocks_per_sm(b->mdl, b->block, b->n_max) <= 0)
            return berr(SIRD_ERR_ARG, "block_size does not fit the batched kernel of this form (its launch bound)");
    } else {
        e = autotune(b, work);
        if (e != cudaSuccess) return bail(e, "autotuning");
    }
    *out = guard.release();
    return SIRD_OK;
}

}  // namespace

extern "C" sird_status sird_batch_create(int W, const sird_problem* problems, const sird_pso_config* configs,
                                         void* cuda_stream, sird_batch_t* out) {
    TraceRange trace("sird_batch_create");
    try {  // no exception crosses the C ABI
        return batch_create(W, problems, configs, cuda_stream, out);
    } catch (const std::bad_alloc&) {
        return berr(SIRD_ERR_NOMEM, "host allocation failed");
    }
}

extern "C" void sird_batch_destroy(sird_batch_t b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_mem);
    if (b->h_out) cudaFreeHost(b->h_out);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->ev_upload) cudaEventDestroy(b->ev_upload);
    if (b->pmem) cudaFree(b->pmem);
    if (b->h_pres) cudaFreeHost(b->h_pres);
    delete b;
}

extern "C" int sird_batch_block_size(sird_batch_t b) { return b ? b->block : 0; }

extern "C" sird_status sird_batch_set_timing(sird_batch_t b, void* event_begin, void* event_end) {
    if (!b) return berr(SIRD_ERR_ARG, "batch is NULL");
    b->ev_begin = (cudaEvent_t)event_begin;
    b->ev_end = (cudaEvent_t)event_end;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return SIRD_OK;
}

extern "C" int sird_batch_launch_mode(sird_batch_t b) {
    return b ? (b->flat ? SIRD_LAUNCH_FLAT : SIRD_LAUNCH_WINDOW_PER_BLOCK) : 0;
}

extern "C" int sird_batch_blocks_per_sm(sird_batch_t b) {
    if (!b) return 0;
    const int maxper = b->flat ? flat_blocks_per_sm(b->mdl, b->block) : batch_blocks_per_sm(b->mdl, b->block, b->n_max);
    return (b->per_sm > 0 && b->per_sm < maxper) ? b->per_sm : maxper;
}

extern "C" sird_status sird_batch_calibrate(sird_batch_t b, sird_result* results) {
    TraceRange trace("sird_batch_calibrate");
    if (!b || !results) return berr(SIRD_ERR_ARG, "batch or results is NULL");
    cudaError_t e = cudaSuccess;
    if (!b->graph) {
        if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        cudaGraph_t g = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = run(b, b->iters, b->block, b->per_sm, b->flat, b->cap, true, true);
            if (e1 == cudaSuccess)
                e1 = cudaMemcpyAsync(b->h_out, b->out, sizeof(BatchOut) * b->W, cudaMemcpyDeviceToHost, b->cap);
            e = cudaStreamEndCapture(b->cap, &g);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return berr(SIRD_ERR_CUDA, std::string("capturing the batch graph: ") + cudaGetErrorString(e));
        }
    }
    e = cudaGraphLaunch(b->graph, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return berr(SIRD_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    }
    if (b->flat) {
        unsigned err = 0;
        e = cudaMemcpy(&err, b->fs.err, sizeof(err), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return berr(SIRD_ERR_CUDA, std::string("reading the error word: ") + cudaGetErrorString(e));
        if (err & kErrTimeout) return berr(SIRD_ERR_TIMEOUT, "a grid barrier wait ran out");
    }
    for (int i = 0; i < b->W; ++i) {
        sird_result& r = results[i];
        std::memset(&r, 0, sizeof(r));
        r.n_params = b->P;
        for (int d = 0; d < b->P; ++d) r.theta[d] = b->h_out[i].theta[d];
        r.loss = b->h_out[i].loss64;
        r.loss_search = (double)b->h_out[i].loss;
        r.r2_D = b->ss_tot[i] > 0 ? 1.0 - b->h_out[i].sse / b->ss_tot[i] : NAN;
        r.index = b->h_out[i].index;
        r.iters_done = b->iters;
    }
    b->calibrated = true;
    return SIRD_OK;
}

extern "C" sird_status sird_batch_polish(sird_batch_t b, int k, int iters, double first_step, sird_result* results) {
    TraceRange trace("sird_batch_polish");
    if (!b || !results) return berr(SIRD_ERR_ARG, "batch or results is NULL");
    if (b->mdl.spd != 10 && b->mdl.spd != 20 && b->mdl.spd > 64)
        return berr(SIRD_ERR_UNSUPPORTED, "polish: FP32 needs steps_per_day <= 64");
    if (b->W > 65535) return berr(SIRD_ERR_UNSUPPORTED, "polish: at most 65535 windows");
    if (!b->calibrated) return berr(SIRD_ERR_STATE, "polish before the first sird_batch_calibrate");
    int m_min = INT32_MAX;
    for (const auto& hw : b->h_wins) m_min = std::min(m_min, hw.M);
    if (k < 1 || k > kTopkTabMax || k > m_min || iters < 0 || !(first_step > 0))
        return berr(SIRD_ERR_ARG, "polish: bad k (1..min(1024, smallest swarm)), iters or first_step");
    const int W = b->W, P = b->P;
    auto r256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t tab_b = r256(sizeof(PolishWin) * W), keys_b = r256(sizeof(unsigned long long) * W * (size_t)k),
                 st_b = r256(polish_scratch_doubles(P, W * k) * sizeof(double)),
                 ck_b = r256(polish_ckpt_floats(b->n_max, k, b->mdl) * sizeof(float) * W),
                 res_b = r256(sizeof(ResultDev) * W);
    const size_t need = tab_b + keys_b + st_b + ck_b + res_b;
    cudaError_t e = cudaSuccess;
    if (b->pmem_bytes < need) {
        if (b->pmem) {
            e = cudaStreamSynchronize(b->stream);
            cudaFree(b->pmem);
            b->pmem = nullptr;
            b->pmem_bytes = 0;
        }
        if (e == cudaSuccess) e = cudaMalloc(&b->pmem, need);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            b->pmem = nullptr;
            return berr(e == cudaErrorMemoryAllocation ? SIRD_ERR_NOMEM : SIRD_ERR_CUDA,
                        std::string("polish scratch: ") + cudaGetErrorString(e));
        }
        b->pmem_bytes = need;
    }
    if (!b->h_pres) {
        e = cudaMallocHost((void**)&b->h_pres, sizeof(ResultDev) * W);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            b->h_pres = nullptr;
            return berr(SIRD_ERR_NOMEM, "polish: pinned results");
        }
    }
    unsigned char* q = (unsigned char*)b->pmem;
    PolishWin* tab = (PolishWin*)q;
    unsigned long long* keys = (unsigned long long*)(q + tab_b);
    double* scratch = (double*)(q + tab_b + keys_b);
    float* ckpt = (float*)(q + tab_b + keys_b + st_b);
    ResultDev* res = (ResultDev*)(q + tab_b + keys_b + st_b + ck_b);
    // the window table: each window's constants (as the last set_observations left them), its
    // observations and its swarm's personal bests
    std::vector<PolishWin> ht(W);
    for (int i = 0; i < W; ++i) {
        const BatchWindow& bw = b->h_wins[i];
        PolishWin& t = ht[i];
        t.w = bw.w;
        t.o.yf = b->yf + bw.obs_off;
        t.o.invyf = b->invy + bw.obs_off;
        t.o.yd = b->yd + bw.obs_off;
        t.pb = b->swarm + bw.sw_off + 2 * (size_t)P * bw.ld;
        t.pbf = b->swarm + bw.sw_off + 3 * (size_t)P * bw.ld;
        t.ld = bw.ld;
        t.M = bw.M;
    }
    e = cudaMemcpyAsync(tab, ht.data(), sizeof(PolishWin) * W, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_topk_tab(tab, W, k, keys, b->stream);
    if (e == cudaSuccess)
        e = launch_polish(tab, W, b->n_max, ht[0].w, ht[0].o, b->mdl, b->c64, keys, k, iters, first_step, 32, scratch,
                          ckpt, 1, res, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_pres, res, sizeof(ResultDev) * W, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return berr(SIRD_ERR_CUDA, std::string("polish: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < W; ++i) {
        const ResultDev& rd = b->h_pres[i];
        sird_result& r = results[i];
        std::memset(&r, 0, sizeof(r));
        r.n_params = P;
        for (int d = 0; d < P; ++d) r.theta[d] = rd.theta[d];
        r.loss = rd.loss;
        r.loss_search = rd.loss_search;
        r.r2_D = b->ss_tot[i] > 0 ? 1.0 - rd.sse / b->ss_tot[i] : NAN;
        r.index = rd.index;
        r.iters_done = b->iters;
    }
    return SIRD_OK;
}

extern "C" sird_status sird_batch_set_observations(sird_batch_t b, const double* y_all, long long n_total,
                                                   size_t* h2d_bytes) {
    TraceRange trace("sird_batch_set_observations");
    if (!b || !y_all) return berr(SIRD_ERR_ARG, "batch or y_all is NULL");
    const int nser = b->mdl.ird ? 3 : 1;  // F_IRD: each window's D, I, R series
    long long need = 0;
    for (const auto& pr : b->probs) need += (long long)nser * pr.n_obs;
    if (n_total != need)
        return berr(SIRD_ERR_ARG, "y_all must hold " + std::to_string(need) + " values (the series of every window)");
    for (long long i = 0; i < n_total; ++i)
        if (!std::isfinite(y_all[i])) return berr(SIRD_ERR_ARG, "non-finite observation in y_all");
    cudaError_t e = cudaSuccess;
    if (!b->h_stage) {
        e = cudaMallocHost((void**)&b->h_stage, b->wins_bytes + b->obs_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_upload, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return berr(SIRD_ERR_NOMEM, std::string("pinned staging: ") + cudaGetErrorString(e));
        }
    } else {
        e = cudaEventSynchronize(b->ev_upload);  // the previous upload has left the staging buffer
        if (e != cudaSuccess) return berr(SIRD_ERR_CUDA, std::string("upload wait: ") + cudaGetErrorString(e));
    }
    BatchWindow* hw = (BatchWindow*)b->h_stage;
    unsigned char* ob = b->h_stage + b->wins_bytes;
    float* yf = (float*)ob;
    float* invy = (float*)(ob + ((unsigned char*)b->invy - (unsigned char*)b->yf));
    double* yd = (double*)(ob + ((unsigned char*)b->yd - (unsigned char*)b->yf));
    std::memset(ob, 0, b->obs_bytes);
    const double* y = y_all;
    for (int i = 0; i < b->W; ++i) {
        sird_problem pr = b->probs[i];
        pr.y_D = y;
        if (nser == 3) {
            pr.y_I = y + pr.n_obs;
            pr.y_R = y + 2 * pr.n_obs;
        }
        ModelDev m{};
        BatchWindow bw = b->h_wins[i];
        sird_fill_window(&pr, bw.w, m);  // D0 = the new first observation; F_IRD ranges
        b->h_wins[i] = bw;
        hw[i] = bw;
        const int ps = obs_stride(pr.n_obs);
        for (int k = 0; k < nser; ++k)
            for (int j = 0; j < pr.n_obs; ++j) {
                const int o = b->obs_off[i] + k * ps + j;
                const double v = y[k * pr.n_obs + j];
                yf[o] = obs_f32(y + k * pr.n_obs, j, k != 1);
                invy[o] = v != 0.0 ? (float)(1.0 / v) : 0.f;
                yd[o] = v;
            }
        double mean = 0.0;
        for (int j = 0; j < pr.n_obs; ++j) mean += y[j];
        mean /= pr.n_obs;
        double ss = 0.0;
        for (int j = 0; j < pr.n_obs; ++j) ss += (y[j] - mean) * (y[j] - mean);
        b->ss_tot[i] = ss;
        y += (long long)nser * pr.n_obs;
    }
    e = cudaMemcpyAsync(b->wins, hw, b->wins_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->yf, ob, b->obs_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_upload, b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return berr(SIRD_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    if (h2d_bytes) *h2d_bytes = b->wins_bytes + b->obs_bytes;
    b->calibrated = false;  // the swarms' personal-best losses belong to the old observations
    return SIRD_OK;
}

extern "C" sird_status sird_pso_calibrate_batched(int W, const sird_problem* problems, const sird_pso_config* configs,
                                                  void* cuda_stream, sird_result* results) {
    if (!results) return berr(SIRD_ERR_ARG, "results is NULL");
    sird_batch_t b = nullptr;
    sird_status st = sird_batch_create(W, problems, configs, cuda_stream, &b);
    if (st != SIRD_OK) return st;
    st = sird_batch_calibrate(b, results);
    sird_batch_destroy(b);
    return st;
}
