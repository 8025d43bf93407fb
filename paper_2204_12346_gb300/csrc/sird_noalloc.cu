// sird_noalloc.cu -- one FP32 PSO iteration on caller-owned buffers, with no allocation.
//
// Some callers cannot allocate device memory at the moment they need a swarm step: a host
// framework that reserves the whole device budget up front and hands plugins only the
// buffers it owns, a latency-critical loop where a cudaMalloc (which may synchronise the
// device) is not acceptable, or code that must not touch the allocator for other reasons.
// For them this file provides sird_pso_step_f32_noalloc: the same fused iteration kernel as
// sird_pso_step, but its only scratch -- the global-best reduction words and, for MAPE, the
// table of reciprocal observations -- lives in a fixed array in device global memory that the
// library declares at file scope.  Every GPU that loads the library keeps that array until
// the process exits; it is small (kNoAllocScratchBytes).
//
// The host never dereferences the array's name: it is only a host-side stand-in for the
// device symbol.  Its device address is fetched once per device with cudaGetSymbolAddress,
// with that device current, by the first call made on that device, and handed to the kernels
// as an ordinary pointer.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/sird_pso.h"
#include "kernels.h"

using namespace sird;

// The handle path's argument checks and window constants (sird_pso_api.cu), so that this entry
// point derives exactly what sird_pso_create derives.
sird_status sird_check_problem(const sird_problem* pb, std::string& why);
void sird_fill_window(const sird_problem* pb, WindowDev& w, ModelDev& m);

namespace {

constexpr int kNoAllocMaxObs = SIRD_NOALLOC_MAX_OBS;
constexpr size_t kNoAllocHeader = 256;  // reduction words (gkey, counter, gbest index/value, error)
constexpr size_t kNoAllocScratchBytes = kNoAllocHeader + (size_t)kNoAllocMaxObs * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (fetched once per device).
cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_ptr[dev];
    return cudaSuccess;
}

// The message goes where sird_last_error(NULL) reads it.
sird_status fail(sird_status s, const char* msg) {
    sird::set_global_error(msg);
    return s;
}

}  // namespace

extern "C" sird_status sird_pso_step_f32_noalloc(const sird_problem* pb, const sird_pso_config* cfg,
                                                 const float* d_obs, float* d_x, float* d_v, float* d_pbest,
                                                 float* d_pbest_f, float* d_gbest, int ld, int iter,
                                                 int* d_gbest_index, void* cuda_stream) {
    if (!pb || !cfg) return fail(SIRD_ERR_ARG, "problem or config is NULL");
    if (pb->n_obs < 2 || pb->n_obs > kNoAllocMaxObs)
        return fail(SIRD_ERR_ARG, "n_obs out of range [2, SIRD_NOALLOC_MAX_OBS]");
    {
        std::string why;  // touched only when a check fails
        const sird_status st = sird_check_problem(pb, why);
        if (st != SIRD_OK) {
            sird::set_global_error(why.c_str());
            return st;
        }
    }
    if (pb->objective != SIRD_FIT_D) return fail(SIRD_ERR_UNSUPPORTED, "only the F_D objective");
    if (cfg->precision != 32) return fail(SIRD_ERR_UNSUPPORTED, "the no-allocation step is FP32 only");
    const int P = (pb->beta_form == SIRD_BETA_RAMP ? 6 : pb->K + 2) + (pb->fit_I0 ? 1 : 0);
    const int M = cfg->particles;
    if (M < 1 || M > SIRD_MAX_PARTICLES || ld < M) return fail(SIRD_ERR_ARG, "particles out of range or ld < particles");
    if (iter < 0) return fail(SIRD_ERR_ARG, "iter < 0");
    if (!d_obs || !d_x || !d_v || !d_pbest || !d_pbest_f || !d_gbest) return fail(SIRD_ERR_ARG, "a device buffer is NULL");
    if (!cfg->lb || !cfg->ub) return fail(SIRD_ERR_ARG, "lb/ub is NULL");
    const int block = cfg->block_size ? cfg->block_size : 128;
    if (block < 32 || block > 1024 || block % 32) return fail(SIRD_ERR_ARG, "block_size must be a multiple of 32 in [32, 1024]");

    // window constants, exactly as the handle path derives them
    WindowDev w{};
    ModelDev m{};
    sird_fill_window(pb, w, m);
    const int n = pb->n_obs;

    PsoCoeffs<float> c{};
    for (int d = 0; d < P; ++d) {
        const bool lg = cfg->log_scale && cfg->log_scale[d];
        if (!std::isfinite(cfg->lb[d]) || !std::isfinite(cfg->ub[d]) || cfg->lb[d] > cfg->ub[d] || (lg && !(cfg->lb[d] > 0)))
            return fail(SIRD_ERR_ARG, "bad bounds");
        if (lg) c.logmask |= 1u << d;
        c.zlb[d] = (float)(lg ? std::log(cfg->lb[d]) : cfg->lb[d]);
        c.zub[d] = (float)(lg ? std::log(cfg->ub[d]) : cfg->ub[d]);
    }
    c.w = (float)cfg->w;
    c.c1 = (float)cfg->c1;
    c.c2 = (float)cfg->c2;
    c.key0 = (uint32_t)cfg->seed;
    c.key1 = (uint32_t)(cfg->seed >> 32);
    c.stream_id = cfg->stream_id;

    unsigned char* s = nullptr;
    cudaError_t e = noalloc_scratch(&s);
    if (e != cudaSuccess) return fail(SIRD_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ReduceScratch r{};
    r.gkey = (unsigned long long*)s;
    r.counter = (unsigned int*)(s + 8);
    r.gbest_idx = (int*)(s + 16);
    r.gbest_f = s + 24;
    r.err = (unsigned*)(s + 32);
    float* inv = (float*)(s + kNoAllocHeader);
    // the reduction words must start from their neutral values: key all ones, the rest zero
    e = cudaMemsetAsync(s, 0, kNoAllocHeader, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.gkey, 0xFF, sizeof(unsigned long long), st);
    if (e == cudaSuccess && m.cost == COST_MAPE) {
        // reciprocals of the double observations, rounded to float as the handle path stores them
        // (a fixed host array: the copy from pageable memory is staged before the call returns)
        float inv_h[kNoAllocMaxObs];
        for (int i = 0; i < n; ++i) inv_h[i] = pb->y_D[i] != 0.0 ? (float)(1.0 / pb->y_D[i]) : 0.f;
        e = cudaMemcpyAsync(inv, inv_h, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return fail(SIRD_ERR_CUDA, cudaGetErrorString(e));
    ObsDev o{d_obs, inv, nullptr};
    SwarmDev<float> sw{d_x, d_v, d_pbest, d_pbest_f, d_gbest, M, ld};
    e = launch_pso_f32(w, m, o, c, sw, r, iter, block, st);
    if (e == cudaSuccess && d_gbest_index)
        e = cudaMemcpyAsync(d_gbest_index, r.gbest_idx, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(SIRD_ERR_CUDA, cudaGetErrorString(e));
    return SIRD_OK;
}
