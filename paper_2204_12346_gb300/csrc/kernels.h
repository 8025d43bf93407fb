// kernels.h -- host-side launchers of the calibration kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sird_model.cuh"

namespace sird {

// Largest block of the per-iteration FP32 kernels (their launch bound: up to 255 registers a
// thread, enough for every form without spilling); larger requested blocks run as this size.
constexpr int kF32IterMaxBlock = 256;

// Dispatch of the FP32 kernels over (steps per day, variant): defines S_ (steps per day fixed at
// compile time, 0 = any) and C_ (cost | form << 2) for the body.  F_D with PWC beta -- the
// benchmark's form -- is unrolled for 10 and 20 steps per day, the ramp for 10, the rest generic.
#define SIRD_F32_COSTS(FORMV, SPDC, ...)                                                        \
    switch (m.cost) {                                                                           \
        case COST_MSE: { constexpr int S_ = SPDC; constexpr int C_ = COST_MSE | (FORMV << 2); __VA_ARGS__; } break;   \
        case COST_MXSE: { constexpr int S_ = SPDC; constexpr int C_ = COST_MXSE | (FORMV << 2); __VA_ARGS__; } break; \
        case COST_MAE: { constexpr int S_ = SPDC; constexpr int C_ = COST_MAE | (FORMV << 2); __VA_ARGS__; } break;   \
        default: { constexpr int S_ = SPDC; constexpr int C_ = COST_MAPE | (FORMV << 2); __VA_ARGS__; } break;        \
    }
#define SIRD_DISPATCH_F32(m, ...)                                                        \
    switch (form_of(m)) {                                                               \
        case FORM_PWC_D:                                                                \
            if (m.spd == 10) { SIRD_F32_COSTS(FORM_PWC_D, 10, __VA_ARGS__) }            \
            else if (m.spd == 20) { SIRD_F32_COSTS(FORM_PWC_D, 20, __VA_ARGS__) }       \
            else { SIRD_F32_COSTS(FORM_PWC_D, 0, __VA_ARGS__) }                         \
            break;                                                                      \
        case FORM_PWC_IRD: { SIRD_F32_COSTS(FORM_PWC_IRD, 0, __VA_ARGS__) } break;      \
        case FORM_RAMP_D:                                                               \
            if (m.spd == 10) { SIRD_F32_COSTS(FORM_RAMP_D, 10, __VA_ARGS__) }           \
            else { SIRD_F32_COSTS(FORM_RAMP_D, 0, __VA_ARGS__) }                        \
            break;                                                                      \
        default:                                                                        \
            if (m.spd == 10) { SIRD_F32_COSTS(FORM_RAMP_IRD, 10, __VA_ARGS__) }         \
            else { SIRD_F32_COSTS(FORM_RAMP_IRD, 0, __VA_ARGS__) }                      \
            break;                                                                      \
    }

// Swarm in structure-of-arrays layout: entry d of particle p at [d*ld + p].
template <typename T>
struct SwarmDev {
    T* x;
    T* v;
    T* pb;      // personal-best positions
    T* pbf;     // [ld] personal-best values
    T* gbest;   // [P] global-best position (written by the last block of each iteration)
    int M, ld;
};

// Global-best bookkeeping and error word.
struct ReduceScratch {
    unsigned long long* gkey;  // FP32 swarms: packed (ordered loss, index), reset to ~0 after use
    MinPair64* partial;        // FP64 swarms: per-block (loss, index)
    unsigned int* counter;     // blocks finished in the current launch (reset by the last block)
    int* gbest_idx;
    void* gbest_f;             // float or double
    unsigned* err;             // kErr* bits
    unsigned* abort;           // persistent kernel: set by a block whose wait ran out
};

// One block's published best of one iteration (persistent kernel).  Every 64-bit word holds
// the iteration number in its high half, so a reader knows a word is current without any
// fence: (tag, ordered loss bits), (tag, particle index), (tag, position bits) x P.
struct ExchangeSlot {
    unsigned long long w_loss;
    unsigned long long w_idx;
    unsigned long long w_pos[kMaxParams];
};

template <typename T>
struct PsoCoeffs {
    T w, c1, c2;
    T zlb[kMaxParams], zub[kMaxParams];
    uint32_t logmask;
    uint32_t key0, key1, stream_id;
    uint32_t p_off;  // global index of the swarm's particle 0 (a shard of a larger swarm; else 0)
};

// FP64 result of the re-evaluation of candidate personal bests.
struct ResultDev {
    double theta[kMaxParams];
    double loss;
    double loss_search;
    double sse;
    int index;
    int count;  // candidates evaluated
};

// Observations on the device (series stacked D | I | R for F_IRD, each padded to obs_stride).
struct ObsDev {
    const float* yf;     // [n_obs] FP32 copy, see obs_f32
    const float* invyf;  // [n_obs] 1/y or 0
    const double* yd;    // [n_obs]
};

// Entry i of a series' FP32 copy: the cumulative counts D and R as their difference from the
// series' first value (the FP32 trajectory uses only differences of consecutive days, which are
// then exact for integer counts that change by less than 2^24 over the window, at any level of
// the series), I as its value.
inline float obs_f32(const double* y, int i, bool diff) { return (float)(diff ? y[i] - y[0] : y[i]); }

size_t smem_bytes_f32(const WindowDev& w, const ModelDev& m, int block, bool with_theta);

// One window of a table-form launch (the polish of many windows at once): its constants, its
// observations and its swarm's personal bests.  A table-form kernel's block row blockIdx.y
// works on window blockIdx.y, with the window's own constants and the arithmetic of the
// one-window kernel, so each window's results equal a one-window launch's bit for bit.
struct PolishWin {
    WindowDev w;
    ObsDev o;
    const float* pb;   // personal-best positions [P][ld], search coordinates
    const float* pbf;  // personal-best values [ld]
    int ld, M;
};

// Table forms of the FP32 evaluation and loss gradient: window i < nw takes its M vectors at
// theta + i * th_ws (leading dimension ld) and writes loss + i * loss_ws (and, for the
// gradient, grad + i * grad_ws with leading dimension ldg; checkpoints at ckpt + i * ck_ws,
// ck_ws >= adjoint_ckpt_bytes_f32 of an n_max-observation window / 4).  n_max bounds the
// windows' n_obs.
cudaError_t launch_eval_f32_tab(const PolishWin* tab, int nw, int n_max, const ModelDev& m, const float* theta,
                                long long th_ws, int ld, int M, float* loss, long long loss_ws, int block,
                                cudaStream_t s);
cudaError_t launch_loss_grad_f32_tab(const PolishWin* tab, int nw, int n_max, const ModelDev& m, const float* theta,
                                     long long th_ws, int ld, int M, float* loss, long long loss_ws, float* grad,
                                     long long grad_ws, int ldg, float* ckpt, long long ck_ws, cudaStream_t s);
// The k smallest keys (packed loss, index) of every window's personal bests, ascending, into
// keys[i * k .. i * k + k - 1]; k <= kTopkTabMax and k <= each window's M.
constexpr int kTopkTabMax = 1024;
cudaError_t launch_topk_tab(const PolishWin* tab, int nw, int k, unsigned long long* keys, cudaStream_t s);

cudaError_t launch_eval_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const float* theta, int ld,
                            int M, float* loss, int block, unsigned* err, cudaStream_t s);
cudaError_t launch_eval_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const double* theta, int ld,
                            int M, double* loss, int block, unsigned* err, cudaStream_t s);

// One PSO iteration (iter >= 1) or the initialisation (iter == 0), fused with the global-best
// reduction.  All blocks read sw.gbest at their start; the last block to finish rewrites it.
cudaError_t launch_pso_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<float>& c,
                           const SwarmDev<float>& sw, const ReduceScratch& r, int iter, int block, cudaStream_t s);
cudaError_t launch_pso_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<double>& c,
                           const SwarmDev<double>& sw, const ReduceScratch& r, int iter, int block, cudaStream_t s);

// All iterations iter0+1 .. iter0+n_iters of an FP32 swarm in one cooperative launch (every
// block co-resident); slots needs 2 * ceil(M / block) entries.  Resets the slots and the abort
// flag first.
size_t smem_bytes_persistent(const WindowDev& w, const ModelDev& m, int block, int grid);
int persistent_capacity(const WindowDev& w, const ModelDev& m, int block, int grid);
constexpr int kMaxPersistentBlocks = 128;
// The same with the grid as one thread-block cluster of at most kMaxClusterBlocks blocks,
// exchanging the blocks' best through distributed shared memory (no slots).
constexpr int kMaxClusterBlocks = 16;
bool cluster_fits(const WindowDev& w, const ModelDev& m, int block, int grid);
cudaError_t launch_pso_f32_cluster(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<float>& c,
                                   const SwarmDev<float>& sw, const ReduceScratch& r, int iter0, int n_iters, int block,
                                   cudaStream_t s);
cudaError_t launch_pso_f32_persistent(const WindowDev& w, const ModelDev& m, const ObsDev& o,
                                      const PsoCoeffs<float>& c, const SwarmDev<float>& sw, const ReduceScratch& r,
                                      ExchangeSlot* slots, int iter0, int n_iters, int block, cudaStream_t s);

// Deaths forecast of k parameter vectors (theta [P][ld], float or double by precision) into
// out[k][horizon] (same type): D on days n_obs .. n_obs+horizon-1 of the window's numbering.
cudaError_t launch_forecast(const WindowDev& w, const ModelDev& m, const void* theta, int ld, int k, int horizon,
                            const float* yf, void* out, int precision, cudaStream_t s);

// The k personal bests named by keys (FP32 swarm), decoded to theta in FP64: theta_out[k][P],
// loss_out[k] = their stored FP32 values.
cudaError_t launch_topk_gather(const unsigned long long* keys, int k, const float* pb, const float* pbf, int ld,
                               int P, uint32_t logmask, double* theta_out, double* loss_out, cudaStream_t s);

// Loss and exact gradient (discrete adjoint) of M parameter vectors in FP64; checkpoints every C
// steps (1..64) in ckpt (adjoint_ckpt_bytes).
size_t adjoint_ckpt_bytes(const WindowDev& w, const ModelDev& m, int M, int C);
cudaError_t launch_loss_grad_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const double* theta, int ld,
                                 int M, double* loss, double* grad, int ldg, double* grad_u0, double* ckpt, int C,
                                 cudaStream_t s);

// The same in FP32 (compensated trajectory; loss identical to the FP32 evaluation), checkpoints
// at every day start in ckpt (adjoint_ckpt_bytes_f32); steps per day 10, 20 or at most 64.
size_t adjoint_ckpt_bytes_f32(const WindowDev& w, const ModelDev& m, int M);
cudaError_t launch_loss_grad_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const float* theta, int ld,
                                 int M, float* loss, float* grad, int ldg, float* grad_u0, float* ckpt,
                                 cudaStream_t s);

// Ensemble statistics (bands.cu): k <= kMaxEnsemble parameter vectors ([P][k] device), their
// FP64 trajectories over n_days days (window + extension) into traj (ensemble_traj_bytes), then
// per day and quantity (beta, R0, S, I, R, D) the median and n_bands central bands, each
// dropping drop[b] sorted values at either end, into out [6][n_days][1 + 2 n_bands].
constexpr int kMaxEnsemble = 4096;
constexpr int kBandQuantities = 6;
size_t ensemble_traj_bytes(int k, int n_days);
cudaError_t launch_ensemble_bands(const WindowDev& w, const ModelDev& m, const double* theta, int k, int n_days,
                                  const int* drop, int n_bands, double* traj, double* out, cudaStream_t s);
// The same summary of the parameters themselves: theta [P][k] (device; the ramp's change times
// are reordered in place to t1 <= t2) into out [P][1 + 2 n_bands].
cudaError_t launch_parameter_bands(const ModelDev& m, double* theta, int k, const int* drop, int n_bands, double* out,
                                   cudaStream_t s);

// L-BFGS polish, for each of the nw windows of tab, of its k candidates named by keys[i * k ..]
// (personal bests of its FP32 swarm): iters iterations with a parallel line search, trials and
// gradient in FP32 (precision 32) or, for one window (nw == 1, w and o its constants and
// observations), FP64 (64); best point kept; each window's best candidate's theta / FP64 loss /
// sse into res[i].  scratch: polish_scratch_doubles(P, nw * k) doubles; ckpt: nw windows of
// polish_ckpt_floats(n_max, k) floats (FP32), or adjoint_ckpt_bytes(w, m, k, ckpt_every) bytes.
size_t polish_scratch_doubles(int P, int k);
size_t polish_ckpt_floats(int n_max, int k, const ModelDev& m);
cudaError_t launch_polish(const PolishWin* tab, int nw, int n_max, const WindowDev& w, const ObsDev& o,
                          const ModelDev& m, const PsoCoeffs<double>& c, const unsigned long long* keys, int k,
                          int iters, double first_step, int precision, double* scratch, void* ckpt, int ckpt_every,
                          ResultDev* res, cudaStream_t s);

// ---------------------------------------------------------------- batched windows
struct BatchWindow {
    WindowDev w;
    int obs_off;         // offset of this window's observations in the packed arrays
    int M, ld;           // particles, leading dimension of its swarm block
    long long sw_off;    // offset (floats) of its swarm block: x, v, pbest [P][ld], pbest_f [ld]
    uint32_t key0, key1, stream_id;
};
struct BatchOut {
    float z[kMaxParams];        // global-best position (search coordinates)
    double theta[kMaxParams];   // decoded in FP64
    double loss64, sse;         // FP64 re-evaluation
    float loss;                 // FP32 global-best loss
    int index;
};
// Poll limit of a device-side bounded wait: dflt, or the positive value of the environment
// variable SIRD_WAIT_LIMIT (read at each launch; a small value makes the waits run out, which
// is how the timeout path is tested).
unsigned bounded_wait_limit(unsigned dflt);

// Flat form of the batch: every thread of a co-resident grid owns the particle pairs
// (w, j0, j1) with item index thread + r * threads; one bounded grid barrier per iteration; the
// last item of a window to finish an iteration publishes the window's global best.
struct FlatScratch {
    unsigned long long* gkey;  // [W] packed (loss, index) minimum of the running iteration
    unsigned* done;            // [W] items finished in the running iteration
    float* gpos;               // [W][kMaxParams] global-best position of the last iteration
    unsigned* bar_count;       // grid barrier arrivals
    unsigned* bar_gen;         // grid barrier generation
    unsigned* err;             // error bits (kErrTimeout)
    unsigned* abort;           // set by a block that gave up waiting
};
size_t flat_smem_bytes(const ModelDev& m, int block);
int flat_blocks_per_sm(const ModelDev& m, int block);
cudaError_t launch_flat(const BatchWindow* wins, const int* n_items_w, const int4* items, int n_items, int W,
                        const ModelDev& m, const PsoCoeffs<float>& c, const float* yf_all, const float* invy_all,
                        float* swarm, const FlatScratch& fs, BatchOut* out, int iters, int block, int grid,
                        cudaStream_t s);
size_t batch_smem_bytes(const ModelDev& m, int block, int n_max);
int batch_blocks_per_sm(const ModelDev& m, int block, int n_max);
cudaError_t launch_batch(const BatchWindow* wins, const int* order, int W, const ModelDev& m, const PsoCoeffs<float>& c,
                         const float* yf_all, const float* invy_all, const double* yd_all, float* swarm,
                         unsigned* queue, BatchOut* out, int iters, int n_max, int block, int grid, bool reeval,
                         cudaStream_t s);
cudaError_t launch_batch_reeval(const BatchWindow* wins, int W, const ModelDev& m, uint32_t logmask,
                                const double* yd_all, BatchOut* out, cudaStream_t s);

// Message returned by sird_last_error(NULL) on this thread.
void set_global_error(const char* msg);

// Smallest k keys (packed loss, index) of the FP32 personal bests, sorted ascending, into out[k].
// tmp_a / tmp_b need topk_scratch_keys(M, k) entries each.
size_t topk_scratch_keys(int M, int k);
cudaError_t launch_topk_f32(const float* pbf, int M, int k, unsigned long long* tmp_a, unsigned long long* tmp_b,
                            unsigned long long** out, cudaStream_t s);

// FP64 re-evaluation of candidates (FP32 personal bests named by keys[0..k-1], or the FP64
// global best when keys == nullptr) and the argmin of them into *res.
cudaError_t launch_reeval(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<float>* c32,
                          const PsoCoeffs<double>* c64, const void* pb, const void* pbf, int ld,
                          const unsigned long long* keys, int k, const int* gbest_idx, ResultDev* res,
                          cudaStream_t s);

}  // namespace sird
