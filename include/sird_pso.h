/*
 * sird_pso.h -- C ABI of the GB300 (sm_103a) SIRD-by-PSO calibration library.
 *
 * The library calibrates the SIRD model of Blaszczyk et al., "On automatic
 * calibration of the SIRD epidemiological model for COVID-19 data in Poland"
 * (arXiv 2204.12346), by particle swarm optimisation on one GPU:
 *
 *   model       Sec. 2.2, eq. (SIRD): S' = -beta S I / N, I' = beta I S / N - (gamma + mu) I,
 *               R' = gamma I, D' = mu I, with N = S + I + R + D constant
 *   beta(t)     Sec. 2.2, eq. (beta): beta1, a linear ramp on [t1, t2), beta2 -- or K equal
 *               constant segments over the window
 *   integrator  Sec. 3.1 and 3.3: explicit Euler from the window's first observation
 *   loss        Sec. 3.1: MXSE / MSE / MAE / MAPE on deceased counts (F_D^C), or the max
 *               over min-max-normalised I, R, D (F_IRD^C)
 *   optimiser   Sec. 3.3: PSO (inertia, cognitive, social coefficients; positions outside
 *               the box are set to the bound)
 *   forecast    Sec. 4.2: the fitted window extended with the last transmission rate,
 *               gamma and mu
 *
 * Conventions for every entry point:
 *   - No exception crosses the ABI.  Every call returns sird_status; SIRD_OK is 0.
 *   - A handle records the first error it meets ("sticky"); later calls on it return
 *     that status until sird_pso_clear_error().  sird_last_error() gives the message.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary CPU memory.  The library never frees caller memory.
 *   - All work of a handle runs on the CUDA stream given at creation (or set later),
 *     in issue order.  A handle is not thread-safe.
 *   - Sizes: at most SIRD_MAX_PARAMS parameters, 2^26 particles and 4096 observations
 *     per window; steps_per_day in 1..1000.
 */
#ifndef SIRD_PSO_H
#define SIRD_PSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIRD_MAX_PARAMS 32
#define SIRD_MAX_OBS 4096
#define SIRD_MAX_PARTICLES (1 << 26)

typedef enum sird_status {
    SIRD_OK = 0,
    SIRD_ERR_ARG = 1,         /* invalid argument: NULL pointer, size out of range, lb > ub,
                                 non-finite observation, log scale with lb <= 0 */
    SIRD_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in sird_last_error) */
    SIRD_ERR_NUMERIC = 3,     /* no finite loss where one is needed (e.g. every particle NaN) */
    SIRD_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out (the kernel returned early;
                                 a wait polls 2^21 (single-window exchange) or 2^22 (flat-batch
                                 barrier) times, a few seconds at most, or as many times as the
                                 environment variable SIRD_WAIT_LIMIT gives, read at launch) */
    SIRD_ERR_STATE = 5,       /* call out of order, or a state blob that does not match the handle */
    SIRD_ERR_NOMEM = 6,       /* device or host allocation failed */
    SIRD_ERR_UNSUPPORTED = 7  /* option combination the library does not implement */
} sird_status;

/* Low-level costs of Sec. 3.1. */
typedef enum sird_cost { SIRD_COST_MSE = 0, SIRD_COST_MXSE = 1, SIRD_COST_MAE = 2, SIRD_COST_MAPE = 3 } sird_cost;

/* Transmission-rate form: K equal constant segments, or the paper's ramp (eq. (beta)). */
typedef enum sird_beta_form { SIRD_BETA_PWC = 0, SIRD_BETA_RAMP = 1 } sird_beta_form;

/* How the swarm iterations are launched (results are identical). */
typedef enum sird_launch_mode {
    SIRD_LAUNCH_AUTO = 0,
    SIRD_LAUNCH_PER_ITER = 1,
    SIRD_LAUNCH_PERSISTENT = 2,
    /* batches (configs[0].launch_mode, with configs[0].block_size given): */
    SIRD_LAUNCH_WINDOW_PER_BLOCK = 3, /* a block runs one window at a time (the default) */
    SIRD_LAUNCH_FLAT = 4,             /* every window's swarm spread over the whole grid */
    /* one window (FP32): all iterations in one launch of one thread-block cluster */
    SIRD_LAUNCH_CLUSTER = 5
} sird_launch_mode;

/* Main objective: F_D^C (deaths only) or F_IRD^C (max over I, R, D), Sec. 3.1. */
typedef enum sird_objective { SIRD_FIT_D = 0, SIRD_FIT_IRD = 1 } sird_objective;

/*
 * One calibration window (Sec. 3.1).  All pointers are host memory and are copied
 * by the call that receives the problem.
 *
 *   n_obs          tau+1 observations on days 0..n_obs-1 of the window (2..SIRD_MAX_OBS)
 *   y_D            [n_obs] cumulative deceased.  The Euler scheme starts from D0 = y_D[0].
 *   y_I, y_R       [n_obs] infectious / recovered, used only by SIRD_FIT_IRD (else NULL)
 *   N              population (constant); S0 = N - I0 - R0 - D0
 *   I0             initial infectious when fit_I0 == 0
 *   R0             initial recovered
 *   fit_I0         1: I0 is the last entry of theta and is fitted
 *   beta_form      SIRD_BETA_PWC or SIRD_BETA_RAMP
 *   K              number of segments for SIRD_BETA_PWC (1..SIRD_MAX_PARAMS-3)
 *   steps_per_day  Euler steps per day; dt = 1/steps_per_day day
 *   cost, objective  see the enums.  SIRD_FIT_IRD: the cost of each of I, R, D against y_I,
 *                  y_R, y_D, errors divided by the series' range max - min (1 for a flat
 *                  series; MAPE unnormalised), the loss the largest of the three.  Every
 *                  evaluation, PSO, re-evaluation, batched, gradient and polish call takes
 *                  it; sird_pso_set_observations answers SIRD_ERR_UNSUPPORTED.
 *
 * theta layout (P entries):
 *   PWC : beta_1..beta_K, gamma, mu [, I0]          segment j covers steps
 *         [ceil(j*S/K), ceil((j+1)*S/K)) of the S = (n_obs-1)*steps_per_day steps
 *   RAMP: beta1, beta2, t1, t2, gamma, mu [, I0]    t1, t2 in days from the window start;
 *         if t1 > t2 the two are swapped.  beta is taken at the left end of each step.
 */
typedef struct sird_problem {
    int n_obs;
    const double* y_D;
    const double* y_I;
    const double* y_R;
    double N;
    double I0;
    double R0;
    int fit_I0;
    int beta_form;
    int K;
    int steps_per_day;
    int cost;
    int objective;
} sird_problem;

/*
 * Swarm configuration (Sec. 3.3).  lb, ub, log_scale are host arrays of P entries,
 * copied at creation.  Dimensions with log_scale[d] != 0 are searched in z = ln(theta)
 * (needs lb > 0) and clamped in z; the others in theta itself.
 *
 *   particles     swarm size M (1..SIRD_MAX_PARTICLES)
 *   iters         PSO iterations run by sird_pso_calibrate
 *   w, c1, c2     inertia, cognitive and social coefficients (the paper uses 0.5 each)
 *   precision     32: FP32 swarm and trajectories (compensated loss); 64: FP64 throughout
 *   seed          Philox4x32-10 key (64 bits)
 *   stream_id     fourth Philox counter word; separates independent swarms on one seed
 *   reeval_topk   FP32 only: at the end, the k best personal bests are re-evaluated in FP64
 *                 and the best of them is reported (0 = report the FP32 global best as is)
 *   block_size    threads per block for the swarm kernels (0 = library default; else a
 *                 multiple of 32 in 32..1024; the FP32 per-iteration kernels run blocks of at
 *                 most 256 threads, the FP64 kernels accept at most 256; results do not depend
 *                 on the block shape)
 *   launch_mode   SIRD_LAUNCH_AUTO, SIRD_LAUNCH_PER_ITER (one kernel per iteration),
 *                 SIRD_LAUNCH_PERSISTENT (FP32 only: all iterations in one cooperative launch
 *                 with the swarm in shared memory, the blocks' best exchanged through global
 *                 memory; needs every block co-resident) or SIRD_LAUNCH_CLUSTER (FP32 only:
 *                 the same in one thread-block cluster of at most 16 blocks, the best
 *                 exchanged through distributed shared memory; block_size 0 = the swarm split
 *                 over 16 blocks).  AUTO picks the cluster when the swarm fills 4 to 16 blocks
 *                 of block_size, else persistent when it fits.  All give bit-identical swarms.
 */
typedef struct sird_pso_config {
    int particles;
    int iters;
    double w, c1, c2;
    const double* lb;
    const double* ub;
    const int* log_scale;
    int precision;
    uint64_t seed;
    uint32_t stream_id;
    int reeval_topk;
    int block_size;
    int launch_mode;
} sird_pso_config;

/* Result of a calibration (host struct written by the library). */
typedef struct sird_result {
    int n_params;
    double theta[SIRD_MAX_PARAMS];  /* parameters of the reported best (decoded, FP64) */
    double loss;                    /* FP64 loss of theta, evaluated on the GPU */
    double loss_search;             /* the personal-best value the search stored for it */
    double r2_D;                    /* coefficient of determination on D (Sec. 3.1) */
    int index;                      /* particle whose personal best is reported */
    int iters_done;                 /* PSO iterations completed */
} sird_result;

typedef struct sird_pso* sird_pso_t;

/* ---------------------------------------------------------------- lifetime */

/* Validates and copies the problem and configuration, allocates the swarm in device
 * memory and binds the handle to cuda_stream (a cudaStream_t; NULL = default stream).
 * On failure *out is NULL and the message is available from sird_last_error(NULL). */
sird_status sird_pso_create(const sird_problem* problem, const sird_pso_config* config,
                            void* cuda_stream, sird_pso_t* out);
/* Waits for the handle's stream, then releases its device memory and graphs.  NULL is a no-op. */
void sird_pso_destroy(sird_pso_t h);
/* Message of the handle's sticky error, or of the last failed create when h is NULL. */
const char* sird_last_error(sird_pso_t h);
sird_status sird_pso_clear_error(sird_pso_t h);
sird_status sird_pso_set_stream(sird_pso_t h, void* cuda_stream);
/* Number of parameters P of the handle's theta layout (0 if h is NULL). */
int sird_pso_num_params(sird_pso_t h);
/* Launch mode the handle uses for its iterations: SIRD_LAUNCH_PER_ITER, SIRD_LAUNCH_PERSISTENT
 * or SIRD_LAUNCH_CLUSTER (what SIRD_LAUNCH_AUTO resolved to); 0 if h is NULL. */
int sird_pso_launch_mode(sird_pso_t h);

/* ---------------------------------------------------------------- fitness */

/*
 * Loss of M parameter vectors (Sec. 3.1: the Euler trajectory of eq. (SIRD) from the
 * window start, then the cost on D).  d_theta is device memory, structure-of-arrays
 * [P][ld] (entry d of vector m at d*ld + m), float for precision 32 and double for 64;
 * d_loss is device memory [M] of the same type.  Runs on the handle's stream; returns
 * after the launch.  ld >= M.  Non-finite losses are written as they come out.
 */
sird_status sird_pso_eval(sird_pso_t h, const void* d_theta, int M, int ld, void* d_loss, int precision);

/* ---------------------------------------------------------------- swarm */

/* Draws positions and velocities (Philox, iteration 0), evaluates them, sets the
 * personal bests and the global best.  Asynchronous. */
sird_status sird_pso_init(sird_pso_t h);
/* Runs n_iters synchronous PSO iterations (Sec. 3.3): velocity, position, clamp to the
 * box, evaluation, personal best (strictly smaller loss), global best (lowest index on
 * ties; NaN counts as +inf).  Needs sird_pso_init or sird_pso_set_state first. */
sird_status sird_pso_step(sird_pso_t h, int n_iters);
/* init + config.iters iterations + (FP32) FP64 re-evaluation of the reeval_topk best,
 * captured once into a CUDA graph and replayed; blocks until the result is on the host. */
sird_status sird_pso_calibrate(sird_pso_t h, sird_result* out);
/* Replaces the handle's observations y_D (host [n_obs], same n_obs as at creation; the
 * first value stays D0 of the Euler scheme) with an asynchronous copy on the handle's
 * stream, so that one handle (and its captured graph) calibrates window after window.
 * y_D is copied into a pinned staging buffer before the call returns. */
sird_status sird_pso_set_observations(sird_pso_t h, const double* y_D, int n_obs);
/* Measurement hook: makes every later sird_pso_calibrate record the two CUDA events
 * (cudaEvent_t; NULL to stop) on the handle's stream right before the first PSO
 * iteration launch and right after the last one.  Re-captures the graph. */
sird_status sird_pso_set_timing(sird_pso_t h, void* event_iter_begin, void* event_iter_end);
/* Current best (re-evaluated in FP64 as in calibrate); blocks. */
sird_status sird_pso_result(sird_pso_t h, sird_result* out);
/* Waits for the handle's stream and returns the sticky status (device-side errors included). */
sird_status sird_pso_sync(sird_pso_t h);

/*
 * Swarm state as a host blob: a header (magic, version, M, P, precision, iteration,
 * gbest index, seed, stream_id) followed by x, v, pbest as [P][M] and pbest_f [M] in
 * the swarm's precision.  get_state with buf == NULL writes the size to *size.
 * set_state restores it exactly (the next step continues bit-identically).
 */
sird_status sird_pso_get_state(sird_pso_t h, void* buf, size_t* size);
sird_status sird_pso_set_state(sird_pso_t h, const void* buf, size_t size);

/* The k best personal bests of an FP32 swarm (k <= min(2048, particles)), best first (lowest
 * index on ties): theta_out (host, [k][P]) decoded in FP64 from the stored positions,
 * loss_out (host, [k]) their stored FP32 losses.  Blocks.  The forecast ensemble of Sec. 4.2
 * is built from these. */
sird_status sird_pso_topk(sird_pso_t h, int k, double* theta_out, double* loss_out);
/* The same, with each one's particle index (host, [k]; global for a shard, see below). */
sird_status sird_pso_topk_indexed(sird_pso_t h, int k, double* theta_out, double* loss_out, int* index_out);

/* ---------------------------------------------------------------- one swarm over several ranks
 *
 * The particles of a swarm are evaluated independently (Sec. 3.3); the synchronous global best
 * is their only coupling.  A swarm of `total` FP32 particles can therefore be split by particle:
 * each rank creates a handle for its particles (config.particles of them, the same seed and
 * stream word on every rank) and declares them particles offset .. offset + particles - 1 of the
 * swarm.  Its random numbers and its argmin keys then use the global particle index, so after
 *     sird_pso_init, then per iteration: sird_pso_shard_best on every rank, the argmin over the
 *     ranks (lowest loss, lowest index on ties), sird_pso_set_gbest of that particle's position
 *     on every rank, sird_pso_step(h, 1)
 * the shards together hold exactly the personal bests of the unsharded swarm.  A shard runs one
 * launch per iteration; sird_pso_calibrate, sird_pso_polish and the state blob calls refuse it;
 * sird_pso_result re-evaluates the shard's own best (its index reported globally).
 *
 * set_shard: before sird_pso_init; FP32 handles only (SIRD_ERR_UNSUPPORTED otherwise);
 *   SIRD_ERR_ARG unless 0 <= offset and offset + particles <= total <= SIRD_MAX_PARTICLES.
 * shard_best: the best personal best among the handle's particles after the last init/step
 *   (blocks): its FP32 loss, global index and position z (host, [P] floats, search
 *   coordinates: ln theta on log-scaled dimensions).
 * set_gbest: the swarm's global best for the next iteration (z host [P], inside the box; index
 *   in 0 .. total - 1); blocks until the copy is on the device.
 */
sird_status sird_pso_set_shard(sird_pso_t h, int offset, int total);
sird_status sird_pso_shard_best(sird_pso_t h, float* loss, int* index, float* z);
sird_status sird_pso_set_gbest(sird_pso_t h, const float* z, float loss, int index);

/* ---------------------------------------------------------------- gradient */

/*
 * Loss and its exact gradient (discrete adjoint of the Euler map; the paper notes that
 * PSO is used because no gradient is available, Sec. 3.3 -- the discrete loss does have
 * one).  d_theta [P][ld], d_loss [M], d_grad [P][ld_grad] (dL/dtheta) and d_grad_u0
 * [4][ld_grad] (dL/d(S0, I0, R0, D0) with the four taken as independent; may be NULL)
 * are device memory of the type `precision` names (32: float, 64: double), for a handle of
 * either precision.  precision 64: the paper's operation order, equal to the plain FP64
 * computation bit for bit; trajectories are recomputed from checkpoints every ckpt_every steps
 * (1..64).  precision 32: the compensated FP32 trajectory (the loss equals sird_pso_eval's FP32
 * loss bit for bit), checkpoints at every day start (ckpt_every is checked but not used),
 * steps_per_day 10, 20 or at most 64 (else SIRD_ERR_UNSUPPORTED); its gradient is the exact
 * adjoint of the discrete map evaluated in FP32 (relative error near 1e-5 of the summed terms).
 * Costs: MSE, MAE, MAPE, MXSE (sub-gradients at kinks).  F_IRD^C: the gradient of the series whose
 * cost attains the maximum (the first of I, R, D on ties, as the loss of that precision picks it),
 * its errors scaled by the series' range, injected into the adjoint of I, R or D on each
 * observation day; checkpoints then also hold R (FP64) or R's misfit (FP32).  Asynchronous on the handle's
 * stream; the checkpoint scratch grows on demand (that call synchronises the stream).
 */
sird_status sird_loss_grad(sird_pso_t h, const void* d_theta, int M, int ld, void* d_loss,
                           void* d_grad, int ld_grad, void* d_grad_u0, int precision, int ckpt_every);

/*
 * Gradient polish of an FP32 swarm's k best personal bests (k <= min(1024, particles)): iters
 * L-BFGS iterations on the search coordinates (dL/dz = theta dL/dtheta on log dimensions;
 * 8 stored pairs, algebra in FP64), each with one sird_loss_grad evaluation and a line search
 * that evaluates 16 step lengths 2^-q in one launch and takes the longest one meeting the
 * Armijo condition; positions are clamped to the box, and a coordinate on a bound whose gradient
 * points out of the box is held while the others move (projected L-BFGS).  precision 64: trials and gradients in
 * the paper's FP64 arithmetic (checkpoints every ckpt_every steps, 1..64); precision 32: the
 * compensated FP32 evaluation and the FP32 adjoint (steps_per_day 10, 20 or <= 64).
 * first_step is the largest change of any search coordinate in the first (steepest-descent)
 * step.  The best point ever evaluated is re-scored in FP64 and reported in *out (FP64 loss;
 * index = the candidate's particle).  The swarm itself is not changed.  Blocks.
 */
sird_status sird_pso_polish(sird_pso_t h, int k, int iters, double first_step, int ckpt_every, int precision,
                            sird_result* out);

/* ---------------------------------------------------------------- forecast */

/*
 * Deaths forecast (Sec. 4.2): for each of k parameter vectors (host, row-major [k][P]),
 * integrates the window and `horizon` more days with the last transmission rate, gamma
 * and mu, and writes D on days n_obs .. n_obs+horizon-1 of the window's numbering to
 * out_D (host, [k][horizon]).  precision 32 or 64; k in 1..SIRD_MAX_PARTICLES, horizon in
 * 1..100000.  Blocks until out_D is written.  SIRD_ERR_ARG on a bad problem, NULL pointers or
 * sizes out of range, SIRD_ERR_NOMEM when host or device memory for k x horizon values runs
 * out, SIRD_ERR_CUDA on a failed launch or copy; sird_last_error(NULL) gives the reason.
 */
sird_status sird_forecast(const sird_problem* problem, const double* theta, int k, int horizon,
                          double* out_D, int precision, void* cuda_stream);

/*
 * Ensemble bands of repeated calibrations (Sec. 4.2): for k parameter vectors (host, row-major
 * [k][P], e.g. the results of k calibrations of one window with different stream_id), each
 * integrated over the window and `horizon` more days with the last transmission rate, gamma
 * and mu (FP64, the paper's operation order), per day d = 0 .. n_obs+horizon-1 and per quantity
 * q = beta(t), R0(t) = beta(t)/(gamma+mu), S, I, R, D (beta and R0 at the day's first step;
 * the compartments after d days): the median of the k values (the mean of the two middle ones
 * for even k) and, for each fractions[b] in (0, 1], the central band holding that fraction:
 * the sorted values at floor(k (1 - f) / 2) from either end.
 *   out (host) [6][n_obs + horizon][1 + 2 n_bands]: median, low_0, high_0, low_1, high_1, ...
 * k in 1..4096, n_bands in 0..16, horizon in 0..100000.  Blocks until out is written.
 * SIRD_ERR_ARG on a bad problem, NULL pointers, sizes out of range, a fraction outside (0, 1]
 * or a non-finite theta; SIRD_ERR_NOMEM when memory runs out; SIRD_ERR_CUDA on a failed launch
 * or copy; sird_last_error(NULL) gives the reason.
 */
sird_status sird_ensemble_bands(const sird_problem* problem, const double* theta, int k, int horizon,
                                const double* fractions, int n_bands, double* out, void* cuda_stream);

/*
 * Stability of the fitted parameters over repeated calibrations (Sec. 4.2): for k parameter
 * vectors (host, row-major [k][P]) the median and the central bands of each parameter, with the
 * order statistics of sird_ensemble_bands (median: the middle value, or the mean of the two
 * middle ones for even k; band b: the sorted values at floor(k (1 - fractions[b]) / 2) from either
 * end).  The parameters in theta's order: beta_1 .. beta_K (PWC) or beta1, beta2, t1, t2 (ramp),
 * then gamma, mu and, when fitted, I0; the ramp's change times enter as t1 = min(t_a, t_b) and
 * t2 = max(t_a, t_b), the order in which the model uses them.
 *   out (host) [P][1 + 2 n_bands]: median, low_0, high_0, low_1, high_1, ...
 * k in 1..4096, n_bands in 0..16.  Blocks until out is written.  SIRD_ERR_ARG on a bad problem
 * (it names the model form), NULL pointers, sizes out of range, a fraction outside (0, 1] or a
 * non-finite theta; SIRD_ERR_NOMEM when memory runs out; SIRD_ERR_CUDA on a failed launch or copy.
 */
sird_status sird_parameter_bands(const sird_problem* problem, const double* theta, int k, const double* fractions,
                                 int n_bands, double* out, void* cuda_stream);

/* ---------------------------------------------------------------- batched */

/*
 * Many calibration windows in one persistent launch (the rolling windows of Sec. 3.1): every
 * block takes the next window from a queue (longest first), runs its whole PSO -- the
 * initialisation and config.iters iterations, global best within the block -- and re-evaluates
 * its global best in FP64.  A window's result equals sird_pso_calibrate with reeval_topk = 0,
 * the same seed and the same stream_id.
 *
 * problems[W], configs[W] are host arrays.  Every window must share beta_form, K,
 * steps_per_day, cost, objective, fit_I0, precision (32), w, c1, c2, iters, the bounds and
 * log_scale; n_obs, observations, N, I0, R0, particles (1..2^20 per window, at most
 * SIRD_MAX_PARTICLES over all windows), seed and stream_id may differ.  SIRD_ERR_ARG on
 * settings that break these rules, SIRD_ERR_NOMEM when host or device memory runs out.
 * Two forms run a batch: one window per block (a block takes the next window from a queue,
 * longest first), or flat (every window's particle pairs spread over all threads of a
 * co-resident grid, one bounded grid barrier per iteration, the last item of a window to
 * finish an iteration publishing its global best; SIRD_ERR_TIMEOUT if a barrier wait runs
 * out).  Both give the same results.  configs[0].block_size = 0 lets the library pick the form,
 * the threads per block and the blocks per SM by timing short trial runs of each candidate
 * (cached in the file named by the environment variable SIRD_TUNE_CACHE when it is set; with
 * SIRD_TUNE_VERBOSE=1 every candidate's time goes to stderr);
 * otherwise a multiple of 32 in 32..1024 with as many blocks per SM as fit, in the form
 * configs[0].launch_mode names (SIRD_LAUNCH_FLAT, else one window per block).  The kernels are
 * compiled for at most 768 threads per block one window per block and 512 flat (PWC beta, F_D),
 * or 384 in both forms (the ramp, F_IRD); a larger block_size is refused with SIRD_ERR_ARG.
 */
typedef struct sird_batch* sird_batch_t;
sird_status sird_batch_create(int W, const sird_problem* problems, const sird_pso_config* configs, void* cuda_stream,
                              sird_batch_t* out);
/* Runs the batch (captured once into a CUDA graph, replayed after); results[W] on the host.  Blocks. */
sird_status sird_batch_calibrate(sird_batch_t b, sird_result* results);
/*
 * New observations for every window of the batch, e.g. the next day's data on the same rolling
 * windows.  y_all (host) holds each window's n_obs values of y_D (the counts given at create) —
 * for an F_IRD batch its y_D, y_I and y_R, n_obs values each — window after window: n_total =
 * sum of n_obs (three times that for F_IRD).  Each window's D0 becomes its new first observation; N,
 * I0, R0 and the PSO settings stay.  The values are packed into pinned staging and copied on
 * the batch's stream, ordered before the next sird_batch_calibrate; y_all may be reused on
 * return.  *h2d_bytes (may be NULL) receives the bytes copied.  SIRD_ERR_ARG on NULL, a wrong
 * n_total or a non-finite value.
 */
sird_status sird_batch_set_observations(sird_batch_t b, const double* y_all, long long n_total, size_t* h2d_bytes);
/*
 * Gradient polish of every window of a calibrated batch (after sird_batch_calibrate): per window,
 * the k best personal bests of its swarm (k in 1..min(1024, smallest swarm)) get iters L-BFGS
 * iterations exactly as sird_pso_polish with precision 32 gives them (FP32 trials and adjoint,
 * FP64 algebra, FP64 re-scoring of the best point), all windows together: each step is one
 * launch over every window, and each window's result equals a one-window sird_pso_polish of the
 * same swarm bit for bit.  results[W] (host): theta, FP64 loss, r2_D, index = the particle whose
 * personal best the reported point started from, loss_search = that personal best's FP32 loss.
 * The swarms are not changed.  F_D objective, steps_per_day 10, 20 or at most 64, W <= 65535
 * (else SIRD_ERR_UNSUPPORTED); SIRD_ERR_STATE before the first calibration; SIRD_ERR_ARG on bad
 * k, iters < 0 or first_step <= 0.  The scratch is kept with the batch and grows on demand.
 * Blocks.
 */
sird_status sird_batch_polish(sird_batch_t b, int k, int iters, double first_step, sird_result* results);
/* Threads per block and blocks per SM the batch runs with (autotuned or given); 0 if b is NULL. */
int sird_batch_block_size(sird_batch_t b);
int sird_batch_blocks_per_sm(sird_batch_t b);
/* The batch's form: SIRD_LAUNCH_FLAT or SIRD_LAUNCH_WINDOW_PER_BLOCK; 0 if b is NULL. */
int sird_batch_launch_mode(sird_batch_t b);
/* Measurement hook: every later sird_batch_calibrate records the two CUDA events (cudaEvent_t;
 * NULL to stop) right before and right after the batch kernel.  Re-captures the graph. */
sird_status sird_batch_set_timing(sird_batch_t b, void* event_begin, void* event_end);
void sird_batch_destroy(sird_batch_t b);
/* One-shot create + calibrate + destroy.  Errors of the batch calls: sird_last_error(NULL). */
sird_status sird_pso_calibrate_batched(int W, const sird_problem* problems, const sird_pso_config* configs,
                                       void* cuda_stream, sird_result* results);

/* ---------------------------------------------------------------- no allocation */

#define SIRD_NOALLOC_MAX_OBS 4096

/*
 * One FP32 PSO iteration (iter >= 1), or the initialisation (iter == 0), on a swarm that the
 * caller owns, without allocating anything.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need a step -- a host
 * framework that owns the whole device budget and lends a plugin only its own buffers, or a
 * latency-critical loop where a cudaMalloc (which can synchronise the device) is not allowed.
 *
 * Same kernel and same results as sird_pso_step with SIRD_LAUNCH_PER_ITER on a handle built
 * from the same problem and config.  Inputs and outputs are the caller's:
 *   problem, config  host structs as for sird_pso_create, checked the same way (precision
 *                    must be 32, objective F_D); y_D gives D0 = y_D[0], the zeros that MAPE
 *                    skips and, for MAPE, the reciprocals 1/y_D rounded to float
 *   d_obs            device [n_obs] float observations of D: y_D[i] - y_D[0] rounded to float,
 *                    as the handle stores them (only differences of consecutive entries are
 *                    used, so the float values of y_D give the same results when y_D[0] = 0 or
 *                    when y_D holds integers below 2^24)
 *   d_x, d_v, d_pbest  device [P][ld] float, read and written (layout of sird_pso_eval)
 *   d_pbest_f        device [ld] float, read and written
 *   d_gbest          device [P] float: read as the previous global best, rewritten
 *   iter             iteration number (the Philox counter word); 0 initialises
 *   d_gbest_index    device int (may be NULL): receives the new global-best index
 *   cuda_stream      cudaStream_t (NULL = default stream); the call returns after enqueueing
 * Its only scratch (the global-best reduction words and, for MAPE, reciprocals of the
 * observations) is a fixed array of 256 + 4*SIRD_NOALLOC_MAX_OBS bytes that the library keeps
 * in every device's global memory until the process exits.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress), so make the first call on each device
 * before any stream capture.  Every call uses the same array: the call clears the words that
 * must start at zero, but calls that overlap on the GPU (different streams, other threads) race
 * on it -- serialise them.  n_obs above SIRD_NOALLOC_MAX_OBS is rejected with SIRD_ERR_ARG; the
 * message is available from sird_last_error(NULL).  No cudaMalloc, cudaFree or other allocating
 * call is made.  The kernels' device-side error bits (a loss that came out NaN, counted as
 * +inf; index checks of a SIRD_DEBUG_BOUNDS build) are not reported by this entry point: the
 * array's error word is cleared by every call and not read back.
 */
sird_status sird_pso_step_f32_noalloc(const sird_problem* problem, const sird_pso_config* config,
                                      const float* d_obs, float* d_x, float* d_v, float* d_pbest,
                                      float* d_pbest_f, float* d_gbest, int ld, int iter,
                                      int* d_gbest_index, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif
