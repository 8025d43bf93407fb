// polish.cu -- L-BFGS polish of the best PSO candidates with a parallel line search.
//
// PSO (Sec. 3.3) needs no gradient; near its optimum the swarm resolves the loss only as far
// as its search does.  The discrete adjoint gives the exact gradient of the FP64 loss, so the
// k best personal bests are refined by projected L-BFGS in the search coordinates (z = ln theta
// on log dimensions, where dL/dz = theta dL/dtheta), positions clamped to the box.  Each
// iteration:
//   1. direction d = -H g by the two-loop recursion over the last kMem (s, y) pairs, on the
//      dimensions not held at a bound of the box (a calibration's optimum often has beta or I0
//      on the box's edge; an unprojected step there is cut back by the clamp and stalls),
//   2. kTrials trial points z + 2^-q d (q = 0..kTrials-1) for every candidate, evaluated in ONE
//      launch -- an evaluation of a few candidates is latency-bound, so 16 trials cost about
//      what one does,
//   3. the largest step that satisfies the Armijo condition (else the best trial if it lowers
//      the loss, else a curvature probe that leaves the point where it is; kProbes + 1
//      failures in a row stop the candidate),
//   4. the gradient at the accepted point (adjoint launch) and the history update.
// The best point ever evaluated is re-scored in FP64 (the paper's operation order) and reported.
// Precision 64 evaluates the trials and the gradient in FP64; precision 32 uses the compensated
// FP32 evaluation and the FP32 adjoint (about 15x faster per iteration) while the L-BFGS
// algebra stays in FP64.
//
// The windows of a batch (Sec. 3.1: rolling windows, each calibrated on its own) are polished
// together: candidate g of the nw * k belongs to window g / k, every step above is one launch
// over all windows (the evaluations and gradients in table form, block row = window), and a
// window's candidates see exactly the arithmetic of a one-window polish.
#include <cmath>

#include "kernels.h"

namespace sird {

namespace {

constexpr int kMem = 8;
constexpr int kTrials = 16;
constexpr int kProbes = 4;  // curvature probes in a row before a candidate stops

// Per-candidate state, structure of arrays with candidate g (window g / k, its candidate g % k)
// at [.. * kk + g], kk = nw * k.  Trial t of candidate g sits at column tcol(g, t) of the
// [.. * kt * nw] trial arrays: each window's kt = k * kTrials trials contiguous, trial-major.
struct PolishState {
    double *z, *g, *f, *d, *zt, *tht, *ft, *S, *Y, *best_f, *best_th, *gth, *lnew;
    float *thf, *ftf, *gthf, *lnewf;  // FP32 mode: trial thetas, their losses, gradient, loss
    int *head, *count, *active, *cand;
    int P, k, nw, kk, f32;
    __device__ __forceinline__ size_t tcol(int g, int t) const {
        return (size_t)(g / k) * k * kTrials + (size_t)t * k + g % k;
    }
    __device__ __forceinline__ size_t tcols() const { return (size_t)kk * kTrials; }
};

__device__ __forceinline__ double decode(double z, bool lg) { return lg ? exp(z) : z; }

// Candidate g starts at its personal best, projected onto the box (the FP32 swarm searches the
// box rounded to FP32, which can reach a hair past the FP64 bounds; a start outside would turn
// every trial's clamp into a step of its own).
__global__ void polish_init_kernel(PolishState s, const PolishWin* __restrict__ tab,
                                   const unsigned long long* __restrict__ keys, PsoCoeffs<double> c) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= s.kk) return;
    const PolishWin& pw = tab[g / s.k];
    const int idx = (int)(keys[g] & 0xFFFFFFFFu);
    s.cand[g] = idx;
    s.head[g] = 0;
    s.count[g] = 0;
    s.active[g] = 1;
    s.best_f[g] = INFINITY;
    const size_t KT = s.tcols(), c0 = s.tcol(g, 0);
    for (int d = 0; d < s.P; ++d) {
        const double z = fmin(fmax((double)pw.pb[(size_t)d * pw.ld + idx], c.zlb[d]), c.zub[d]);
        s.z[(size_t)d * s.kk + g] = z;
        const double th = decode(z, (c.logmask >> d) & 1u);
        s.tht[(size_t)d * KT + c0] = th;  // slot 0: gradient point
        if (s.f32) s.thf[(size_t)d * KT + c0] = (float)th;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);  // every lane: the same sum
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

// After an adjoint launch at the accepted points (theta in tht slot 0, loss lnew, gradient gth):
// convert the gradient to z, push (s, y) into the history, keep the best point.  One warp per
// candidate, lane = dimension (P <= 32).
__global__ void polish_accept_kernel(PolishState s, uint32_t logmask, int first) {
    const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= s.kk) return;  // whole warps
    const int P = s.P, k = s.kk, d = lane;
    const size_t KT = s.tcols(), c0 = s.tcol(j, 0);
    const bool on = lane < P;
    const double fnew = s.f32 ? (double)s.lnewf[j] : s.lnew[j];
    const int head = s.head[j], cnt = s.count[j];
    const bool probe = !first && s.active[j] >= 2;  // keep the point, take only the pair
    const double best = s.best_f[j];
    double sd = 0.0, yd = 0.0;
    if (on) {
        const bool lg = (logmask >> d) & 1u;
        const double th = s.tht[(size_t)d * KT + c0];
        const double gr = s.f32 ? (double)s.gthf[(size_t)d * k + j] : s.gth[(size_t)d * k + j];
        const double gz = lg ? th * gr : gr;
        if (!first) {
            sd = s.zt[(size_t)d * k + j] - s.z[(size_t)d * k + j];
            yd = gz - s.g[(size_t)d * k + j];
            s.S[((size_t)head * P + d) * k + j] = sd;
            s.Y[((size_t)head * P + d) * k + j] = yd;
            if (!probe) s.z[(size_t)d * k + j] = s.zt[(size_t)d * k + j];
        }
        if (!probe) s.g[(size_t)d * k + j] = gz;
        if (fnew < best) s.best_th[(size_t)d * k + j] = th;
    }
    if (!first) {
        const double sy = warp_sum_d(sd * yd), yy = warp_sum_d(yd * yd), ss = warp_sum_d(sd * sd);
        if (lane == 0 && sy > 1e-14 * sqrt(ss * yy)) {  // curvature condition: keep the pair
            s.head[j] = (head + 1) % kMem;
            if (cnt < kMem) s.count[j] = cnt + 1;
        }
    }
    __syncwarp();
    if (lane == 0) {
        if (!probe) s.f[j] = fnew;
        if (fnew < best) s.best_f[j] = fnew;
    }
}

// Direction of projected L-BFGS: one warp per candidate, lane = dimension (P <= 32), dot
// products summed across the warp.  A dimension whose coordinate sits on a bound of the box with
// the gradient pointing out of the box (z at its lower bound and g > 0, or at its upper bound and
// g < 0) is held; the gradient and the stored pairs (s, y) are restricted to the free dimensions,
// each pair's curvature s.y recomputed there (a pair without positive curvature on them drops
// out), and the two-loop recursion gives d = -H g on the free dimensions, 0 on the held ones.
// With no dimension held this is plain L-BFGS.  Not a descent direction: scaled steepest descent
// on the free dimensions, history cleared.
__global__ void polish_direction_kernel(PolishState s, PsoCoeffs<double> c, double first_step) {
    const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= s.kk) return;  // whole warps
    const int P = s.P, k = s.kk;
    const bool on = lane < P;
    const double g = on ? s.g[(size_t)lane * k + j] : 0.0;
    const double z = on ? s.z[(size_t)lane * k + j] : 0.0;
    const bool held = on && ((z <= c.zlb[lane] && g > 0.0) || (z >= c.zub[lane] && g < 0.0));
    const bool fr = on && !held;
    const double gf = fr ? g : 0.0;
    const int cnt = s.count[j], head = s.head[j];
    double Sh[kMem], Yh[kMem], rh[kMem], a[kMem];
    int newest = -1;  // the most recent pair with curvature on the free dimensions
    double yy_newest = 0.0;
#pragma unroll
    for (int i = 0; i < kMem; ++i) {  // i-th most recent pair
        const int h = (head - 1 - i + 2 * kMem) % kMem;
        const bool use = fr && i < cnt;
        Sh[i] = use ? s.S[((size_t)h * P + lane) * k + j] : 0.0;
        Yh[i] = use ? s.Y[((size_t)h * P + lane) * k + j] : 0.0;
        rh[i] = 0.0;
        if (i < cnt) {
            const double sy = warp_sum_d(Sh[i] * Yh[i]), yy = warp_sum_d(Yh[i] * Yh[i]),
                         ss = warp_sum_d(Sh[i] * Sh[i]);
            if (sy > 1e-14 * sqrt(ss * yy) && sy > 0.0) {
                rh[i] = 1.0 / sy;
                if (newest < 0) {
                    newest = i;
                    yy_newest = yy;
                }
            }
        }
    }
    double q = gf;
#pragma unroll
    for (int i = 0; i < kMem; ++i) {
        if (rh[i] != 0.0) {
            a[i] = rh[i] * warp_sum_d(Sh[i] * q);
            q -= a[i] * Yh[i];
        }
    }
    if (newest >= 0) {
        q *= 1.0 / (rh[newest] * yy_newest);
    } else {
        const double gmax = warp_max_d(fabs(q));
        q *= gmax > 0.0 ? first_step / gmax : 0.0;
    }
#pragma unroll
    for (int i = kMem - 1; i >= 0; --i) {
        if (rh[i] != 0.0) {
            const double b = rh[i] * warp_sum_d(Yh[i] * q);
            q += (a[i] - b) * Sh[i];
        }
    }
    const double gd = -warp_sum_d(q * g);
    double dir = -q;
    if (!(gd < 0.0)) {  // not a descent direction: restart along the scaled steepest descent
        const double gmax = warp_max_d(fabs(gf));
        dir = -(gmax > 0.0 ? first_step / gmax : 0.0) * gf;
        if (lane == 0) s.count[j] = 0;
    }
    if (on) s.d[(size_t)lane * k + j] = dir;
}

// The trial points z + 2^-t d, clamped to the box and decoded: one thread per (dimension, trial
// column), so that the decodes (an exp each on log dimensions) run side by side.
__global__ void polish_trials_kernel(PolishState s, PsoCoeffs<double> c) {
    const int k = s.k, kt = k * kTrials;
    const size_t KT = s.tcols();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)s.P * KT) return;
    const size_t col = i % KT;
    const int d = (int)(i / KT), wi = (int)(col / kt), r = (int)(col % kt);
    const int t = r / k, g = wi * k + r % k;
    const double alpha = ldexp(1.0, -t);
    const double zn = fmin(fmax(s.z[(size_t)d * s.kk + g] + alpha * s.d[(size_t)d * s.kk + g], c.zlb[d]), c.zub[d]);
    const double th = decode(zn, (c.logmask >> d) & 1u);
    s.tht[i] = th;
    if (s.f32) s.thf[i] = (float)th;
}

// Armijo choice among the evaluated trials; the accepted theta goes to trial slot 0 and z to zt.
// One warp per candidate: lane t tests trial t, lane d decodes dimension d.
__global__ void polish_select_kernel(PolishState s, PsoCoeffs<double> c) {
    const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= s.kk) return;  // whole warps
    const int P = s.P, k = s.kk, d = lane;
    const size_t KT = s.tcols();
    const bool on = lane < P;
    const double f0 = s.f[j];
    const double gd = warp_sum_d(on ? s.g[(size_t)d * k + j] * s.d[(size_t)d * k + j] : 0.0);
    double ft = INFINITY;
    bool armijo = false;
    if (lane < kTrials) {
        const size_t ct = s.tcol(j, lane);
        ft = s.f32 ? (double)s.ftf[ct] : s.ft[ct];
        armijo = ft <= f0 + 1e-4 * ldexp(1.0, -lane) * gd;
    }
    const unsigned ok = __ballot_sync(0xFFFFFFFFu, armijo);
    int pick = ok ? __ffs(ok) - 1 : -1;  // the largest step that satisfies the Armijo condition
    if (pick < 0) {  // else the lowest trial below f0 (the first of equals)
        double fb = ft < f0 ? ft : INFINITY;
        int tb = ft < f0 ? lane : 32;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double fo = __shfl_xor_sync(0xFFFFFFFFu, fb, o);
            const int to = __shfl_xor_sync(0xFFFFFFFFu, tb, o);
            if (fo < fb || (fo == fb && to < tb)) {
                fb = fo;
                tb = to;
            }
        }
        pick = tb < 32 ? tb : -1;
    }
    // No trial lowers the loss: on a badly scaled valley the first steps can only lower it by
    // less than the FP32 evaluation resolves.  Instead of stopping, the candidate stays put and
    // takes the gradient at a probe point, the longest trial step whose loss rose by at most
    // 1e-4 relative, whose (s, y) pair gives the next direction more curvature.  kProbes failures
    // in a row stop the candidate for good.
    const int active = s.active[j];  // 0 stopped, 1 moving, 1 + n slot 0 holds the n-th probe in a row
    const unsigned near = __ballot_sync(0xFFFFFFFFu, lane < kTrials && ft <= f0 + 1e-4 * fabs(f0));
    __syncwarp();
    int probe = -1;
    if (pick >= 0 && active) {
        if (lane == 0) s.active[j] = 1;
    } else {
        if (active >= 1 && active <= kProbes) probe = near ? __ffs(near) - 1 : kTrials - 1;
        if (lane == 0) s.active[j] = probe >= 0 ? active + 1 : 0;
        pick = -1;
    }
    if (!on) return;
    double zn;
    if (pick >= 0 || probe >= 0) {
        const int t = pick >= 0 ? pick : probe;
        zn = fmin(fmax(s.z[(size_t)d * k + j] + ldexp(1.0, -t) * s.d[(size_t)d * k + j], c.zlb[d]), c.zub[d]);
    } else {
        zn = s.z[(size_t)d * k + j];
    }
    s.zt[(size_t)d * k + j] = zn;
    const double th = decode(zn, (c.logmask >> d) & 1u);
    const size_t c0 = s.tcol(j, 0);
    s.tht[(size_t)d * KT + c0] = th;
    if (s.f32) s.thf[(size_t)d * KT + c0] = (float)th;
}

// Each window's best candidate (one block per window): theta, FP64 loss and sum of squared
// errors (for R^2) into res[window].
__global__ void polish_pick_kernel(const PolishWin* __restrict__ tab, ModelDev m, PolishState s, ResultDev* res) {
    extern __shared__ double dsm[];
    __shared__ double wf[32];
    __shared__ int wi[32];
    const int tid = threadIdx.x, B = blockDim.x, k = s.k, win = blockIdx.x, g0 = win * k;
    const WindowDev w = tab[win].w;
    const double* yd = tab[win].o.yd;
    for (int i = tid, span = obs_span(w, m); i < span; i += B) dsm[i] = yd[i];
    double f = tid < k ? s.best_f[g0 + tid] : INFINITY;
    int j = tid < k ? tid : INT_MAX;
    warp_min_pair(f, j);
    if ((tid & 31) == 0) {
        wf[tid >> 5] = f;
        wi[tid >> 5] = j;
    }
    __syncthreads();
    if (tid < 32) {
        double f2 = tid < (B + 31) / 32 ? wf[tid] : INFINITY;
        int j2 = tid < (B + 31) / 32 ? wi[tid] : INT_MAX;
        warp_min_pair(f2, j2);
        if (tid == 0 && j2 < k) {
            double sse = 0.0, fl = 0.0;
            const double* th = s.best_th + g0 + j2;
            const int ld = s.kk;
            switch (m.cost) {
                case COST_MSE: fl = fitness_f64<COST_MSE>(w, m, dsm, th, ld, &sse); break;
                case COST_MXSE: fl = fitness_f64<COST_MXSE>(w, m, dsm, th, ld, &sse); break;
                case COST_MAE: fl = fitness_f64<COST_MAE>(w, m, dsm, th, ld, &sse); break;
                default: fl = fitness_f64<COST_MAPE>(w, m, dsm, th, ld, &sse); break;
            }
            ResultDev* r = res + win;
            for (int d = 0; d < m.P; ++d) r->theta[d] = th[(size_t)d * ld];
            r->loss = fl;
            r->sse = sse;
            r->index = s.cand[g0 + j2];
            r->loss_search = (double)tab[win].pbf[s.cand[g0 + j2]];
            r->count = k;
        }
    }
}

PolishState carve(double* base, int P, int k, int nw, int f32) {
    PolishState s{};
    s.P = P;
    s.k = k;
    s.nw = nw;
    s.kk = k * nw;
    s.f32 = f32;
    const int kk = s.kk;
    const size_t pk = (size_t)P * kk;
    double* q = base;
    s.z = q; q += pk;
    s.g = q; q += pk;
    s.d = q; q += pk;
    s.zt = q; q += pk;
    s.gth = q; q += pk;
    s.best_th = q; q += pk;
    s.tht = q; q += pk * kTrials;
    s.S = q; q += pk * kMem;
    s.Y = q; q += pk * kMem;
    s.f = q; q += kk;
    s.ft = q; q += (size_t)kk * kTrials;
    s.best_f = q; q += kk;
    s.lnew = q; q += kk;
    float* fq = (float*)q;
    s.thf = fq; fq += pk * kTrials;
    s.ftf = fq; fq += (size_t)kk * kTrials;
    s.gthf = fq; fq += pk;
    s.lnewf = fq; fq += kk;
    int* iq = (int*)fq;
    s.head = iq; iq += kk;
    s.count = iq; iq += kk;
    s.active = iq; iq += kk;
    s.cand = iq;
    return s;
}

}  // namespace

// k here is the number of candidates over all windows (nw * k of launch_polish).
size_t polish_scratch_doubles(int P, int k) {
    const size_t pk = (size_t)P * k;
    const size_t floats = pk * (kTrials + 1) + (size_t)k * (kTrials + 1);
    return pk * (6 + kTrials + 2 * kMem) + (size_t)k * (kTrials + 3) + (floats + 1) / 2 + 2 * (size_t)k + 8;
}

size_t polish_ckpt_floats(int n_max, int k, const ModelDev& m) {
    const size_t kpad = ((size_t)k + 31) / 32 * 32;  // the adjoint's vectors, padded to whole warps
    return (size_t)(n_max - 1) * (m.ird ? 5 : 4) * kpad;  // F_IRD: R's misfit too
}

int polish_trials() { return kTrials; }

cudaError_t launch_polish(const PolishWin* tab, int nw, int n_max, const WindowDev& w, const ObsDev& o,
                          const ModelDev& m, const PsoCoeffs<double>& c, const unsigned long long* keys, int k,
                          int iters, double first_step, int precision, double* scratch, void* ckpt, int ckpt_every,
                          ResultDev* res, cudaStream_t st) {
    const int P = m.P;
    const bool f32 = precision == 32;
    if (nw < 1 || nw > 65535 || (!f32 && nw != 1)) return cudaErrorInvalidValue;
    PolishState s = carve(scratch, P, k, nw, f32 ? 1 : 0);
    const int kk = s.kk, kt = k * kTrials;
    const long long KT = (long long)kk * kTrials;
    const long long ck_ws = (long long)polish_ckpt_floats(n_max, k, m);
    // loss and gradient at every candidate's accepted point (trial slot 0 of its window)
    auto grad_at_slot0 = [&]() {
        return f32 ? launch_loss_grad_f32_tab(tab, nw, n_max, m, s.thf, kt, (int)KT, k, s.lnewf, k, s.gthf, k, kk,
                                              (float*)ckpt, ck_ws, st)
                   : launch_loss_grad_f64(w, m, o, s.tht, kt, k, s.lnew, s.gth, k, nullptr, (double*)ckpt,
                                          ckpt_every, st);
    };
    (void)cudaGetLastError();
    const unsigned grid = (unsigned)((kk + 127) / 128);
    const unsigned grid_warps = (unsigned)((32 * (size_t)kk + 127) / 128);  // a warp per candidate
    polish_init_kernel<<<grid, 128, 0, st>>>(s, tab, keys, c);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = grad_at_slot0();
    if (e == cudaSuccess) {
        polish_accept_kernel<<<grid_warps, 128, 0, st>>>(s, c.logmask, 1);
        e = cudaGetLastError();
    }
    const unsigned grid_trials = (unsigned)(((size_t)P * KT + 127) / 128);
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        polish_direction_kernel<<<grid_warps, 128, 0, st>>>(s, c, first_step);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            polish_trials_kernel<<<grid_trials, 128, 0, st>>>(s, c);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = f32 ? launch_eval_f32_tab(tab, nw, n_max, m, s.thf, kt, (int)KT, kt, s.ftf, kt, 128, st)
                    : launch_eval_f64(w, m, o, s.tht, kt, kt, s.ft, 64, nullptr, st);
        if (e != cudaSuccess) break;
        polish_select_kernel<<<grid_warps, 128, 0, st>>>(s, c);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = grad_at_slot0();
        if (e != cudaSuccess) break;
        polish_accept_kernel<<<grid_warps, 128, 0, st>>>(s, c.logmask, 0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int block = ((k + 31) / 32) * 32;
    WindowDev wmax{};
    wmax.n_obs = n_max;
    const size_t sm = (size_t)obs_span(wmax, m) * sizeof(double);
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(polish_pick_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    polish_pick_kernel<<<(unsigned)nw, block, sm, st>>>(tab, m, s, res);
    return cudaGetLastError();
}

}  // namespace sird
