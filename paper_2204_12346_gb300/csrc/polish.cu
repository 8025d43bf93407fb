// polish.cu -- L-BFGS polish of the best PSO candidates with a parallel line search.
//
// PSO (Sec. 3.3) needs no gradient; near its optimum the swarm resolves the loss only as far
// as its search does.  The discrete adjoint gives the exact gradient of the FP64 loss, so the
// k best personal bests are refined by L-BFGS in the search coordinates (z = ln theta on log
// dimensions, where dL/dz = theta dL/dtheta), positions clamped to the box.  Each iteration:
//   1. direction d = -H g by the two-loop recursion over the last kMem (s, y) pairs,
//   2. kTrials trial points z + 2^-q d (q = 0..kTrials-1) for every candidate, evaluated in ONE
//      launch -- an evaluation of a few candidates is latency-bound, so 16 trials cost about
//      what one does,
//   3. the largest step that satisfies the Armijo condition (else the best trial if it lowers
//      the loss, else the candidate stops),
//   4. the gradient at the accepted point (adjoint launch) and the history update.
// The best point ever evaluated is re-scored in FP64 (the paper's operation order) and reported.
// Precision 64 evaluates the trials and the gradient in FP64; precision 32 uses the compensated
// FP32 evaluation and the FP32 adjoint (about 15x faster per iteration) while the L-BFGS
// algebra stays in FP64.
#include <cmath>

#include "kernels.h"

namespace sird {

namespace {

constexpr int kMem = 8;
constexpr int kTrials = 16;

// Per-candidate state, structure of arrays with candidate j at [.. * k + j].
struct PolishState {
    double *z, *g, *f, *d, *zt, *tht, *ft, *S, *Y, *rho, *best_f, *best_th, *gth, *lnew;
    float *thf, *ftf, *gthf, *lnewf;  // FP32 mode: trial thetas, their losses, gradient, loss
    int *head, *count, *active, *cand;
    int P, k, f32;
};

__device__ __forceinline__ double decode(double z, bool lg) { return lg ? exp(z) : z; }

__global__ void polish_init_kernel(PolishState s, const unsigned long long* __restrict__ keys, const float* __restrict__ pb,
                                   int ld, uint32_t logmask) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s.k) return;
    const int idx = (int)(keys[j] & 0xFFFFFFFFu);
    s.cand[j] = idx;
    s.head[j] = 0;
    s.count[j] = 0;
    s.active[j] = 1;
    s.best_f[j] = INFINITY;
    for (int d = 0; d < s.P; ++d) {
        const double z = (double)pb[(size_t)d * ld + idx];
        s.z[(size_t)d * s.k + j] = z;
        const double th = decode(z, (logmask >> d) & 1u);
        s.tht[(size_t)d * s.k * kTrials + j] = th;  // slot 0: gradient point
        if (s.f32) s.thf[(size_t)d * s.k * kTrials + j] = (float)th;
    }
}

// After an adjoint launch at the accepted points (theta in tht slot 0, loss lnew, gradient gth):
// convert the gradient to z, push (s, y) into the history, keep the best point.
__global__ void polish_accept_kernel(PolishState s, uint32_t logmask, int first) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s.k) return;
    const int P = s.P, k = s.k, kt = k * kTrials;
    const double fnew = s.f32 ? (double)s.lnewf[j] : s.lnew[j];
    double sy = 0.0, yy = 0.0, ss = 0.0;
    for (int d = 0; d < P; ++d) {
        const bool lg = (logmask >> d) & 1u;
        const double th = s.tht[(size_t)d * kt + j];
        const double gr = s.f32 ? (double)s.gthf[(size_t)d * k + j] : s.gth[(size_t)d * k + j];
        const double gz = lg ? th * gr : gr;
        if (!first) {
            const double sd = s.zt[(size_t)d * k + j] - s.z[(size_t)d * k + j];
            const double yd = gz - s.g[(size_t)d * k + j];
            sy += sd * yd;
            yy += yd * yd;
            ss += sd * sd;
            s.S[((size_t)s.head[j] * P + d) * k + j] = sd;
            s.Y[((size_t)s.head[j] * P + d) * k + j] = yd;
        }
        s.g[(size_t)d * k + j] = gz;
    }
    if (!first) {
        for (int d = 0; d < P; ++d) s.z[(size_t)d * k + j] = s.zt[(size_t)d * k + j];
        if (sy > 1e-14 * sqrt(ss * yy)) {  // curvature condition: keep the pair
            s.rho[(size_t)s.head[j] * k + j] = 1.0 / sy;
            s.head[j] = (s.head[j] + 1) % kMem;
            if (s.count[j] < kMem) ++s.count[j];
        }
    }
    s.f[j] = fnew;
    if (fnew < s.best_f[j]) {
        s.best_f[j] = fnew;
        for (int d = 0; d < P; ++d) s.best_th[(size_t)d * k + j] = s.tht[(size_t)d * kt + j];
    }
}

// Two-loop recursion and the trial points z + 2^-q d, clamped to the box.
__global__ void polish_direction_kernel(PolishState s, PsoCoeffs<double> c, double first_step) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s.k) return;
    const int P = s.P, k = s.k;
    double q[kMaxParams], a[kMem];
    for (int d = 0; d < P; ++d) q[d] = s.g[(size_t)d * k + j];
    const int cnt = s.count[j];
    for (int i = 0; i < cnt; ++i) {
        const int h = (s.head[j] - 1 - i + 2 * kMem) % kMem;
        double dot = 0.0;
        for (int d = 0; d < P; ++d) dot += s.S[((size_t)h * P + d) * k + j] * q[d];
        a[i] = s.rho[(size_t)h * k + j] * dot;
        for (int d = 0; d < P; ++d) q[d] -= a[i] * s.Y[((size_t)h * P + d) * k + j];
    }
    if (cnt > 0) {
        const int h = (s.head[j] - 1 + kMem) % kMem;
        double yy = 0.0;
        for (int d = 0; d < P; ++d) yy += s.Y[((size_t)h * P + d) * k + j] * s.Y[((size_t)h * P + d) * k + j];
        const double gamma = 1.0 / (s.rho[(size_t)h * k + j] * yy);
        for (int d = 0; d < P; ++d) q[d] *= gamma;
    } else {
        double gmax = 0.0;
        for (int d = 0; d < P; ++d) gmax = fmax(gmax, fabs(q[d]));
        const double sc = gmax > 0.0 ? first_step / gmax : 0.0;
        for (int d = 0; d < P; ++d) q[d] *= sc;
    }
    for (int i = cnt - 1; i >= 0; --i) {
        const int h = (s.head[j] - 1 - i + 2 * kMem) % kMem;
        double dot = 0.0;
        for (int d = 0; d < P; ++d) dot += s.Y[((size_t)h * P + d) * k + j] * q[d];
        const double b = s.rho[(size_t)h * k + j] * dot;
        for (int d = 0; d < P; ++d) q[d] += (a[i] - b) * s.S[((size_t)h * P + d) * k + j];
    }
    double gd = 0.0;
    for (int d = 0; d < P; ++d) {
        s.d[(size_t)d * k + j] = -q[d];
        gd -= q[d] * s.g[(size_t)d * k + j];
    }
    if (!(gd < 0.0)) {  // not a descent direction: restart along the scaled steepest descent
        double gmax = 0.0;
        for (int d = 0; d < P; ++d) gmax = fmax(gmax, fabs(s.g[(size_t)d * k + j]));
        const double sc = gmax > 0.0 ? first_step / gmax : 0.0;
        for (int d = 0; d < P; ++d) s.d[(size_t)d * k + j] = -sc * s.g[(size_t)d * k + j];
        s.count[j] = 0;
    }
}

// The trial points z + 2^-t d, clamped to the box and decoded: one thread per (dimension, trial,
// candidate), so that the decodes (an exp each on log dimensions) run side by side.
__global__ void polish_trials_kernel(PolishState s, PsoCoeffs<double> c) {
    const int k = s.k, kt = k * kTrials;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.P * kt) return;
    const int j = i % k, t = (i / k) % kTrials, d = i / kt;
    const double alpha = ldexp(1.0, -t);
    const double zn = fmin(fmax(s.z[(size_t)d * k + j] + alpha * s.d[(size_t)d * k + j], c.zlb[d]), c.zub[d]);
    const double th = decode(zn, (c.logmask >> d) & 1u);
    s.tht[(size_t)d * kt + (size_t)t * k + j] = th;
    if (s.f32) s.thf[(size_t)d * kt + (size_t)t * k + j] = (float)th;
}

// Armijo choice among the evaluated trials; the accepted theta goes to trial slot 0 and z to zt.
// One thread per (dimension, candidate): each makes the candidate's (identical) choice and
// decodes its own dimension; the dimension-0 thread records whether the candidate stops.
__global__ void polish_select_kernel(PolishState s, PsoCoeffs<double> c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.P * s.k) return;
    const int P = s.P, k = s.k, kt = k * kTrials;
    const int j = i % k, dd = i / k;
    const double f0 = s.f[j];
    double gd = 0.0;
    for (int d = 0; d < P; ++d) gd += s.g[(size_t)d * k + j] * s.d[(size_t)d * k + j];
    int pick = -1;
    double fbest = f0;
    int tbest = -1;
    for (int t = 0; t < kTrials; ++t) {
        const double ft = s.f32 ? (double)s.ftf[(size_t)t * k + j] : s.ft[(size_t)t * k + j];
        if (pick < 0 && ft <= f0 + 1e-4 * ldexp(1.0, -t) * gd) pick = t;
        if (ft < fbest) {
            fbest = ft;
            tbest = t;
        }
    }
    if (pick < 0) pick = tbest;  // no Armijo step: take the lowest trial if it improves
    if (pick < 0 || !s.active[j]) {
        // a candidate stops for good; its other threads reach pick = -1 as well, whichever value
        // of active[j] they read, since the trial choice above is the same in all of them
        if (dd == 0) s.active[j] = 0;
        pick = -1;
    }
    const int d = dd;
    double zn;
    if (pick >= 0) {
        zn = fmin(fmax(s.z[(size_t)d * k + j] + ldexp(1.0, -pick) * s.d[(size_t)d * k + j], c.zlb[d]), c.zub[d]);
    } else {
        zn = s.z[(size_t)d * k + j];
    }
    s.zt[(size_t)d * k + j] = zn;
    const double th = decode(zn, (c.logmask >> d) & 1u);
    s.tht[(size_t)d * kt + j] = th;
    if (s.f32) s.thf[(size_t)d * kt + j] = (float)th;
}

// Best candidate: theta, FP64 loss and sum of squared errors (for R^2) into *res.
__global__ void polish_pick_kernel(WindowDev w, ModelDev m, ObsDev o, PolishState s, const float* __restrict__ pbf,
                                   ResultDev* res) {
    extern __shared__ double dsm[];
    __shared__ double wf[32];
    __shared__ int wi[32];
    const int tid = threadIdx.x, B = blockDim.x, k = s.k;
    for (int i = tid, span = obs_span(w, m); i < span; i += B) dsm[i] = o.yd[i];
    double f = tid < k ? s.best_f[tid] : INFINITY;
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
            const double* th = s.best_th + j2;
            switch (m.cost) {
                case COST_MSE: fl = fitness_f64<COST_MSE>(w, m, dsm, th, k, &sse); break;
                case COST_MXSE: fl = fitness_f64<COST_MXSE>(w, m, dsm, th, k, &sse); break;
                case COST_MAE: fl = fitness_f64<COST_MAE>(w, m, dsm, th, k, &sse); break;
                default: fl = fitness_f64<COST_MAPE>(w, m, dsm, th, k, &sse); break;
            }
            for (int d = 0; d < m.P; ++d) res->theta[d] = th[(size_t)d * k];
            res->loss = fl;
            res->sse = sse;
            res->index = s.cand[j2];
            res->loss_search = (double)pbf[s.cand[j2]];
            res->count = k;
        }
    }
}

PolishState carve(double* base, int P, int k, int f32) {
    PolishState s{};
    s.P = P;
    s.k = k;
    s.f32 = f32;
    const size_t pk = (size_t)P * k;
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
    s.rho = q; q += (size_t)k * kMem;
    s.f = q; q += k;
    s.ft = q; q += (size_t)k * kTrials;
    s.best_f = q; q += k;
    s.lnew = q; q += k;
    float* fq = (float*)q;
    s.thf = fq; fq += pk * kTrials;
    s.ftf = fq; fq += (size_t)k * kTrials;
    s.gthf = fq; fq += pk;
    s.lnewf = fq; fq += k;
    int* iq = (int*)fq;
    s.head = iq; iq += k;
    s.count = iq; iq += k;
    s.active = iq; iq += k;
    s.cand = iq;
    return s;
}

}  // namespace

size_t polish_scratch_doubles(int P, int k) {
    const size_t pk = (size_t)P * k;
    const size_t floats = pk * (kTrials + 1) + (size_t)k * (kTrials + 1);
    return pk * (6 + kTrials + 2 * kMem) + (size_t)k * (kMem + kTrials + 3) + (floats + 1) / 2 + 2 * (size_t)k + 8;
}

int polish_trials() { return kTrials; }

cudaError_t launch_polish(const WindowDev& w, const ModelDev& m, const ObsDev& o, const PsoCoeffs<double>& c,
                          const unsigned long long* keys, int k, const float* pb, const float* pbf, int ld, int iters,
                          double first_step, int precision, double* scratch, void* ckpt, int ckpt_every,
                          ResultDev* res, cudaStream_t st) {
    const int P = m.P;
    const bool f32 = precision == 32;
    PolishState s = carve(scratch, P, k, f32 ? 1 : 0);
    const unsigned grid = (unsigned)((k + 127) / 128);
    const int kt = k * kTrials;
    auto grad_at_slot0 = [&]() {
        return f32 ? launch_loss_grad_f32(w, m, o, s.thf, kt, k, s.lnewf, s.gthf, k, nullptr, (float*)ckpt, st)
                   : launch_loss_grad_f64(w, m, o, s.tht, kt, k, s.lnew, s.gth, k, nullptr, (double*)ckpt,
                                          ckpt_every, st);
    };
    (void)cudaGetLastError();
    polish_init_kernel<<<grid, 128, 0, st>>>(s, keys, pb, ld, c.logmask);
    cudaError_t e = cudaGetLastError();
    // loss and gradient at the starting points (trial slot 0 holds their theta)
    if (e == cudaSuccess) e = grad_at_slot0();
    if (e == cudaSuccess) {
        polish_accept_kernel<<<grid, 128, 0, st>>>(s, c.logmask, 1);
        e = cudaGetLastError();
    }
    const unsigned grid_trials = (unsigned)((P * kt + 127) / 128), grid_dims = (unsigned)((P * k + 127) / 128);
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        polish_direction_kernel<<<grid, 128, 0, st>>>(s, c, first_step);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            polish_trials_kernel<<<grid_trials, 128, 0, st>>>(s, c);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = f32 ? launch_eval_f32(w, m, o, s.thf, kt, kt, s.ftf, 128, nullptr, st)
                    : launch_eval_f64(w, m, o, s.tht, kt, kt, s.ft, 64, nullptr, st);
        if (e != cudaSuccess) break;
        polish_select_kernel<<<grid_dims, 128, 0, st>>>(s, c);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = grad_at_slot0();
        if (e != cudaSuccess) break;
        polish_accept_kernel<<<grid, 128, 0, st>>>(s, c.logmask, 0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int block = ((k + 31) / 32) * 32;
    polish_pick_kernel<<<1, block, (size_t)obs_span(w, m) * sizeof(double), st>>>(w, m, o, s, pbf, res);
    return cudaGetLastError();
}

}  // namespace sird
