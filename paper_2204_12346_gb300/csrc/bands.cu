// bands.cu -- ensemble statistics of repeated calibrations (Sec. 4.2).
//
// The paper repeats the calibration of a window many times and summarises the resulting
// parameter sets per day as a median and central bands holding 95%, 90% and 50% of the values,
// for beta(t), the basic reproduction number R0(t) = beta(t) / (gamma + mu) and the compartments
// over the window and its extension past the last day (the last transmission rate, gamma, mu).
//
// The fitted parameters themselves (beta's segments or the ramp's beta1, beta2, t1, t2, then gamma,
// mu and a fitted I0) get the same summary over the repetitions: the stability of the estimates
// is what the repetitions measure.
//
// Two kernels: one thread per ensemble member integrates the window and the extension in FP64
// (the paper's operation order, as the forecast) and writes per day beta, R0, S, I, R, D into
// [quantity][day][member]; then one block per (day, quantity) sorts the k member values in
// shared memory (bitonic network) and writes the median and each band's two ends.
#include <climits>

#include "kernels.h"

namespace sird {

namespace {

constexpr int kBandsThreads = 1024;

__device__ __forceinline__ int seg_past_window(long long k, int steps_window, int K) {
    return k >= steps_window ? K - 1 : (int)((k * K) / steps_window);
}

// beta at step k of the window's numbering (eq. (beta) or the PWC segments, the last one past
// the window), in the paper's operation order.
__device__ __forceinline__ double beta_at_step(const ModelDev& m, const double* th, int stride, long long k,
                                               int steps_window, double rb1, double rb2, double rt1, double rt2) {
    if (m.beta_form == BETA_RAMP) {
        const double t = __ddiv_rn((double)k, (double)m.spd);
        if (t < rt1) return rb1;
        if (t < rt2)
            return __dadd_rn(rb1, __dmul_rn(__ddiv_rn(__dsub_rn(rb2, rb1), __dsub_rn(rt2, rt1)), __dsub_rn(t, rt1)));
        return rb2;
    }
    return th[seg_past_window(k, steps_window, m.K) * stride];
}

__global__ void ensemble_traj_f64_kernel(WindowDev w, ModelDev m, const double* __restrict__ theta, int ld, int k,
                                         int n_days, double* __restrict__ traj) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double* th = theta + j;
    const int stride = ld;
    const int spd = m.spd, L = w.n_obs - 1, steps_w = L * spd;
    const long long steps = (long long)(n_days - 1) * spd;
    const int gi = (m.beta_form == BETA_RAMP) ? 4 : m.K;
    const double gam = th[gi * stride], mu = th[(gi + 1) * stride];
    const double I0 = m.fit_I0 ? th[(gi + 2) * stride] : w.I0;
    const double gm = __dadd_rn(gam, mu), dt = w.dt;
    double S = __dsub_rn(__dsub_rn(__dsub_rn(w.N, I0), w.R0), w.D0), I = I0, R = w.R0, D = w.D0;
    double rb1 = 0, rb2 = 0, rt1 = 0, rt2 = 0;
    if (m.beta_form == BETA_RAMP) {
        rb1 = th[0];
        rb2 = th[stride];
        const double ta = th[2 * stride], tb = th[3 * stride];
        rt1 = ta < tb ? ta : tb;
        rt2 = ta < tb ? tb : ta;
    }
    const size_t plane = (size_t)n_days * k;  // one quantity
    auto put = [&](int day) {
        const double b = beta_at_step(m, th, stride, (long long)day * spd, steps_w, rb1, rb2, rt1, rt2);
        const size_t o = (size_t)day * k + j;
        traj[o] = b;
        traj[plane + o] = __ddiv_rn(b, gm);
        traj[2 * plane + o] = S;
        traj[3 * plane + o] = I;
        traj[4 * plane + o] = R;
        traj[5 * plane + o] = D;
    };
    put(0);
    for (long long s = 0; s < steps; ++s) {
        const double beta = beta_at_step(m, th, stride, s, steps_w, rb1, rb2, rt1, rt2);
        const double bN = __ddiv_rn(beta, w.N);
        const double fS = __dmul_rn(__dmul_rn(-bN, S), I);
        const double fI = __dsub_rn(__dmul_rn(__dmul_rn(bN, I), S), __dmul_rn(gm, I));
        const double fR = __dmul_rn(gam, I);
        const double fD = __dmul_rn(mu, I);
        S = __dadd_rn(S, __dmul_rn(dt, fS));
        I = __dadd_rn(I, __dmul_rn(dt, fI));
        R = __dadd_rn(R, __dmul_rn(dt, fR));
        D = __dadd_rn(D, __dmul_rn(dt, fD));
        if ((s + 1) % spd == 0) put((int)((s + 1) / spd));
    }
}

// out[(q * n_days + day) * (1 + 2 n_bands) + ...] = median, then (low, high) of each band; band b
// leaves drop[b] values out at each end of the sorted k values.
__global__ void __launch_bounds__(kBandsThreads) bands_kernel(const double* __restrict__ traj, int k, int n_days,
                                                              const int* __restrict__ drop, int n_bands,
                                                              double* __restrict__ out) {
    __shared__ double v[kMaxEnsemble];
    const int day = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    const double* src = traj + ((size_t)q * n_days + day) * k;
    int n2 = 1;
    while (n2 < k) n2 <<= 1;
    for (int i = tid; i < n2; i += kBandsThreads) v[i] = i < k ? src[i] : INFINITY;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n2 / 2; i += kBandsThreads) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const double a = v[lo], b = v[hi];
                if ((a > b) == asc) {
                    v[lo] = b;
                    v[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        double* o = out + ((size_t)q * n_days + day) * (1 + 2 * n_bands);
        o[0] = (k & 1) ? v[k / 2] : __dmul_rn(__dadd_rn(v[k / 2 - 1], v[k / 2]), 0.5);
        for (int b = 0; b < n_bands; ++b) {
            o[1 + 2 * b] = v[drop[b]];
            o[2 + 2 * b] = v[k - 1 - drop[b]];
        }
    }
}

// The ramp's two change times form an unordered pair (beta follows the earlier one first), so
// their bands summarise t1 = min(t_a, t_b) and t2 = max(t_a, t_b): reordered in place in the
// parameter-major copy theta [P][k].
__global__ void ramp_times_kernel(double* __restrict__ theta, int k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double ta = theta[2 * (size_t)k + j], tb = theta[3 * (size_t)k + j];
    theta[2 * (size_t)k + j] = ta < tb ? ta : tb;
    theta[3 * (size_t)k + j] = ta < tb ? tb : ta;
}

}  // namespace

cudaError_t launch_parameter_bands(const ModelDev& m, double* theta, int k, const int* drop, int n_bands, double* out,
                                   cudaStream_t s) {
    if (k < 1 || k > kMaxEnsemble) return cudaErrorInvalidValue;
    (void)cudaGetLastError();
    if (m.beta_form == BETA_RAMP) {
        ramp_times_kernel<<<(k + 127) / 128, 128, 0, s>>>(theta, k);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // one "day" per parameter: block (0, d) sorts parameter d's k values
    bands_kernel<<<dim3(1u, (unsigned)m.P), kBandsThreads, 0, s>>>(theta, k, 1, drop, n_bands, out);
    return cudaGetLastError();
}

size_t ensemble_traj_bytes(int k, int n_days) { return (size_t)kBandQuantities * n_days * k * sizeof(double); }

cudaError_t launch_ensemble_bands(const WindowDev& w, const ModelDev& m, const double* theta, int k, int n_days,
                                  const int* drop, int n_bands, double* traj, double* out, cudaStream_t s) {
    if (k < 1 || k > kMaxEnsemble || n_days < 1) return cudaErrorInvalidValue;
    (void)cudaGetLastError();
    ensemble_traj_f64_kernel<<<(k + 127) / 128, 128, 0, s>>>(w, m, theta, k, k, n_days, traj);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bands_kernel<<<dim3((unsigned)n_days, kBandQuantities), kBandsThreads, 0, s>>>(traj, k, n_days, drop, n_bands, out);
    return cudaGetLastError();
}

}  // namespace sird
