// forecast.cu -- deaths forecast: the fitted window extended past its last day (Sec. 4.2).
//
// One thread per parameter vector integrates the window from its start (the same Euler
// scheme as the fitness: FP64 in the paper's operation order, or the FP32 trajectory of
// traj_f32.cuh) and `horizon` more days with the last transmission rate (the last PWC segment,
// or beta2 of the ramp), gamma and mu, writing D on the days after the window.
#include <climits>

#include "kernels.h"

namespace sird {

namespace {

// beta at step k (t = k*dt): PWC segment floor(k*K/steps_window), the last one past the
// window; the ramp of eq. (beta) otherwise.
__device__ __forceinline__ int pwc_seg(long long k, int steps_window, int K) {
    return k >= steps_window ? K - 1 : (int)((k * K) / steps_window);
}

__global__ void forecast_f64_kernel(WindowDev w, ModelDev m, const double* __restrict__ theta, int ld, int k,
                                    int horizon, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double* th = theta + j;
    const int stride = ld;
    const int spd = m.spd, L = w.n_obs - 1, steps_w = L * spd;
    const long long steps = (long long)(L + horizon) * spd;
    const int gi = (m.beta_form == BETA_RAMP) ? 4 : m.K;
    const double gam = th[gi * stride], mu = th[(gi + 1) * stride];
    const double I0 = m.fit_I0 ? th[(gi + 2) * stride] : w.I0;
    const double gm = __dadd_rn(gam, mu), dt = w.dt;
    double S = __dsub_rn(__dsub_rn(__dsub_rn(w.N, I0), w.R0), w.D0), I = I0, D = w.D0;
    double rb1 = 0, rb2 = 0, rt1 = 0, rt2 = 0;
    if (m.beta_form == BETA_RAMP) {
        rb1 = th[0];
        rb2 = th[stride];
        const double ta = th[2 * stride], tb = th[3 * stride];
        rt1 = ta < tb ? ta : tb;
        rt2 = ta < tb ? tb : ta;
    }
    for (long long s = 0; s < steps; ++s) {
        double beta;
        if (m.beta_form == BETA_RAMP) {
            const double t = __ddiv_rn((double)s, (double)spd);
            if (t < rt1) beta = rb1;
            else if (t < rt2) beta = __dadd_rn(rb1, __dmul_rn(__ddiv_rn(__dsub_rn(rb2, rb1), __dsub_rn(rt2, rt1)),
                                                              __dsub_rn(t, rt1)));
            else beta = rb2;
        } else {
            beta = th[pwc_seg(s, steps_w, m.K) * stride];
        }
        const double bN = __ddiv_rn(beta, w.N);
        const double fS = __dmul_rn(__dmul_rn(-bN, S), I);
        const double fI = __dsub_rn(__dmul_rn(__dmul_rn(bN, I), S), __dmul_rn(gm, I));
        const double fD = __dmul_rn(mu, I);
        S = __dadd_rn(S, __dmul_rn(dt, fS));
        I = __dadd_rn(I, __dmul_rn(dt, fI));
        D = __dadd_rn(D, __dmul_rn(dt, fD));
        if ((s + 1) % spd == 0) {
            const long long day = (s + 1) / spd;
            if (day > L) out[(size_t)j * horizon + (day - L - 1)] = D;
        }
    }
}

// D on the days after the window: the trajectory run with its misfit tracking -D (DTRACK), so
// that D keeps its own relative accuracy whatever the fit.
struct ForecastObs {
    int L, horizon;
    float* out;
    __device__ __forceinline__ void day_start(int, float, float, float, float, float) {}
    __device__ __forceinline__ void day_end(int day, float e, float, float, float) {
        if (day > L) out[day - L - 1] = -e;
    }
};

__global__ void forecast_f32_kernel(WindowDev w, ModelDev m, const float* __restrict__ theta, int ld, int k,
                                    int horizon, const float* __restrict__ yf, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const int L = w.n_obs - 1;
    ForecastObs o{L, horizon, out + (size_t)j * horizon};
    const ThetaF1 th{theta + j, ld};
    if (m.beta_form == BETA_RAMP) trajectory_f32<float, 0, true, false, true, true>(w, m, yf, nullptr, th, L + horizon, o);
    else trajectory_f32<float, 0, false, false, true, true>(w, m, yf, nullptr, th, L + horizon, o);
}

}  // namespace

cudaError_t launch_forecast(const WindowDev& w, const ModelDev& m, const void* theta, int ld, int k, int horizon,
                            const float* yf, void* out, int precision, cudaStream_t s) {
    if (k <= 0 || horizon <= 0) return cudaSuccess;
    (void)cudaGetLastError();
    const int block = 128;
    const unsigned grid = (unsigned)((k + block - 1) / block);
    if (precision == 64)
        forecast_f64_kernel<<<grid, block, 0, s>>>(w, m, (const double*)theta, ld, k, horizon, (double*)out);
    else
        forecast_f32_kernel<<<grid, block, 0, s>>>(w, m, (const float*)theta, ld, k, horizon, yf, (float*)out);
    return cudaGetLastError();
}

}  // namespace sird
