// sird_model.cuh -- per-particle Euler integration of eq. (SIRD) and the window loss.
//
// One thread integrates one particle's trajectory in registers; the window's observations
// sit in shared memory.  Two arithmetic forms:
//
//  FP32 (fitness_f32, fitness_f32x2): the trajectory of traj_f32.cuh -- Q = S + I and the day's
//   growth rate G = cb Q - a carried as (hi, lo) pairs, two FMAs for g and one for I per step
//   with I's rounding error recovered exactly, the day's sum of I exact to ~1e-9 from exact
//   per-step decrements, the deaths' misfit e = y - Dhat followed directly -- and a Kahan sum of
//   the daily costs whose terms e^2 (|e|/y for MAPE) enter unrounded.  One trajectory per
//   thread, or two in packed f32x2 pairs with identical results.
//
//  FP64 (fitness_f64): S, I, D in double precision in the paper's own operation order, with
//   no contraction into FMA, so the trajectory is the one the equations prescribe bit for bit.
//
// Window and coefficient conventions (Sec. 3.1): n = tau+1 observations on days 0..L, Euler
// starts from D0 = y_0, observation i is compared with the state after i*spd steps,
// e_i = y_i - Dhat_i.  PWC segment j covers steps [ceil(j*S/K), ceil((j+1)*S/K)).
#pragma once

#include <climits>

#include "device_common.cuh"

namespace sird {

enum : int { COST_MSE = 0, COST_MXSE = 1, COST_MAE = 2, COST_MAPE = 3 };
enum : int { BETA_PWC = 0, BETA_RAMP = 1 };

// Window constants shared by every particle of a launch.
struct WindowDev {
    int n_obs;      // tau+1
    int n_kept;     // observations with y != 0 (MAPE denominator)
    double N, I0, R0, D0, dt;
    float Nh, Nl;       // N = Nh + Nl
    float RD0h, RD0l;   // R0 + D0 = RD0h + RD0l
    float I0f, I0l;     // a given I0 = I0f + I0l
    float cbn_h, cbn_l; // dt/N = cbn_h + cbn_l
    float dt_h, dt_l;   // dt = dt_h + dt_l
    // F_IRD (Sec. 3.1): the reported I and R series' ranges max - min (1 for a flat series) used by
    // the min-max normalisation, their reciprocals, their counts of nonzero values, R0 split
    double rng_I, rng_R, rng_D;
    float inv_rng_I, inv_rng_R, inv_rng_D;
    int n_kept_I, n_kept_R;
    float R0h, R0l;
    // the FP32 trajectory: Q0 = S0 + I0 = N - R0 - D0 as a pair, and y_R0 - R0 (F_IRD)
    float Q0h, Q0l;
    float eR0;
};

struct ModelDev {
    int P, K, spd, beta_form, fit_I0, cost;
    int ird;  // objective F_IRD (else F_D)
};

// Observation layout: the series are stacked D | I | R (I and R only for F_IRD), each padded to
// obs_stride(n_obs) entries, in every float and double copy.
__host__ __device__ __forceinline__ int obs_stride(int n_obs) { return (n_obs + 3) & ~3; }
// Entries of one staged copy of the observations: n (F_D) or the three stacked series (F_IRD);
// obs_span_pad rounds the F_D case up to obs_stride.
__host__ __device__ __forceinline__ int obs_span(const WindowDev& w, const ModelDev& m) {
    return m.ird ? 3 * obs_stride(w.n_obs) : w.n_obs;
}
__host__ __device__ __forceinline__ int obs_span_pad(const WindowDev& w, const ModelDev& m) {
    return (m.ird ? 3 : 1) * obs_stride(w.n_obs);
}

// First step of PWC segment j: ceil(j*steps/K).
__device__ __forceinline__ int segment_start(int j, int steps, int K) {
    return (int)(((long long)j * steps + K - 1) / K);
}

}  // namespace sird

#include "traj_f32.cuh"

namespace sird {

// ---------------------------------------------------------------- FP32
// The trajectory itself lives in traj_f32.cuh; here are the losses built on it.

// F_D^C (Sec. 3.1): the cost of the deaths' misfit e_i = y_i - Dhat_i over days 0..L.  LEAN:
// the calling kernel is at its register bound (see obs_lean in traj_f32.cuh).
template <class T, int COST, bool LEAN = false>
struct LossObsD {
    static constexpr bool kLeanRegs = LEAN;
    CostT<T, COST> c;
    const float* invys;
    __device__ __forceinline__ void day_start(int, T, T, T, T, T) {}
    __device__ __forceinline__ void day_end(int day, T e, T, T, T) { c.add(e, COST == COST_MAPE ? invys[day] : 0.f); }
};

// F_IRD^C (Sec. 3.1): the cost of each of I, R, D against its reported series (errors divided
// by the series' range, the min-max normalisation; MAPE on the raw values), the largest of the
// three.  ys / invys hold the series stacked D | I | R with stride obs_stride(n).
template <class T, int COST, bool LEAN = false>
struct LossObsIRD {
    static constexpr bool kLeanRegs = LEAN;
    CostT<T, COST> cI, cR, cD;
    const float *ys, *invys;
    int ps;
    float sI, sR, sD;
    __device__ __forceinline__ void day_start(int, T, T, T, T, T) {}
    __device__ __forceinline__ void day_end(int day, T e, T Ih, T Il, T eR) {
        const T eI = tsub(tsub(tsplat<T>(ys[ps + day]), Ih), Il);
        if (COST == COST_MAPE) {
            cI.add(eI, invys[ps + day]);
            cR.add(eR, invys[2 * ps + day]);
            cD.add(e, invys[day]);
        } else {
            cI.add(tmul(eI, tsplat<T>(sI)), 0.f);
            cR.add(tmul(eR, tsplat<T>(sR)), 0.f);
            cD.add(tmul(e, tsplat<T>(sD)), 0.f);
        }
    }
};

__device__ __forceinline__ float max3(float a, float b, float c) {
    float r = a;
    if (b > r) r = b;
    if (c > r) r = c;
    return r;
}

// Compile-time variant of the FP32 kernels: the cost in bits 0-1 and the form in bits 2-3
// (0: PWC beta and F_D, 1: PWC and F_IRD, 2: ramp and F_D, 3: ramp and F_IRD), so that every
// form is its own kernel with its own register allocation.
enum : int { FORM_PWC_D = 0, FORM_PWC_IRD = 1, FORM_RAMP_D = 2, FORM_RAMP_IRD = 3 };
__host__ __device__ __forceinline__ constexpr int variant_cost(int v) { return v & 3; }
__host__ __device__ __forceinline__ constexpr int variant_form(int v) { return v >> 2; }
__host__ __device__ __forceinline__ int form_of(const ModelDev& m) {
    return (m.beta_form == BETA_RAMP ? 2 : 0) + (m.ird ? 1 : 0);
}

// Losses of the vectors th (T = float: one, fa = fb; T = F2: two, one per lane); CV is the
// variant (cost | form << 2), which must match m.
template <class T, int SPD, int CV, bool LEAN, class Th>
__device__ __forceinline__ void fitness_lanes(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                                              const float* __restrict__ invys, Th th, float& fa, float& fb) {
    constexpr int COST = variant_cost(CV), FORM = variant_form(CV);
    constexpr bool RAMP = FORM >= 2, IRD = (FORM & 1) != 0;
    const int L = w.n_obs - 1;
    if constexpr (IRD) {
        LossObsIRD<T, COST, LEAN> o;
        o.cI.init();
        o.cR.init();
        o.cD.init();
        o.ys = ys;
        o.invys = invys;
        o.ps = obs_stride(w.n_obs);
        o.sI = w.inv_rng_I;
        o.sR = w.inv_rng_R;
        o.sD = w.inv_rng_D;
        if (L * (SPD > 0 ? SPD : m.spd) > kExactGrowthSteps)
            trajectory_f32<T, SPD, RAMP, true, false, true>(w, m, ys, ys + 2 * o.ps, th, L, o);
        else
            trajectory_f32<T, SPD, RAMP, true>(w, m, ys, ys + 2 * o.ps, th, L, o);
        float ia, ib, ra, rb, da, db;
        o.cI.result(w.n_obs, w.n_kept_I, ia, ib);
        o.cR.result(w.n_obs, w.n_kept_R, ra, rb);
        o.cD.result(w.n_obs, w.n_kept, da, db);
        fa = max3(ia, ra, da);
        fb = max3(ib, rb, db);
    } else {
        LossObsD<T, COST, LEAN> o;
        o.c.init();
        o.invys = invys;
        if (L * (SPD > 0 ? SPD : m.spd) > kExactGrowthSteps)
            trajectory_f32<T, SPD, RAMP, false, false, true>(w, m, ys, nullptr, th, L, o);
        else
            trajectory_f32<T, SPD, RAMP, false>(w, m, ys, nullptr, th, L, o);
        o.c.result(w.n_obs, w.n_kept, fa, fb);
    }
}

// Loss of one parameter vector, theta_d at th[d*stride].  ys / invys: observations and their
// reciprocals (0 where y == 0) in shared memory.  SPD > 0 fixes steps per day at compile time;
// COST is the variant (cost | form << 2); LEAN for kernels at their register bound (same losses).
template <int SPD, int COST, bool LEAN = false>
__device__ float fitness_f32(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                             const float* __restrict__ invys, const float* th, int stride) {
    float fa, fb;
    fitness_lanes<float, SPD, COST, LEAN>(w, m, ys, invys, ThetaF1{th, stride}, fa, fb);
    return fa;
}

// Losses of two parameter vectors (theta_d at tha[d*stride], thb[d*stride]) integrated together
// in packed f32x2 form; each equals fitness_f32's loss of that vector bit for bit.
template <int SPD, int COST, bool LEAN = false>
__device__ void fitness_f32x2(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                              const float* __restrict__ invys, const float* tha, const float* thb, int stride,
                              float& fa, float& fb) {
    fitness_lanes<F2, SPD, COST, LEAN>(w, m, ys, invys, ThetaF2{tha, thb, stride}, fa, fb);
}

// One Euler step in the C-form (C = N - S carried, S = Sday - cday) with I's rounding error
// collected in Il; the adjoint re-integrates a day with it from a day-start checkpoint (its
// per-step states feed the reverse sweep, whose sensitivity to them is far below the loss's).
__device__ __forceinline__ void euler_f32(float cb, float a, float dm, float Sday, float& cday, float& dday,
                                          float& I, float& Il) {
    const float S = __fsub_rn(Sday, cday);
    const float g = __fmaf_rn(cb, S, -a);
    const float t = __fmul_rn(cb, I);
    cday = __fmaf_rn(t, S, cday);
    dday = __fmaf_rn(dm, I, dday);
    const float r = __fmaf_rn(g, I, I);
    Il = __fmaf_rn(g, I, __fadd_rn(Il, __fsub_rn(I, r)));
    I = r;
}

// ---------------------------------------------------------------- FP64

template <int COST>
struct LossF64 {
    double acc = 0.0, sse = 0.0;
    __device__ __forceinline__ void add(double y, double yhat) {
        const double e = __dsub_rn(y, yhat);
        const double e2 = __dmul_rn(e, e);
        sse = __dadd_rn(sse, e2);
        if (COST == COST_MSE) acc = __dadd_rn(acc, e2);
        else if (COST == COST_MXSE) { if (e2 > acc) acc = e2; }
        else if (COST == COST_MAE) acc = __dadd_rn(acc, fabs(e));
        else if (y != 0.0) acc = __dadd_rn(acc, fabs(__ddiv_rn(e, y)));
    }
    __device__ __forceinline__ double result(int n, int n_kept) const {
        if (COST == COST_MSE || COST == COST_MAE) return __ddiv_rn(acc, (double)n);
        if (COST == COST_MAPE) return n_kept > 0 ? __ddiv_rn(__dmul_rn(100.0, acc), (double)n_kept) : 0.0;
        return acc;
    }
};

// One series' cost in FP64 (Sec. 3.1) with errors e = (y - yhat) / scale, accumulated in day
// order: MSE and MAE over n, MXSE the largest e^2, MAPE 100 |y - yhat| / |y| over the nonzero y.
template <int COST>
struct SeriesCostF64 {
    double acc = 0.0;
    int kept = 0;
    __device__ __forceinline__ void add(double y, double yhat, double scale) {
        const double e = __ddiv_rn(__dsub_rn(y, yhat), scale);
        if (COST == COST_MSE) acc = __dadd_rn(acc, __dmul_rn(e, e));
        else if (COST == COST_MXSE) { if (__dmul_rn(e, e) > acc) acc = __dmul_rn(e, e); }
        else if (COST == COST_MAE) acc = __dadd_rn(acc, fabs(e));
        else if (y != 0.0) {
            acc = __dadd_rn(acc, fabs(__ddiv_rn(__dsub_rn(y, yhat), y)));
            ++kept;
        }
    }
    __device__ __forceinline__ double result(int n) const {
        if (COST == COST_MSE || COST == COST_MAE) return __ddiv_rn(acc, (double)n);
        if (COST == COST_MAPE) return kept > 0 ? __ddiv_rn(__dmul_rn(100.0, acc), (double)kept) : 0.0;
        return acc;
    }
};

// F_IRD^C in FP64, the paper's operation order (R' = gamma I added after D'), no contraction.
template <int COST>
__device__ double fitness_f64_ird(const WindowDev& w, const ModelDev& m, const double* __restrict__ ys,
                                  const double* th, int stride, double* sse_out) {
    const int spd = m.spd, n = w.n_obs, L = n - 1, steps = L * spd, ps = obs_stride(n);
    const double *yI = ys + ps, *yR = ys + 2 * ps;
    const bool ramp = (m.beta_form == BETA_RAMP);
    const int gi = ramp ? 4 : m.K, K = ramp ? 1 : m.K;
    const double gam = th[gi * stride], mu = th[(gi + 1) * stride];
    const double I0 = m.fit_I0 ? th[(gi + 2) * stride] : w.I0;
    const double gm = __dadd_rn(gam, mu);
    const double dt = w.dt;
    double S = __dsub_rn(__dsub_rn(__dsub_rn(w.N, I0), w.R0), w.D0);
    double I = I0, R = w.R0, D = w.D0;
    const bool mape = COST == COST_MAPE;
    const double sI = mape ? 1.0 : w.rng_I, sR = mape ? 1.0 : w.rng_R, sD = mape ? 1.0 : w.rng_D;
    SeriesCostF64<COST> cI, cR, cD;
    double sse = 0.0;
    auto observe = [&](int day) {
        cI.add(yI[day], I, sI);
        cR.add(yR[day], R, sR);
        cD.add(ys[day], D, sD);
        const double e = __dsub_rn(ys[day], D);
        sse = __dadd_rn(sse, __dmul_rn(e, e));
    };
    observe(0);
    double rb1 = 0, rb2 = 0, rt1 = 0, rt2 = 0;
    if (ramp) {
        rb1 = th[0];
        rb2 = th[stride];
        const double ta = th[2 * stride], tb = th[3 * stride];
        rt1 = ta < tb ? ta : tb;
        rt2 = ta < tb ? tb : ta;
    }
    int seg = 0, prev_seg = -1;
    double bN = 0.0;
    int next_b = (!ramp && K > 1) ? segment_start(1, steps, K) : INT_MAX;
    for (int k = 0; k < steps; ++k) {
        if (ramp) {
            const double t = __ddiv_rn((double)k, (double)spd);
            double beta;
            if (t < rt1) beta = rb1;
            else if (t < rt2) beta = __dadd_rn(rb1, __dmul_rn(__ddiv_rn(__dsub_rn(rb2, rb1), __dsub_rn(rt2, rt1)),
                                                              __dsub_rn(t, rt1)));
            else beta = rb2;
            bN = __ddiv_rn(beta, w.N);
        } else {
            while (k == next_b) {
                ++seg;
                next_b = (seg + 1 < K) ? segment_start(seg + 1, steps, K) : INT_MAX;
            }
            if (k == 0 || seg != prev_seg) bN = __ddiv_rn(th[seg * stride], w.N);
            prev_seg = seg;
        }
        const double fS = __dmul_rn(__dmul_rn(-bN, S), I);
        const double fI = __dsub_rn(__dmul_rn(__dmul_rn(bN, I), S), __dmul_rn(gm, I));
        const double fR = __dmul_rn(gam, I);
        const double fD = __dmul_rn(mu, I);
        S = __dadd_rn(S, __dmul_rn(dt, fS));
        I = __dadd_rn(I, __dmul_rn(dt, fI));
        R = __dadd_rn(R, __dmul_rn(dt, fR));
        D = __dadd_rn(D, __dmul_rn(dt, fD));
        if ((k + 1) % spd == 0) observe((k + 1) / spd);
    }
    if (sse_out) *sse_out = sse;
    const double a = cI.result(n), b = cR.result(n), c = cD.result(n);
    double r = a;
    if (b > r) r = b;
    if (c > r) r = c;
    return r;
}

// Loss of one parameter vector in FP64 (theta_d at th[d*stride]); *sse_out gets sum e_i^2.
// Observation i is compared after i*spd steps; the sum runs over days in order.
template <int COST>
__device__ double fitness_f64(const WindowDev& w, const ModelDev& m, const double* __restrict__ ys,
                              const double* th, int stride, double* sse_out) {
    if (m.ird) return fitness_f64_ird<COST>(w, m, ys, th, stride, sse_out);
    const int spd = m.spd;
    const int L = w.n_obs - 1;
    const int steps = L * spd;
    const int gi = (m.beta_form == BETA_RAMP) ? 4 : m.K;
    const double gam = th[gi * stride], mu = th[(gi + 1) * stride];
    const double I0 = m.fit_I0 ? th[(gi + 2) * stride] : w.I0;
    const double gm = __dadd_rn(gam, mu);
    const double dt = w.dt;
    double S = __dsub_rn(__dsub_rn(__dsub_rn(w.N, I0), w.R0), w.D0);
    double I = I0, D = w.D0;
    LossF64<COST> loss;
    loss.add(ys[0], D);

    const bool ramp = (m.beta_form == BETA_RAMP);
    double rb1 = 0, rb2 = 0, rt1 = 0, rt2 = 0;
    if (ramp) {
        rb1 = th[0];
        rb2 = th[stride];
        const double ta = th[2 * stride], tb = th[3 * stride];
        rt1 = ta < tb ? ta : tb;
        rt2 = ta < tb ? tb : ta;
    }
    const int K = ramp ? 1 : m.K;
    int seg = 0;
    double bN = 0.0;
    int prev_seg = -1;
    int next_b = (!ramp && K > 1) ? segment_start(1, steps, K) : INT_MAX;
    for (int k = 0; k < steps; ++k) {
        if (ramp) {
            const double t = __ddiv_rn((double)k, (double)spd);
            double beta;
            if (t < rt1) beta = rb1;
            else if (t < rt2) beta = __dadd_rn(rb1, __dmul_rn(__ddiv_rn(__dsub_rn(rb2, rb1), __dsub_rn(rt2, rt1)),
                                                              __dsub_rn(t, rt1)));
            else beta = rb2;
            bN = __ddiv_rn(beta, w.N);
        } else {
            while (k == next_b) {
                ++seg;
                next_b = (seg + 1 < K) ? segment_start(seg + 1, steps, K) : INT_MAX;
            }
            if (k == 0 || seg != prev_seg) bN = __ddiv_rn(th[seg * stride], w.N);
            prev_seg = seg;
        }
        // eq. (SIRD): fS = -(beta/N) S I, fI = (beta/N) I S - (gamma+mu) I, fD = mu I
        const double fS = __dmul_rn(__dmul_rn(-bN, S), I);
        const double fI = __dsub_rn(__dmul_rn(__dmul_rn(bN, I), S), __dmul_rn(gm, I));
        const double fD = __dmul_rn(mu, I);
        S = __dadd_rn(S, __dmul_rn(dt, fS));
        I = __dadd_rn(I, __dmul_rn(dt, fI));
        D = __dadd_rn(D, __dmul_rn(dt, fD));
        if ((k + 1) % spd == 0) loss.add(ys[(k + 1) / spd], D);
    }
    if (sse_out) *sse_out = loss.sse;
    return loss.result(w.n_obs, w.n_kept);
}

}  // namespace sird
