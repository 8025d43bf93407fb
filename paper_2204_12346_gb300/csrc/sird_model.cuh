// sird_model.cuh -- per-particle Euler integration of eq. (SIRD) and the window loss.
//
// One thread integrates one particle's trajectory in registers; the window's observations
// sit in shared memory.  Two arithmetic forms:
//
//  FP32 (fitness_f32): the state is carried as C = N - S (everyone ever infected), I and D.
//   Per step, with cb = dt*beta/N, a = dt*(gamma+mu), dm = dt*mu and S = N - C:
//       g = cb*S - a ;  C += cb*I*S ;  D += dm*I ;  I += g*I
//   which is the explicit Euler step of eq. (SIRD) rearranged (R is not needed for F_D: it
//   only receives gamma*I).  Over thousands of steps plain FP32 rounding of these updates
//   drifts by more than 1e-5 in the loss, so the state is compensated where it pays:
//     - I: the rounding error of r = fma(g, I, I) is recovered exactly as fma(g, I, I - r)
//       (I - r is exact) and summed into a low part that is folded back once a day;
//     - C and D: the day's increments are summed apart from the totals and folded in once a
//       day, C with an exact TwoSum into a (hi, lo) pair;
//     - the loss is a Kahan sum whose terms e^2 (|e|/y for MAPE) enter unrounded, the
//       compensation subtracted within the product's FMA.
//   Nine FP32 instructions per step; the dependence chain through I is one FMA per step.
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
    float I0f;
    float cbn_h, cbn_l; // dt/N = cbn_h + cbn_l
    float dt_h, dt_l;   // dt = dt_h + dt_l
    // F_IRD (Sec. 3.1): the reported I and R series' ranges max - min (1 for a flat series) used by
    // the min-max normalisation, their reciprocals, their counts of nonzero values, R0 split
    double rng_I, rng_R, rng_D;
    float inv_rng_I, inv_rng_R, inv_rng_D;
    int n_kept_I, n_kept_R;
    float R0h, R0l;
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

// ---------------------------------------------------------------- FP32

template <int COST>
struct LossF32 {
    Kahan sum;
    float mx = 0.f;
    __device__ __forceinline__ void add(float e, float invy) {
        if (COST == COST_MSE) sum.add_prod(e, e);
        else if (COST == COST_MAE) sum.add(fabsf(e));
        else if (COST == COST_MAPE) sum.add_prod(fabsf(e), invy);
        else mx = fmaxf(mx, __fmul_rn(e, e));
    }
    __device__ __forceinline__ float result(int n, int n_kept) const {
        if (COST == COST_MSE || COST == COST_MAE) return __fdiv_rn(sum.sum, (float)n);
        if (COST == COST_MAPE) return n_kept > 0 ? __fdiv_rn(__fmul_rn(100.f, sum.sum), (float)n_kept) : 0.f;
        return mx;
    }
};

// One Euler step in the C-form (see the file comment).  cday / dday are the day's increments;
// Il collects the rounding errors of I.
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

// Folds the day's increments into the totals and returns e_i = y_i - Dhat_i.
struct DayStateF32 {
    float Ch, Cl, Sday, Dh;
    __device__ __forceinline__ void init(const WindowDev& w, float I0, float y0) {
        two_sum(I0, w.RD0h, Ch, Cl);
        Cl = __fadd_rn(Cl, w.RD0l);
        Sday = __fadd_rn(__fsub_rn(w.Nh, Ch), __fsub_rn(w.Nl, Cl));
        Dh = y0;
    }
    __device__ __forceinline__ float close_day(const WindowDev& w, float cday, float dday, float y, float& I,
                                               float& Il) {
        // I: fold the low part in (|I| >= |Il|, so Fast2Sum is exact)
        const float si = __fadd_rn(I, Il);
        Il = __fsub_rn(Il, __fsub_rn(si, I));
        I = si;
        float s, e;
        two_sum(Ch, cday, s, e);
        Ch = s;
        Cl = __fadd_rn(Cl, e);
        Sday = __fadd_rn(__fsub_rn(w.Nh, Ch), __fsub_rn(w.Nl, Cl));
        Dh = __fadd_rn(Dh, dday);
        return __fsub_rn(y, Dh);
    }
};

// F_IRD^C (Sec. 3.1): the cost of each of I, R, D against its reported series, errors divided by
// the series' range (min-max normalisation; MAPE unnormalised), and the largest of the three.
// R is carried as a compensated (hi, lo) pair with its day increments summed apart, like C.
// Both beta forms, any steps per day; cb is formed per step as in fitness_f32.
template <int COST>
__device__ float fitness_f32_ird(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                                 const float* __restrict__ invys, const float* th, int stride) {
    const int spd = m.spd, n = w.n_obs, L = n - 1, steps = L * spd, ps = obs_stride(n);
    const float *yI = ys + ps, *yR = ys + 2 * ps, *iyI = invys + ps, *iyR = invys + 2 * ps;
    const bool ramp = m.beta_form == BETA_RAMP;
    const int gi = ramp ? 4 : m.K, K = ramp ? 1 : m.K;
    const float gam = th[gi * stride], mu = th[(gi + 1) * stride];
    float I = m.fit_I0 ? th[(gi + 2) * stride] : w.I0f;
    float Il = 0.f;
    const float gm = __fadd_rn(gam, mu);
    const float a = __fmaf_rn(gm, w.dt_h, __fmul_rn(gm, w.dt_l));
    const float dm = __fmaf_rn(mu, w.dt_h, __fmul_rn(mu, w.dt_l));
    const float dr = __fmaf_rn(gam, w.dt_h, __fmul_rn(gam, w.dt_l));
    float rb1 = 0.f, rb2 = 0.f, rt1 = 0.f, rt2 = 0.f, slope = 0.f;
    if (ramp) {
        rb1 = th[0];
        rb2 = th[stride];
        const float ta = th[2 * stride], tb = th[3 * stride];
        rt1 = fminf(ta, tb);
        rt2 = fmaxf(ta, tb);
        slope = (rt2 > rt1) ? __fdiv_rn(__fsub_rn(rb2, rb1), __fsub_rn(rt2, rt1)) : 0.f;
    }
    const float dtf = __fadd_rn(w.dt_h, w.dt_l);
    DayStateF32 ds;
    ds.init(w, I, ys[0]);
    float Rh = w.R0h, Rl = w.R0l;
    LossF32<COST> lI, lR, lD;
    auto observe = [&](int day, float eD) {
        const float eI = __fsub_rn(yI[day], I);
        const float eR = __fsub_rn(__fsub_rn(yR[day], Rh), Rl);
        if (COST == COST_MAPE) {
            lI.add(eI, iyI[day]);
            lR.add(eR, iyR[day]);
            lD.add(eD, invys[day]);
        } else {
            lI.add(__fmul_rn(eI, w.inv_rng_I), 0.f);
            lR.add(__fmul_rn(eR, w.inv_rng_R), 0.f);
            lD.add(__fmul_rn(eD, w.inv_rng_D), 0.f);
        }
    };
    observe(0, 0.f);  // e_D(0) = 0: D0 is the first observation
    int seg = 0, next_b = (!ramp && K > 1) ? segment_start(1, steps, K) : INT_MAX;
    float cb = ramp ? 0.f : __fmaf_rn(th[0], w.cbn_h, __fmul_rn(th[0], w.cbn_l));
    int k = 0;
    for (int day = 1; day <= L; ++day) {
        float cday = 0.f, dday = 0.f, rday = 0.f;
        for (int s = 0; s < spd; ++s, ++k) {
            if (ramp) {
                const float t = __fmul_rn((float)k, dtf);
                const float beta = (t < rt1) ? rb1 : ((t < rt2) ? __fmaf_rn(slope, __fsub_rn(t, rt1), rb1) : rb2);
                cb = __fmaf_rn(beta, w.cbn_h, __fmul_rn(beta, w.cbn_l));
            } else {
                while (k == next_b) {
                    ++seg;
                    cb = __fmaf_rn(th[seg * stride], w.cbn_h, __fmul_rn(th[seg * stride], w.cbn_l));
                    next_b = (seg + 1 < K) ? segment_start(seg + 1, steps, K) : INT_MAX;
                }
            }
            rday = __fmaf_rn(dr, I, rday);  // R' = gamma I, from the state at the start of the step
            euler_f32(cb, a, dm, ds.Sday, cday, dday, I, Il);
        }
        const float eD = ds.close_day(w, cday, dday, ys[day], I, Il);
        float sr, er;
        two_sum(Rh, rday, sr, er);
        Rh = sr;
        Rl = __fadd_rn(Rl, er);
        observe(day, eD);
    }
    const float cI = lI.result(n, w.n_kept_I), cR = lR.result(n, w.n_kept_R), cD = lD.result(n, w.n_kept);
    float c = cI;
    if (cR > c) c = cR;
    if (cD > c) c = cD;
    return c;
}

// Loss of one parameter vector, theta_d at th[d*stride].  ys / invys: observations and their
// reciprocals (0 where y == 0) in shared memory.  SPD > 0 fixes steps per day at compile time.
template <int SPD, int COST>
__device__ float fitness_f32(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                             const float* __restrict__ invys, const float* th, int stride) {
    if (m.ird) return fitness_f32_ird<COST>(w, m, ys, invys, th, stride);
    const int spd = SPD > 0 ? SPD : m.spd;
    const int L = w.n_obs - 1;
    const int steps = L * spd;
    const int gi = (m.beta_form == BETA_RAMP) ? 4 : m.K;
    const float gam = th[gi * stride], mu = th[(gi + 1) * stride];
    float I = m.fit_I0 ? th[(gi + 2) * stride] : w.I0f;
    float Il = 0.f;
    const float gm = __fadd_rn(gam, mu);
    const float a = __fmaf_rn(gm, w.dt_h, __fmul_rn(gm, w.dt_l));
    const float dm = __fmaf_rn(mu, w.dt_h, __fmul_rn(mu, w.dt_l));
    DayStateF32 ds;
    ds.init(w, I, ys[0]);
    LossF32<COST> loss;  // day 0: e_0 = y_0 - D_0 = 0 contributes nothing

    if (m.beta_form == BETA_RAMP) {
        // eq. (beta): beta1 before t1, linear to beta2 on [t1, t2), beta2 after (t1 <= t2 by swap)
        const float b1 = th[0], b2 = th[stride];
        const float ta = th[2 * stride], tb = th[3 * stride];
        const float t1 = fminf(ta, tb), t2 = fmaxf(ta, tb);
        const float slope = (t2 > t1) ? __fdiv_rn(__fsub_rn(b2, b1), __fsub_rn(t2, t1)) : 0.f;
        const float dtf = __fadd_rn(w.dt_h, w.dt_l);
        int k = 0;
        for (int day = 1; day <= L; ++day) {
            float cday = 0.f, dday = 0.f;
            for (int s = 0; s < spd; ++s, ++k) {
                const float t = __fmul_rn((float)k, dtf);
                float beta = (t < t1) ? b1 : ((t < t2) ? __fmaf_rn(slope, __fsub_rn(t, t1), b1) : b2);
                const float cb = __fmaf_rn(beta, w.cbn_h, __fmul_rn(beta, w.cbn_l));
                euler_f32(cb, a, dm, ds.Sday, cday, dday, I, Il);
            }
            loss.add(ds.close_day(w, cday, dday, ys[day], I, Il), COST == COST_MAPE ? invys[day] : 0.f);
        }
        return loss.result(w.n_obs, w.n_kept);
    }

    // Segment-major: every segment runs its whole days through one straight-line unrolled day
    // body (a single coefficient cb per day keeps the step chain short); a day split by a
    // segment start is finished step by step.  Several segments may start on one day.
    const int K = m.K;
    int k = 0, day = 0, in_day = 0;
    float cday = 0.f, dday = 0.f;
    for (int seg = 0; seg < K; ++seg) {
        const float b = th[seg * stride];
        const float cb = __fmaf_rn(b, w.cbn_h, __fmul_rn(b, w.cbn_l));
        const int kend = segment_start(seg + 1, steps, K);
        while (in_day != 0 && k < kend) {  // finish a day begun by the previous segment
            euler_f32(cb, a, dm, ds.Sday, cday, dday, I, Il);
            ++k;
            if (++in_day == spd) {
                ++day;
                in_day = 0;
                loss.add(ds.close_day(w, cday, dday, ys[day], I, Il), COST == COST_MAPE ? invys[day] : 0.f);
                cday = 0.f;
                dday = 0.f;
            }
        }
        while (k + spd <= kend) {  // whole days
            if (SPD > 0) {
#pragma unroll
                for (int s = 0; s < (SPD > 0 ? SPD : 1); ++s) euler_f32(cb, a, dm, ds.Sday, cday, dday, I, Il);
            } else {
                for (int s = 0; s < spd; ++s) euler_f32(cb, a, dm, ds.Sday, cday, dday, I, Il);
            }
            k += spd;
            ++day;
            loss.add(ds.close_day(w, cday, dday, ys[day], I, Il), COST == COST_MAPE ? invys[day] : 0.f);
            cday = 0.f;
            dday = 0.f;
        }
        while (k < kend) {  // start a day the next segment finishes
            euler_f32(cb, a, dm, ds.Sday, cday, dday, I, Il);
            ++k;
            ++in_day;
        }
    }
    return loss.result(w.n_obs, w.n_kept);
}

// ---------------------------------------------------------------- FP32, two particles per thread
// The same arithmetic for two parameter vectors of one window at once in packed f32x2 form:
// every lane performs exactly fitness_f32's operations in the same order, so each loss equals
// fitness_f32's bit for bit, while one instruction advances both trajectories.

__device__ __forceinline__ void euler_f32x2(F2 cb, F2 na, F2 dm, F2 Sday, F2& cday, F2& dday, F2& I, F2& Il) {
    const F2 S = sub2(Sday, cday);
    const F2 g = fma2(cb, S, na);
    const F2 t = mul2(cb, I);
    cday = fma2(t, S, cday);
    dday = fma2(dm, I, dday);
    const F2 r = fma2(g, I, I);
    Il = fma2(g, I, add2(Il, sub2(I, r)));
    I = r;
}

struct DayStateF32x2 {
    F2 Ch, Cl, Sday, Dh, Nh, Nl;
    __device__ __forceinline__ void init(const WindowDev& w, float I0a, float I0b, float y0) {
        float ha, la, hb, lb;
        two_sum(I0a, w.RD0h, ha, la);
        two_sum(I0b, w.RD0h, hb, lb);
        Ch = f2(ha, hb);
        Cl = add2(f2(la, lb), f2(w.RD0l));
        Nh = f2(w.Nh);
        Nl = f2(w.Nl);
        Sday = add2(sub2(Nh, Ch), sub2(Nl, Cl));
        Dh = f2(y0);
    }
    __device__ __forceinline__ F2 close_day(F2 cday, F2 dday, float y, F2& I, F2& Il) {
        const F2 si = add2(I, Il);
        Il = sub2(Il, sub2(si, I));
        I = si;
        F2 s, e;
        two_sum2(Ch, cday, s, e);
        Ch = s;
        Cl = add2(Cl, e);
        Sday = add2(sub2(Nh, Ch), sub2(Nl, Cl));
        Dh = add2(Dh, dday);
        return sub2(f2(y), Dh);
    }
};

template <int COST>
struct LossF32x2 {
    Kahan2 sum;
    float mxa = 0.f, mxb = 0.f;
    __device__ __forceinline__ void add(F2 e, float invy) {
        if (COST == COST_MSE) sum.add_prod(e, e);
        else if (COST == COST_MAE) sum.add(abs2(e));
        else if (COST == COST_MAPE) sum.add_prod(abs2(e), f2(invy));
        else {
            const F2 e2 = mul2(e, e);
            mxa = fmaxf(mxa, f2lo(e2));
            mxb = fmaxf(mxb, f2hi(e2));
        }
    }
    __device__ __forceinline__ void result(int n, int n_kept, float& fa, float& fb) const {
        if (COST == COST_MXSE) {
            fa = mxa;
            fb = mxb;
            return;
        }
        LossF32<COST> la, lb;
        la.sum.sum = f2lo(sum.sum);
        lb.sum.sum = f2hi(sum.sum);
        fa = la.result(n, n_kept);
        fb = lb.result(n, n_kept);
    }
};

// eq. (beta) for one particle at step k, and its cb = dt beta / N, as fitness_f32 computes them.
struct RampCoefF32 {
    float b1, b2, t1, t2, slope;
    __device__ __forceinline__ void init(const float* th, int stride) {
        b1 = th[0];
        b2 = th[stride];
        const float ta = th[2 * stride], tb = th[3 * stride];
        t1 = fminf(ta, tb);
        t2 = fmaxf(ta, tb);
        slope = (t2 > t1) ? __fdiv_rn(__fsub_rn(b2, b1), __fsub_rn(t2, t1)) : 0.f;
    }
    __device__ __forceinline__ float cb(float t, const WindowDev& w) const {
        const float beta = (t < t1) ? b1 : ((t < t2) ? __fmaf_rn(slope, __fsub_rn(t, t1), b1) : b2);
        return __fmaf_rn(beta, w.cbn_h, __fmul_rn(beta, w.cbn_l));
    }
};

// F_IRD^C for two parameter vectors in packed form: each lane performs fitness_f32_ird's
// operations in the same order.
template <int COST>
__device__ void fitness_f32x2_ird(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                                  const float* __restrict__ invys, const float* tha, const float* thb, int stride,
                                  float& fa, float& fb) {
    const int spd = m.spd, n = w.n_obs, L = n - 1, steps = L * spd, ps = obs_stride(n);
    const float *yI = ys + ps, *yR = ys + 2 * ps, *iyI = invys + ps, *iyR = invys + 2 * ps;
    const bool ramp = m.beta_form == BETA_RAMP;
    const int gi = ramp ? 4 : m.K, K = ramp ? 1 : m.K;
    const F2 gam = f2(tha[gi * stride], thb[gi * stride]), mu = f2(tha[(gi + 1) * stride], thb[(gi + 1) * stride]);
    F2 I = m.fit_I0 ? f2(tha[(gi + 2) * stride], thb[(gi + 2) * stride]) : f2(w.I0f);
    F2 Il = f2(0.f);
    const F2 gm = add2(gam, mu);
    const F2 dth = f2(w.dt_h), dtl = f2(w.dt_l);
    const F2 a = fma2(gm, dth, mul2(gm, dtl));
    const F2 na = F2{a.v ^ 0x8000000080000000ull};
    const F2 dm = fma2(mu, dth, mul2(mu, dtl));
    const F2 dr = fma2(gam, dth, mul2(gam, dtl));
    const F2 cbnh = f2(w.cbn_h), cbnl = f2(w.cbn_l);
    RampCoefF32 ra{}, rb{};
    if (ramp) {
        ra.init(tha, stride);
        rb.init(thb, stride);
    }
    const float dtf = __fadd_rn(w.dt_h, w.dt_l);
    DayStateF32x2 ds;
    ds.init(w, f2lo(I), f2hi(I), ys[0]);
    F2 Rh = f2(w.R0h), Rl = f2(w.R0l);
    LossF32x2<COST> lI, lR, lD;
    const F2 sI = f2(w.inv_rng_I), sR = f2(w.inv_rng_R), sD = f2(w.inv_rng_D);
    auto observe = [&](int day, F2 eD) {
        const F2 eI = sub2(f2(yI[day]), I);
        const F2 eR = sub2(sub2(f2(yR[day]), Rh), Rl);
        if (COST == COST_MAPE) {
            lI.add(eI, iyI[day]);
            lR.add(eR, iyR[day]);
            lD.add(eD, invys[day]);
        } else {
            lI.add(mul2(eI, sI), 0.f);
            lR.add(mul2(eR, sR), 0.f);
            lD.add(mul2(eD, sD), 0.f);
        }
    };
    observe(0, f2(0.f));
    int seg = 0, next_b = (!ramp && K > 1) ? segment_start(1, steps, K) : INT_MAX;
    F2 cb = f2(0.f);
    if (!ramp) {
        const F2 b = f2(tha[0], thb[0]);
        cb = fma2(b, cbnh, mul2(b, cbnl));
    }
    int k = 0;
    for (int day = 1; day <= L; ++day) {
        F2 cday = f2(0.f), dday = f2(0.f), rday = f2(0.f);
        for (int s = 0; s < spd; ++s, ++k) {
            if (ramp) {
                const float t = __fmul_rn((float)k, dtf);
                cb = f2(ra.cb(t, w), rb.cb(t, w));
            } else {
                while (k == next_b) {
                    ++seg;
                    const F2 b = f2(tha[seg * stride], thb[seg * stride]);
                    cb = fma2(b, cbnh, mul2(b, cbnl));
                    next_b = (seg + 1 < K) ? segment_start(seg + 1, steps, K) : INT_MAX;
                }
            }
            rday = fma2(dr, I, rday);
            euler_f32x2(cb, na, dm, ds.Sday, cday, dday, I, Il);
        }
        const F2 eD = ds.close_day(cday, dday, ys[day], I, Il);
        F2 sr, er;
        two_sum2(Rh, rday, sr, er);
        Rh = sr;
        Rl = add2(Rl, er);
        observe(day, eD);
    }
    float cIa, cIb, cRa, cRb, cDa, cDb;
    lI.result(n, w.n_kept_I, cIa, cIb);
    lR.result(n, w.n_kept_R, cRa, cRb);
    lD.result(n, w.n_kept, cDa, cDb);
    fa = cIa;
    if (cRa > fa) fa = cRa;
    if (cDa > fa) fa = cDa;
    fb = cIb;
    if (cRb > fb) fb = cRb;
    if (cDb > fb) fb = cDb;
}

// Losses of two parameter vectors (theta_d at tha[d*stride], thb[d*stride]).
template <int SPD, int COST>
__device__ void fitness_f32x2(const WindowDev& w, const ModelDev& m, const float* __restrict__ ys,
                              const float* __restrict__ invys, const float* tha, const float* thb, int stride,
                              float& fa, float& fb) {
    if (m.ird) {
        fitness_f32x2_ird<COST>(w, m, ys, invys, tha, thb, stride, fa, fb);
        return;
    }
    const int spd = SPD > 0 ? SPD : m.spd;
    if (m.beta_form == BETA_RAMP) {
        // the ramp changes beta every step: each lane's cb is formed as in fitness_f32, the
        // step itself is packed
        const int L = w.n_obs - 1;
        const F2 gam = f2(tha[4 * stride], thb[4 * stride]), mu = f2(tha[5 * stride], thb[5 * stride]);
        F2 I = m.fit_I0 ? f2(tha[6 * stride], thb[6 * stride]) : f2(w.I0f);
        F2 Il = f2(0.f);
        const F2 gm = add2(gam, mu);
        const F2 dth = f2(w.dt_h), dtl = f2(w.dt_l);
        const F2 a = fma2(gm, dth, mul2(gm, dtl));
        const F2 na = F2{a.v ^ 0x8000000080000000ull};
        const F2 dm = fma2(mu, dth, mul2(mu, dtl));
        RampCoefF32 ra, rb;
        ra.init(tha, stride);
        rb.init(thb, stride);
        const float dtf = __fadd_rn(w.dt_h, w.dt_l);
        DayStateF32x2 ds;
        ds.init(w, f2lo(I), f2hi(I), ys[0]);
        LossF32x2<COST> loss;
        int k = 0;
        for (int day = 1; day <= L; ++day) {
            F2 cday = f2(0.f), dday = f2(0.f);
            for (int s = 0; s < spd; ++s, ++k) {
                const float t = __fmul_rn((float)k, dtf);
                euler_f32x2(f2(ra.cb(t, w), rb.cb(t, w)), na, dm, ds.Sday, cday, dday, I, Il);
            }
            loss.add(ds.close_day(cday, dday, ys[day], I, Il), COST == COST_MAPE ? invys[day] : 0.f);
        }
        loss.result(w.n_obs, w.n_kept, fa, fb);
        return;
    }
    const int L = w.n_obs - 1;
    const int steps = L * spd;
    const int K = m.K;
    const F2 gam = f2(tha[K * stride], thb[K * stride]), mu = f2(tha[(K + 1) * stride], thb[(K + 1) * stride]);
    F2 I = m.fit_I0 ? f2(tha[(K + 2) * stride], thb[(K + 2) * stride]) : f2(w.I0f);
    F2 Il = f2(0.f);
    const F2 gm = add2(gam, mu);
    const F2 dth = f2(w.dt_h), dtl = f2(w.dt_l);
    const F2 a = fma2(gm, dth, mul2(gm, dtl));
    const F2 na = F2{a.v ^ 0x8000000080000000ull};  // -a, exact
    const F2 dm = fma2(mu, dth, mul2(mu, dtl));
    const F2 cbnh = f2(w.cbn_h), cbnl = f2(w.cbn_l);
    DayStateF32x2 ds;
    ds.init(w, f2lo(I), f2hi(I), ys[0]);
    LossF32x2<COST> loss;

    int k = 0, day = 0, in_day = 0;
    F2 cday = f2(0.f), dday = f2(0.f);
    for (int seg = 0; seg < K; ++seg) {
        const F2 b = f2(tha[seg * stride], thb[seg * stride]);
        const F2 cb = fma2(b, cbnh, mul2(b, cbnl));
        const int kend = segment_start(seg + 1, steps, K);
        while (in_day != 0 && k < kend) {
            euler_f32x2(cb, na, dm, ds.Sday, cday, dday, I, Il);
            ++k;
            if (++in_day == spd) {
                ++day;
                in_day = 0;
                loss.add(ds.close_day(cday, dday, ys[day], I, Il), COST == COST_MAPE ? invys[day] : 0.f);
                cday = f2(0.f);
                dday = f2(0.f);
            }
        }
        while (k + spd <= kend) {
            if (SPD > 0) {
#pragma unroll
                for (int s = 0; s < (SPD > 0 ? SPD : 1); ++s) euler_f32x2(cb, na, dm, ds.Sday, cday, dday, I, Il);
            } else {
                for (int s = 0; s < spd; ++s) euler_f32x2(cb, na, dm, ds.Sday, cday, dday, I, Il);
            }
            k += spd;
            ++day;
            loss.add(ds.close_day(cday, dday, ys[day], I, Il), COST == COST_MAPE ? invys[day] : 0.f);
            cday = f2(0.f);
            dday = f2(0.f);
        }
        while (k < kend) {
            euler_f32x2(cb, na, dm, ds.Sday, cday, dday, I, Il);
            ++k;
            ++in_day;
        }
    }
    loss.result(w.n_obs, w.n_kept, fa, fb);
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
