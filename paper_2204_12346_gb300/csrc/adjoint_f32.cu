// adjoint_f32.cu -- FP32 loss and gradient of the discrete loss (discrete adjoint, eq. (SIRD)).
//
// Same mathematics as the FP64 adjoint: with u_{k+1} = u_k + dt f(u_k, theta), the reverse sweep
//     lambda_S <- lambda_S + cb I (lambda_I - lambda_S)
//     lambda_I <- lambda_I + cb S (lambda_I - lambda_S) - a lambda_I + dm lambda_D
//     lambda_D <- lambda_D + dL/dDhat_i                      (after the first step of day i)
// (cb = dt beta/N, a = dt (gamma + mu), dm = dt mu) accumulates
//     dL/dbeta_j = dt/N sum_{k in segment j} S_k I_k (lambda_I - lambda_S)_{k+1}
//     dL/dgamma  = -dt sum_k I_k lambda_I,{k+1}
//     dL/dmu     =  dt sum_k I_k (lambda_D - lambda_I)_{k+1}
// and dL/dI0 = lambda_I(0) - lambda_S(0) (S0 = N - I0 - R0 - D0).  For F_IRD^C the cost
// gradient of the dominant series (the first of I, R, D attaining the maximum, as the evaluation
// picks it; errors scaled by the series' range, MAPE unscaled) enters lambda_I, lambda_R or
// lambda_D on its observation days, lambda_R (constant between them) adds dt gamma lambda_R to
// lambda_I's step and dL/dgamma becomes dt sum_k I_k (lambda_R - lambda_I)_{k+1}.
//
// The forward pass is the FP32 trajectory of the evaluation kernels (traj_f32.cuh), operation for
// operation, so the loss equals the FP32 evaluation's bit for bit.  It stores the state at the
// start of every day (S, I, its low part, and the day's error e_d) in global scratch
// [day][4][M]; the reverse pass re-integrates one day at a time from it in the C-form step
// (euler_f32), staging each step's S, I and coefficient in shared memory, and sweeps the day
// backwards.  lambda_S and lambda_I carry
// their rounding errors in low parts folded in once a day (their per-step increments are tiny
// against them, so plain FP32 sums would drift by up to steps x 2^-24); the gradient's per-step
// terms are summed per day in FP32 and the day sums in FP64.
#include <climits>

#include "kernels.h"
#include "sird_model.cuh"

namespace sird {

namespace {

constexpr int kMaxSpdGeneric = 64;

__device__ __forceinline__ int seg_of_step(int k, int steps, int K) { return (int)(((long long)k * K) / steps); }

struct RampF32 {
    float b1, b2, t1, t2, slope, inv_len, dtf;
    bool swapped;
    __device__ __forceinline__ float beta(int k) const {
        const float t = __fmul_rn((float)k, dtf);
        return (t < t1) ? b1 : ((t < t2) ? __fmaf_rn(slope, __fsub_rn(t, t1), b1) : b2);
    }
    // d beta / d(beta1, beta2, t_a, t_b) at step k (t_a, t_b as given; swapped maps them back)
    __device__ __forceinline__ void dbeta(int k, float db[4]) const {
        const float t = __fmul_rn((float)k, dtf);
        float d1 = 0.f, d2 = 0.f, dt1 = 0.f, dt2 = 0.f;
        if (t < t1) {
            d1 = 1.f;
        } else if (t < t2) {
            const float sr = __fmul_rn(__fsub_rn(t, t1), inv_len);
            d1 = __fsub_rn(1.f, sr);
            d2 = sr;
            const float db21 = __fmul_rn(__fsub_rn(b2, b1), __fmul_rn(inv_len, inv_len));
            dt1 = __fmul_rn(db21, __fsub_rn(t, t2));
            dt2 = -__fmul_rn(db21, __fsub_rn(t, t1));
        } else {
            d2 = 1.f;
        }
        db[0] = d1;
        db[1] = d2;
        db[2] = swapped ? dt2 : dt1;
        db[3] = swapped ? dt1 : dt2;
    }
};

template <int COST>
__device__ __forceinline__ float grad_D(float e, float invy, int n, int n_kept, bool is_max) {
    // dL/dDhat for e = y - Dhat
    const float sg = (float)((e > 0.f) - (e < 0.f));
    if (COST == COST_MSE) return __fdiv_rn(__fmul_rn(-2.f, e), (float)n);
    if (COST == COST_MAE) return __fdiv_rn(-sg, (float)n);
    if (COST == COST_MAPE) return n_kept > 0 ? __fdiv_rn(__fmul_rn(__fmul_rn(-100.f, sg), invy), (float)n_kept) : 0.f;
    return is_max ? __fmul_rn(-2.f, e) : 0.f;
}

// dC/dyhat of one F_IRD series on a day with scaled error es = (y - yhat) s (s = 1 / range; MAPE:
// es = y - yhat unscaled, invy = 1/y) -- grad_D's formulas in the scaled error, times s.
template <int COST>
__device__ __forceinline__ float grad_series(float es, float s, float invy, int n, int n_kept, bool is_max) {
    if (COST == COST_MAPE) return grad_D<COST>(es, invy, n, n_kept, false);
    return __fmul_rn(grad_D<COST>(es, invy, n, n_kept, is_max), s);
}

// One day of Euler steps from (Sday, I, Il) with the day's coefficients; when stage is set, the
// S, I and cb each step uses are written to shared memory (stS/stI/stC at [s * B]).  Days inside
// one PWC segment run straight-line (SPD unrolled); a day holding a segment start, or the ramp
// form, updates cb step by step.  seg / next_b track the PWC segment of the day's first step.
template <int SPD, bool RAMP, bool STAGE>
__device__ __forceinline__ void day_steps(int day, int spd, int steps, int K, const float* th, int B,
                                          const RampF32& rp, float a, float dm, const WindowDev& w, float Sday,
                                          float& cday, float& dday, float& I, float& Il, int& seg, int& next_b,
                                          float& cb, float* stS, float* stI, float* stC) {
    auto cb_of = [&](float beta) { return __fmaf_rn(beta, w.cbn_h, __fmul_rn(beta, w.cbn_l)); };
    const int k0 = day * spd;
    if (!RAMP && next_b >= k0 + spd) {
        if (SPD > 0) {
#pragma unroll
            for (int s = 0; s < (SPD > 0 ? SPD : 1); ++s) {
                if (STAGE) {
                    stS[s * B] = __fsub_rn(Sday, cday);
                    stI[s * B] = I;
                    stC[s * B] = cb;
                }
                euler_f32(cb, a, dm, Sday, cday, dday, I, Il);
            }
        } else {
            for (int s = 0; s < spd; ++s) {
                if (STAGE) {
                    stS[s * B] = __fsub_rn(Sday, cday);
                    stI[s * B] = I;
                    stC[s * B] = cb;
                }
                euler_f32(cb, a, dm, Sday, cday, dday, I, Il);
            }
        }
        return;
    }
    for (int s = 0; s < spd; ++s) {
        const int k = k0 + s;
        if (RAMP) {
            cb = cb_of(rp.beta(k));
        } else {
            while (k == next_b) {
                ++seg;
                cb = cb_of(th[seg * B]);
                next_b = seg + 1 < K ? segment_start(seg + 1, steps, K) : INT_MAX;
            }
        }
        if (STAGE) {
            stS[s * B] = __fsub_rn(Sday, cday);
            stI[s * B] = I;
            stC[s * B] = cb;
        }
        euler_f32(cb, a, dm, Sday, cday, dday, I, Il);
    }
}

// Loss, gradient and the state shared by the kernels below: theta of one vector at th[d * B].
struct CoefF32 {
    float a, dm, I0;
    RampF32 rp;
};

template <bool RAMP>
__device__ __forceinline__ CoefF32 coef_f32(const WindowDev& w, const ModelDev& m, const float* th, int B) {
    CoefF32 c{};
    const int gi = RAMP ? 4 : m.K;
    const float gam = th[gi * B], mu = th[(gi + 1) * B];
    c.I0 = m.fit_I0 ? th[(gi + 2) * B] : w.I0f;
    const float gm = __fadd_rn(gam, mu);
    c.a = __fmaf_rn(gm, w.dt_h, __fmul_rn(gm, w.dt_l));
    c.dm = __fmaf_rn(mu, w.dt_h, __fmul_rn(mu, w.dt_l));
    if (RAMP) {
        RampF32& rp = c.rp;
        rp.b1 = th[0];
        rp.b2 = th[B];
        const float ta = th[2 * B], tb = th[3 * B];
        rp.swapped = ta > tb;
        rp.t1 = fminf(ta, tb);
        rp.t2 = fmaxf(ta, tb);
        rp.slope = (rp.t2 > rp.t1) ? __fdiv_rn(__fsub_rn(rp.b2, rp.b1), __fsub_rn(rp.t2, rp.t1)) : 0.f;
        rp.inv_len = (rp.t2 > rp.t1) ? __fdiv_rn(1.f, __fsub_rn(rp.t2, rp.t1)) : 0.f;
        rp.dtf = __fadd_rn(w.dt_h, w.dt_l);
    }
    return c;
}

__device__ __forceinline__ float cb_of_f32(const WindowDev& w, float beta) {
    return __fmaf_rn(beta, w.cbn_h, __fmul_rn(beta, w.cbn_l));
}

// Forward pass: the FP32 evaluation's trajectory and cost (traj_f32.cuh), so the loss equals
// the FP32 evaluation's bit for bit, plus the day-start checkpoints (S, I, its low part, and the
// day's error e_d) at ck[(day * 4 + q) * cs].  Returns the loss; e_last = e_L, imax = the MXSE
// day (the first with the largest e^2).
template <int COST>
struct CkptObs {
    static constexpr bool kWantsQ = true;  // day_start stores S = Q - I
    CostT<float, COST> c;
    const float* invys;
    float* ck;
    size_t cs;
    float emax, e_last;
    int imax;
    __device__ __forceinline__ void day_start(int day, float Qh, float Ql, float Ih, float Il, float e) {
        float* q = ck + (size_t)day * 4 * cs;
        q[0] = __fadd_rn(__fsub_rn(Qh, Ih), __fsub_rn(Ql, Il));  // S = Q - I at the day's start
        q[cs] = Ih;
        q[2 * cs] = Il;
        q[3 * cs] = e;
    }
    __device__ __forceinline__ void day_end(int day, float e, float, float, float) {
        c.add(e, COST == COST_MAPE ? invys[day] : 0.f);
        if (COST == COST_MXSE) {
            const float e2 = __fmul_rn(e, e);
            if (e2 > emax) {
                emax = e2;
                imax = day;
            }
        }
        e_last = e;
    }
};

// F_IRD forward pass: the three series' costs exactly as the FP32 evaluation forms them
// (LossObsIRD), the day-start checkpoints (S, I, its low part, D's misfit) and R's misfit of
// observation d at slot 4 of day d ([day][5][cs]); the last observation's misfits and I pair, the
// first day of each series' largest scaled e^2 (MXSE) and the dominant series (0 I, 1 R, 2 D).
template <int COST>
struct CkptObsIRD {
    static constexpr bool kWantsQ = true;
    CostT<float, COST> cI, cR, cD;
    const float *ys, *invys;
    int ps, L;
    float sI, sR, sD;
    float* ck;
    size_t cs;
    float mxI, mxR, mxD;
    int imI, imR, imD;
    float eD_last, eR_last, Ih_last, Il_last;
    __device__ __forceinline__ void day_start(int day, float Qh, float Ql, float Ih, float Il, float e) {
        float* q = ck + (size_t)day * 5 * cs;
        q[0] = __fadd_rn(__fsub_rn(Qh, Ih), __fsub_rn(Ql, Il));  // S = Q - I at the day's start
        q[cs] = Ih;
        q[2 * cs] = Il;
        q[3 * cs] = e;
    }
    __device__ __forceinline__ void day_end(int day, float e, float Ih, float Il, float eR) {
        const float eI = __fsub_rn(__fsub_rn(ys[ps + day], Ih), Il);
        float a, b, c;
        if (COST == COST_MAPE) {
            cI.add(eI, invys[ps + day]);
            cR.add(eR, invys[2 * ps + day]);
            cD.add(e, invys[day]);
            a = eI, b = eR, c = e;
        } else {
            a = __fmul_rn(eI, sI), b = __fmul_rn(eR, sR), c = __fmul_rn(e, sD);
            cI.add(a, 0.f);
            cR.add(b, 0.f);
            cD.add(c, 0.f);
        }
        if (COST == COST_MXSE) {  // the first day of each series' largest e^2 (tmaxsq's order)
            if (__fmul_rn(a, a) > mxI) mxI = __fmul_rn(a, a), imI = day;
            if (__fmul_rn(b, b) > mxR) mxR = __fmul_rn(b, b), imR = day;
            if (__fmul_rn(c, c) > mxD) mxD = __fmul_rn(c, c), imD = day;
        }
        if (day < L) ck[((size_t)day * 5 + 4) * cs] = eR;
        eD_last = e;
        eR_last = eR;
        Ih_last = Ih;
        Il_last = Il;
    }
};

template <int SPD, int COST, bool RAMP>
__device__ __forceinline__ float forward_checkpointed(const WindowDev& w, const ModelDev& m, const float* ys,
                                                      const float* invys, const float* th, int B, const CoefF32&,
                                                      float* ck, size_t cs, float& e_last, int& imax) {
    CkptObs<COST> o;
    o.c.init();
    o.invys = invys;
    o.ck = ck;
    o.cs = cs;
    o.emax = 0.f;
    o.e_last = 0.f;
    o.imax = 0;
    // the evaluation's arithmetic, including its choice of the compensated growth rate
    const int L = w.n_obs - 1;
    if (L * (SPD > 0 ? SPD : m.spd) > kExactGrowthSteps)
        trajectory_f32<float, SPD, RAMP, false, false, true>(w, m, ys, nullptr, ThetaF1{th, B}, L, o);
    else
        trajectory_f32<float, SPD, RAMP, false>(w, m, ys, nullptr, ThetaF1{th, B}, L, o);
    e_last = o.e_last;
    imax = o.imax;
    float fa, fb;
    o.c.result(w.n_obs, w.n_kept, fa, fb);
    return fa;
}

// Re-integrates one day from its checkpoint (ck as above), staging each step's S, I and cb at
// stS/stI/stC[s * B].
template <int SPD, bool RAMP, int NQ = 4>
__device__ __forceinline__ void restage_day(const WindowDev& w, const ModelDev& m, const float* th, int B,
                                            const CoefF32& cf, const float* ck, size_t cs, int day, float* stS,
                                            float* stI, float* stC) {
    const int spd = SPD > 0 ? SPD : m.spd, steps = (w.n_obs - 1) * spd, K = m.K;
    const float* c = ck + (size_t)day * NQ * cs;
    const float Sday = c[0];
    float Ir = c[cs], Ilr = c[2 * cs];
    int sg = RAMP ? 0 : seg_of_step(day * spd, steps, K);
    int nb = (!RAMP && sg + 1 < K) ? segment_start(sg + 1, steps, K) : INT_MAX;
    float cb = RAMP ? 0.f : cb_of_f32(w, th[sg * B]);
    float cday = 0.f, dday = 0.f;
    day_steps<SPD, RAMP, true>(day, spd, steps, K, th, B, cf.rp, cf.a, cf.dm, w, Sday, cday, dday, Ir, Ilr, sg, nb, cb,
                               stS, stI, stC);
}

// Adjoint state of one vector through the reverse sweep: lambda_S, lambda_I with their low parts,
// lambda_D, the segment being swept and the gradient sums.  Kept as separate scalars so that
// they stay in registers (the sums are indexed by segment and live in local memory).
struct RevF32 {
    float lS, lI, lSl, lIl, lD, lR;
    int cur, seg_lo;
};

template <int COST, bool RAMP>
__device__ __forceinline__ void rev_begin(RevF32& r, double* gacc, const WindowDev& w, const ModelDev& m,
                                          const float* invys, int steps, float e_last, int imax) {
    const int n = w.n_obs, L = n - 1;
    for (int d = 0; d < m.P; ++d) gacc[d] = 0.0;
    r.lS = r.lI = r.lSl = r.lIl = 0.f;
    r.lD = grad_D<COST>(e_last, invys[L], n, w.n_kept, imax == L);
    r.cur = RAMP ? 0 : seg_of_step(steps - 1, steps, m.K);
    r.seg_lo = RAMP ? 0 : segment_start(r.cur, steps, m.K);
}

// The reverse sweep of one staged day (steps spd-1 .. 0), then the day's folds and dL/dDhat_day
// (F_IRD: the caller adds the day's cost gradient; dr = dt gamma enters with lambda_R).
template <int SPD, int COST, bool RAMP, bool IRD = false>
__device__ __forceinline__ void rev_day(RevF32& r, double* gacc, const WindowDev& w, const ModelDev& m, const float* invys,
                                        const CoefF32& cf, int day, int steps, const float* stS, const float* stI,
                                        const float* stC, int B, float e_d, int imax, float dr = 0.f) {
    const int spd = SPD > 0 ? SPD : m.spd, K = m.K, n = w.n_obs, gi = RAMP ? 4 : K;
    const float a = cf.a;
    float pb = 0.f, pg = 0.f, pm = 0.f, pr[4] = {0.f, 0.f, 0.f, 0.f};
    // lambda_D (and lambda_R) are constant within the day
    const float dmlD = IRD ? __fmaf_rn(dr, r.lR, __fmul_rn(cf.dm, r.lD)) : __fmul_rn(cf.dm, r.lD);
#pragma unroll 4
    for (int s = spd - 1; s >= 0; --s) {
        const int k = day * spd + s;
        const float S = stS[s * B], Iv = stI[s * B], c = stC[s * B];
        if (!RAMP && k < r.seg_lo) {  // entering the previous segment (uniform across the warp)
            gacc[r.cur] += (double)pb;
            pb = 0.f;
            r.cur = seg_of_step(k, steps, K);
            r.seg_lo = segment_start(r.cur, steps, K);
        }
        const float q = __fsub_rn(r.lI, r.lS);
        const float SI = __fmul_rn(S, Iv);
        if (RAMP) {
            float db[4];
            cf.rp.dbeta(k, db);
            const float rr = __fmul_rn(SI, q);
#pragma unroll
            for (int j = 0; j < 4; ++j) pr[j] = __fmaf_rn(rr, db[j], pr[j]);
        } else {
            pb = __fmaf_rn(SI, q, pb);
        }
        pg = IRD ? __fmaf_rn(Iv, __fsub_rn(r.lI, r.lR), pg) : __fmaf_rn(Iv, r.lI, pg);
        pm = __fmaf_rn(Iv, __fsub_rn(r.lD, r.lI), pm);
        // lambda_S and lambda_I change by small increments per step; as for I in the forward
        // pass, each sum's rounding error is kept (Fast2Sum) and folded in once a day
        const float dS = __fmul_rn(__fmul_rn(c, Iv), q);
        const float dI = __fmaf_rn(__fmul_rn(c, S), q, __fmaf_rn(-a, r.lI, dmlD));
        const float rS = __fadd_rn(r.lS, dS), rI = __fadd_rn(r.lI, dI);
        r.lSl = __fadd_rn(r.lSl, __fsub_rn(dS, __fsub_rn(rS, r.lS)));
        r.lIl = __fadd_rn(r.lIl, __fsub_rn(dI, __fsub_rn(rI, r.lI)));
        r.lS = rS;
        r.lI = rI;
    }
    {
        const float fs = __fadd_rn(r.lS, r.lSl), fi = __fadd_rn(r.lI, r.lIl);
        r.lSl = __fsub_rn(r.lSl, __fsub_rn(fs, r.lS));
        r.lIl = __fsub_rn(r.lIl, __fsub_rn(fi, r.lI));
        r.lS = fs;
        r.lI = fi;
    }
    if (!IRD) r.lD = __fadd_rn(r.lD, grad_D<COST>(e_d, invys[day], n, w.n_kept, COST == COST_MXSE && imax == day));
    if (RAMP) {
#pragma unroll
        for (int j = 0; j < 4; ++j) gacc[j] += (double)pr[j];
    } else {
        gacc[r.cur] += (double)pb;
    }
    gacc[gi] += (double)pg;
    gacc[gi + 1] += (double)pm;
}

template <bool RAMP, bool IRD = false>
__device__ __forceinline__ void rev_write(const RevF32& r, const double* gacc, const WindowDev& w, const ModelDev& m, int p, float Lval,
                                          float* loss, float* grad, int ldg, float* grad_u0) {
    const int K = m.K, gi = RAMP ? 4 : K;
    const double dtN = w.dt / w.N;
    const int nbeta = RAMP ? 4 : K;
    for (int d = 0; d < nbeta; ++d) grad[(size_t)d * ldg + p] = (float)(gacc[d] * dtN);
    grad[(size_t)gi * ldg + p] = (float)(-w.dt * gacc[gi]);
    grad[(size_t)(gi + 1) * ldg + p] = (float)(w.dt * gacc[gi + 1]);
    const float lS = __fadd_rn(r.lS, r.lSl);
    const float lI = __fadd_rn(r.lI, r.lIl);
    if (m.fit_I0) grad[(size_t)(gi + 2) * ldg + p] = __fsub_rn(lI, lS);
    loss[p] = Lval;
    if (grad_u0) {
        grad_u0[p] = lS;
        grad_u0[(size_t)ldg + p] = lI;
        grad_u0[2 * (size_t)ldg + p] = IRD ? r.lR : 0.f;
        grad_u0[3 * (size_t)ldg + p] = r.lD;
    }
}

// One thread per parameter vector: forward pass, then per day (last to first) re-integration
// into shared memory and the reverse sweep.  Any form and steps per day.
template <int SPD, int COST, bool RAMP>
__device__ __forceinline__ void loss_grad_f32_body(const WindowDev& w, const ModelDev& m, const ObsDev& o,
                                                   const float* __restrict__ theta, int ld, int M,
                                                   float* __restrict__ loss, float* __restrict__ grad, int ldg,
                                                   float* __restrict__ grad_u0, float* __restrict__ ckpt, int blk) {
    extern __shared__ float smem[];
    const int B = blockDim.x, tid = threadIdx.x, P = m.P;
    const int n = w.n_obs;
    const int spd = SPD > 0 ? SPD : m.spd;
    float* ys = smem;
    float* invys = ys + ((n + 3) & ~3);
    float* th_all = invys + ((n + 3) & ~3);
    float* stS = th_all + P * B + tid;  // per-step staging [spd][B] x 3
    float* stI = stS + spd * B;
    float* stC = stI + spd * B;
    for (int i = tid; i < n; i += B) {
        ys[i] = o.yf[i];
        invys[i] = o.invyf[i];
    }
    const int p = blk * B + tid;
    const bool active = p < M;
    if (active)
        for (int d = 0; d < P; ++d) th_all[d * B + tid] = theta[(size_t)d * ld + p];
    __syncthreads();
    if (!active) return;
    const float* th = th_all + tid;
    const int L = n - 1, steps = L * spd;
    const CoefF32 cf = coef_f32<RAMP>(w, m, th, B);
    float e_last;
    int imax;
    float* ck = ckpt + p;
    const float Lval = forward_checkpointed<SPD, COST, RAMP>(w, m, ys, invys, th, B, cf, ck, (size_t)M, e_last, imax);
    RevF32 r;
    double gacc[kMaxParams];
    rev_begin<COST, RAMP>(r, gacc, w, m, invys, steps, e_last, imax);
    for (int day = L - 1; day >= 0; --day) {
        restage_day<SPD, RAMP>(w, m, th, B, cf, ck, (size_t)M, day, stS, stI, stC);
        rev_day<SPD, COST, RAMP>(r, gacc, w, m, invys, cf, day, steps, stS, stI, stC, B, ck[((size_t)day * 4 + 3) * M],
                                 imax);
    }
    rev_write<RAMP>(r, gacc, w, m, p, Lval, loss, grad, ldg, grad_u0);
}

// F_IRD^C: one thread per parameter vector, as loss_grad_f32_body, with the three series staged
// (D | I | R, stride obs_stride(n)), checkpoints [day][5][cs] and the dominant series' gradient
// injected day by day.
template <int SPD, int COST, bool RAMP>
__device__ __forceinline__ void loss_grad_f32_ird_body(const WindowDev& w, const ModelDev& m, const ObsDev& o,
                                                       const float* __restrict__ theta, int ld, int M,
                                                       float* __restrict__ loss, float* __restrict__ grad, int ldg,
                                                       float* __restrict__ grad_u0, float* __restrict__ ckpt, int blk) {
    extern __shared__ float smem[];
    const int B = blockDim.x, tid = threadIdx.x, P = m.P;
    const int n = w.n_obs, ps = obs_stride(n), span = 3 * ps;
    const int spd = SPD > 0 ? SPD : m.spd;
    float* ys = smem;
    float* invys = ys + span;
    float* th_all = invys + span;
    float* stS = th_all + P * B + tid;  // per-step staging [spd][B] x 3
    float* stI = stS + spd * B;
    float* stC = stI + spd * B;
    for (int i = tid; i < span; i += B) {
        ys[i] = o.yf[i];
        invys[i] = o.invyf[i];
    }
    const int p = blk * B + tid;
    const bool active = p < M;
    if (active)
        for (int d = 0; d < P; ++d) th_all[d * B + tid] = theta[(size_t)d * ld + p];
    __syncthreads();
    if (!active) return;
    const float* th = th_all + tid;
    const int L = n - 1, steps = L * spd, gi = RAMP ? 4 : m.K;
    const CoefF32 cf = coef_f32<RAMP>(w, m, th, B);
    const float gam = th[gi * B];
    const float dr = __fmaf_rn(gam, w.dt_h, __fmul_rn(gam, w.dt_l));
    float* ck = ckpt + p;
    const size_t cs = (size_t)M;
    CkptObsIRD<COST> ob;
    ob.cI.init();
    ob.cR.init();
    ob.cD.init();
    ob.ys = ys;
    ob.invys = invys;
    ob.ps = ps;
    ob.L = L;
    ob.sI = w.inv_rng_I;
    ob.sR = w.inv_rng_R;
    ob.sD = w.inv_rng_D;
    ob.ck = ck;
    ob.cs = cs;
    ob.mxI = ob.mxR = ob.mxD = 0.f;
    ob.imI = ob.imR = ob.imD = -1;
    ob.eD_last = ob.eR_last = ob.Ih_last = ob.Il_last = 0.f;
    // the evaluation's arithmetic, including its choice of the compensated growth rate
    if (steps > kExactGrowthSteps)
        trajectory_f32<float, SPD, RAMP, true, false, true>(w, m, ys, ys + 2 * ps, ThetaF1{th, B}, L, ob);
    else
        trajectory_f32<float, SPD, RAMP, true>(w, m, ys, ys + 2 * ps, ThetaF1{th, B}, L, ob);
    float ia, ib, ra, rb, da, db;
    ob.cI.result(n, w.n_kept_I, ia, ib);
    ob.cR.result(n, w.n_kept_R, ra, rb);
    ob.cD.result(n, w.n_kept, da, db);
    float Lval = ia;
    int which = 0;  // the dominant series, the first of I, R, D on ties (max3's order)
    if (ra > Lval) Lval = ra, which = 1;
    if (da > Lval) Lval = da, which = 2;
    // the dominant series' cost gradient on observation d from the misfits there
    const bool mape = COST == COST_MAPE;
    auto inject = [&](RevF32& r, int d, float Ih, float Il, float eR, float eD) {
        if (which == 0) {
            const float eI = __fsub_rn(__fsub_rn(ys[ps + d], Ih), Il);
            const float g = grad_series<COST>(mape ? eI : __fmul_rn(eI, w.inv_rng_I), w.inv_rng_I, invys[ps + d], n,
                                              w.n_kept_I, d == ob.imI);
            float sh, sl;  // lambda_I carries a low part: add with TwoSum
            two_sum(r.lI, g, sh, sl);
            r.lI = sh;
            r.lIl = __fadd_rn(r.lIl, sl);
        } else if (which == 1) {
            r.lR = __fadd_rn(r.lR, grad_series<COST>(mape ? eR : __fmul_rn(eR, w.inv_rng_R), w.inv_rng_R,
                                                      invys[2 * ps + d], n, w.n_kept_R, d == ob.imR));
        } else {
            r.lD = __fadd_rn(r.lD, grad_series<COST>(mape ? eD : __fmul_rn(eD, w.inv_rng_D), w.inv_rng_D, invys[d], n,
                                                      w.n_kept, d == ob.imD));
        }
    };
    RevF32 r;
    double gacc[kMaxParams];
    for (int d = 0; d < P; ++d) gacc[d] = 0.0;
    r.lS = r.lI = r.lSl = r.lIl = r.lD = r.lR = 0.f;
    r.cur = RAMP ? 0 : seg_of_step(steps - 1, steps, m.K);
    r.seg_lo = RAMP ? 0 : segment_start(r.cur, steps, m.K);
    inject(r, L, ob.Ih_last, ob.Il_last, ob.eR_last, ob.eD_last);
    for (int day = L - 1; day >= 0; --day) {
        restage_day<SPD, RAMP, 5>(w, m, th, B, cf, ck, cs, day, stS, stI, stC);
        rev_day<SPD, COST, RAMP, true>(r, gacc, w, m, invys, cf, day, steps, stS, stI, stC, B, 0.f, 0, dr);
        const float* c = ck + (size_t)day * 5 * cs;
        inject(r, day, c[cs], c[2 * cs], c[4 * cs], c[3 * cs]);
    }
    rev_write<RAMP, true>(r, gacc, w, m, p, Lval, loss, grad, ldg, grad_u0);
}

template <int SPD, int COST, bool RAMP, bool IRD>
__global__ void __launch_bounds__(64) loss_grad_f32_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                            const float* __restrict__ theta, int ld, int M,
                                                            float* __restrict__ loss, float* __restrict__ grad,
                                                            int ldg, float* __restrict__ grad_u0,
                                                            float* __restrict__ ckpt) {
    if constexpr (IRD)
        loss_grad_f32_ird_body<SPD, COST, RAMP>(w, m, o, theta, ld, M, loss, grad, ldg, grad_u0, ckpt, blockIdx.x);
    else
        loss_grad_f32_body<SPD, COST, RAMP>(w, m, o, theta, ld, M, loss, grad, ldg, grad_u0, ckpt, blockIdx.x);
}

// Table form: block row blockIdx.y takes window blockIdx.y (PolishWin) with its own constants.
template <int SPD, int COST, bool RAMP, bool IRD>
__global__ void __launch_bounds__(64) loss_grad_f32_tab_kernel(const PolishWin* __restrict__ tab, ModelDev m,
                                                                const float* __restrict__ theta, long long th_ws,
                                                                int ld, int M, float* __restrict__ loss,
                                                                long long loss_ws, float* __restrict__ grad,
                                                                long long grad_ws, int ldg, float* __restrict__ ckpt,
                                                                long long ck_ws) {
    const int i = blockIdx.y;
    const WindowDev w = tab[i].w;
    const ObsDev o = tab[i].o;
    if constexpr (IRD)
        loss_grad_f32_ird_body<SPD, COST, RAMP>(w, m, o, theta + i * th_ws, ld, M, loss + i * loss_ws,
                                                grad + i * grad_ws, ldg, nullptr, ckpt + i * ck_ws, blockIdx.x);
    else
        loss_grad_f32_body<SPD, COST, RAMP>(w, m, o, theta + i * th_ws, ld, M, loss + i * loss_ws, grad + i * grad_ws,
                                            ldg, nullptr, ckpt + i * ck_ws, blockIdx.x);
}

// Warp-specialised form (PWC, 10 or 20 steps per day): a block of two warps owns 32 parameter
// vectors.  Warp 0 runs the forward pass and then re-integrates the days, last to first, into a
// double-buffered stage in shared memory; warp 1 sweeps each staged day backwards while warp 0
// re-integrates the day before it, one block barrier per day handing the buffers over.  The two
// halves of the per-vector work run on two warp schedulers at once; each chain's arithmetic and
// order are those of loss_grad_f32_kernel, so the results are identical.  A lane past the end of
// the vectors integrates a copy of the last one and writes nothing but its own checkpoints.
constexpr int kWsVectors = 32;

template <int SPD, int COST>
__device__ __forceinline__ void loss_grad_f32_ws_body(const WindowDev& w, const ModelDev& m, const ObsDev& o,
                                                      const float* __restrict__ theta, int ld, int M,
                                                      float* __restrict__ loss, float* __restrict__ grad, int ldg,
                                                      float* __restrict__ grad_u0, float* __restrict__ ckpt, int Mpad,
                                                      int blk) {
    extern __shared__ float smem[];
    constexpr int V = kWsVectors;
    const int tid = threadIdx.x, lane = tid & 31, P = m.P, n = w.n_obs, L = n - 1, steps = L * SPD;
    const bool fwd = tid < V;
    float* ys = smem;
    float* invys = ys + ((n + 3) & ~3);
    float* th_all = invys + ((n + 3) & ~3);  // [P][V]
    float* stage = th_all + P * V;           // [2 buffers][S, I, cb][SPD][V]
    float* xch = stage + 6 * SPD * V;        // e_L, MXSE day and loss of each vector
    for (int i = tid; i < n; i += 2 * V) {
        ys[i] = o.yf[i];
        invys[i] = o.invyf[i];
    }
    const int p = blk * V + lane;
    const bool active = p < M;
    if (fwd) {
        const int src = active ? p : M - 1;
        for (int d = 0; d < P; ++d) th_all[d * V + lane] = theta[(size_t)d * ld + src];
    }
    __syncthreads();
    const float* th = th_all + lane;
    const CoefF32 cf = coef_f32<false>(w, m, th, V);
    float* ck = ckpt + p;
    const size_t cs = (size_t)Mpad;
    auto buf = [&](int b, int q) { return stage + (size_t)(b * 3 + q) * SPD * V + lane; };
    if (fwd) {
        float e_last;
        int imax;
        const float Lval = forward_checkpointed<SPD, COST, false>(w, m, ys, invys, th, V, cf, ck, cs, e_last, imax);
        xch[lane] = e_last;
        xch[V + lane] = __int_as_float(imax);
        xch[2 * V + lane] = Lval;
        restage_day<SPD, false>(w, m, th, V, cf, ck, cs, L - 1, buf(0, 0), buf(0, 1), buf(0, 2));
    }
    __syncthreads();
    RevF32 r{};
    double gacc[kMaxParams];
    int imax = 0;
    float e_d = 0.f;
    if (!fwd) {
        imax = __float_as_int(xch[V + lane]);
        rev_begin<COST, false>(r, gacc, w, m, invys, steps, xch[lane], imax);
        e_d = ck[((size_t)(L - 1) * 4 + 3) * cs];
    }
    for (int day = L - 1; day >= 0; --day) {
        const int b = (L - 1 - day) & 1;
        if (fwd) {
            if (day > 0) restage_day<SPD, false>(w, m, th, V, cf, ck, cs, day - 1, buf(b ^ 1, 0), buf(b ^ 1, 1), buf(b ^ 1, 2));
        } else {
            const float e_next = day > 0 ? ck[((size_t)(day - 1) * 4 + 3) * cs] : 0.f;
            rev_day<SPD, COST, false>(r, gacc, w, m, invys, cf, day, steps, buf(b, 0), buf(b, 1), buf(b, 2), V, e_d, imax);
            e_d = e_next;
        }
        __syncthreads();
    }
    if (!fwd && active) rev_write<false>(r, gacc, w, m, p, xch[2 * V + lane], loss, grad, ldg, grad_u0);
}

template <int SPD, int COST>
__global__ void __launch_bounds__(64) loss_grad_f32_ws_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                               const float* __restrict__ theta, int ld, int M,
                                                               float* __restrict__ loss, float* __restrict__ grad,
                                                               int ldg, float* __restrict__ grad_u0,
                                                               float* __restrict__ ckpt, int Mpad) {
    loss_grad_f32_ws_body<SPD, COST>(w, m, o, theta, ld, M, loss, grad, ldg, grad_u0, ckpt, Mpad, blockIdx.x);
}

template <int SPD, int COST>
__global__ void __launch_bounds__(64) loss_grad_f32_ws_tab_kernel(const PolishWin* __restrict__ tab, ModelDev m,
                                                                   const float* __restrict__ theta, long long th_ws,
                                                                   int ld, int M, float* __restrict__ loss,
                                                                   long long loss_ws, float* __restrict__ grad,
                                                                   long long grad_ws, int ldg,
                                                                   float* __restrict__ ckpt, long long ck_ws,
                                                                   int Mpad) {
    const int i = blockIdx.y;
    const WindowDev w = tab[i].w;
    const ObsDev o = tab[i].o;
    loss_grad_f32_ws_body<SPD, COST>(w, m, o, theta + i * th_ws, ld, M, loss + i * loss_ws, grad + i * grad_ws, ldg,
                                     nullptr, ckpt + i * ck_ws, Mpad, blockIdx.x);
}

}  // namespace

size_t adjoint_ckpt_bytes_f32(const WindowDev& w, const ModelDev& m, int M) {
    const size_t Mpad = ((size_t)M + kWsVectors - 1) / kWsVectors * kWsVectors;
    return (size_t)(w.n_obs - 1) * (m.ird ? 5 : 4) * Mpad * sizeof(float);
}

cudaError_t launch_loss_grad_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const float* theta, int ld,
                                 int M, float* loss, float* grad, int ldg, float* grad_u0, float* ckpt,
                                 cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (m.spd < 1 || m.spd > kMaxSpdGeneric) return cudaErrorInvalidValue;
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
    const size_t obs = 2 * (size_t)((w.n_obs + 3) & ~3) * (m.ird ? 3 : 1);
    if (m.beta_form != BETA_RAMP && !m.ird && (m.spd == 10 || m.spd == 20)) {
        // two warps per 32 vectors: the re-integration and the reverse sweep side by side
        const int Mpad = (M + kWsVectors - 1) / kWsVectors * kWsVectors;
        const size_t sm = (obs + (size_t)m.P * kWsVectors + 6 * (size_t)m.spd * kWsVectors + 3 * kWsVectors) * sizeof(float);
#define SIRD_LGWS(SV, CV)                                                                                            \
    {                                                                                                                \
        auto kern = loss_grad_f32_ws_kernel<SV, CV>;                                                                 \
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);   \
        if (e == cudaSuccess)                                                                                        \
            kern<<<Mpad / kWsVectors, 2 * kWsVectors, sm, s>>>(w, m, o, theta, ld, M, loss, grad, ldg, grad_u0, ckpt, \
                                                             Mpad);                                                  \
    }
#define SIRD_LGWS_COST(SV)                                \
    switch (m.cost) {                                     \
        case COST_MSE: SIRD_LGWS(SV, COST_MSE) break;     \
        case COST_MXSE: SIRD_LGWS(SV, COST_MXSE) break;   \
        case COST_MAE: SIRD_LGWS(SV, COST_MAE) break;     \
        default: SIRD_LGWS(SV, COST_MAPE) break;          \
    }
        if (m.spd == 10) {
            SIRD_LGWS_COST(10)
        } else {
            SIRD_LGWS_COST(20)
        }
#undef SIRD_LGWS_COST
#undef SIRD_LGWS
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    // 64 threads per block: the work is one long serial chain per parameter vector, so a few
    // warps per SM on as many SMs as possible
    const int block = 64;
    const size_t sm = (obs + (size_t)m.P * block + 3 * (size_t)m.spd * block) * sizeof(float);
#define SIRD_LG32(SV, CV, RV)                                                                                 \
    {                                                                                                         \
        auto kern = m.ird ? loss_grad_f32_kernel<SV, CV, RV, true> : loss_grad_f32_kernel<SV, CV, RV, false>;  \
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e == cudaSuccess)                                                                                 \
            kern<<<(M + block - 1) / block, block, sm, s>>>(w, m, o, theta, ld, M, loss, grad, ldg, grad_u0, ckpt); \
    }
#define SIRD_LG32_COST(SV, RV)                              \
    switch (m.cost) {                                       \
        case COST_MSE: SIRD_LG32(SV, COST_MSE, RV) break;   \
        case COST_MXSE: SIRD_LG32(SV, COST_MXSE, RV) break; \
        case COST_MAE: SIRD_LG32(SV, COST_MAE, RV) break;   \
        default: SIRD_LG32(SV, COST_MAPE, RV) break;        \
    }
    if (m.beta_form == BETA_RAMP) {
        SIRD_LG32_COST(0, true)
    } else {
        SIRD_LG32_COST(0, false)
    }
#undef SIRD_LG32_COST
#undef SIRD_LG32
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_loss_grad_f32_tab(const PolishWin* tab, int nw, int n_max, const ModelDev& m, const float* theta,
                                     long long th_ws, int ld, int M, float* loss, long long loss_ws, float* grad,
                                     long long grad_ws, int ldg, float* ckpt, long long ck_ws, cudaStream_t s) {
    if (M <= 0 || nw <= 0) return cudaSuccess;
    if (m.spd < 1 || m.spd > kMaxSpdGeneric || nw > 65535) return cudaErrorInvalidValue;
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
    const size_t obs = 2 * (size_t)((n_max + 3) & ~3) * (m.ird ? 3 : 1);
    if (m.beta_form != BETA_RAMP && !m.ird && (m.spd == 10 || m.spd == 20)) {
        const int Mpad = (M + kWsVectors - 1) / kWsVectors * kWsVectors;
        const size_t sm = (obs + (size_t)m.P * kWsVectors + 6 * (size_t)m.spd * kWsVectors + 3 * kWsVectors) * sizeof(float);
        const dim3 grid((unsigned)(Mpad / kWsVectors), (unsigned)nw);
#define SIRD_LGWS(SV, CV)                                                                                            \
    {                                                                                                                \
        auto kern = loss_grad_f32_ws_tab_kernel<SV, CV>;                                                             \
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);   \
        if (e == cudaSuccess)                                                                                        \
            kern<<<grid, 2 * kWsVectors, sm, s>>>(tab, m, theta, th_ws, ld, M, loss, loss_ws, grad, grad_ws, ldg,     \
                                                  ckpt, ck_ws, Mpad);                                                \
    }
#define SIRD_LGWS_COST(SV)                                \
    switch (m.cost) {                                     \
        case COST_MSE: SIRD_LGWS(SV, COST_MSE) break;     \
        case COST_MXSE: SIRD_LGWS(SV, COST_MXSE) break;   \
        case COST_MAE: SIRD_LGWS(SV, COST_MAE) break;     \
        default: SIRD_LGWS(SV, COST_MAPE) break;          \
    }
        if (m.spd == 10) {
            SIRD_LGWS_COST(10)
        } else {
            SIRD_LGWS_COST(20)
        }
#undef SIRD_LGWS_COST
#undef SIRD_LGWS
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int block = 64;
    const size_t sm = (obs + (size_t)m.P * block + 3 * (size_t)m.spd * block) * sizeof(float);
    const dim3 grid((unsigned)((M + block - 1) / block), (unsigned)nw);
#define SIRD_LG32(SV, CV, RV)                                                                                 \
    {                                                                                                         \
        auto kern = m.ird ? loss_grad_f32_tab_kernel<SV, CV, RV, true> : loss_grad_f32_tab_kernel<SV, CV, RV, false>; \
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e == cudaSuccess)                                                                                 \
            kern<<<grid, block, sm, s>>>(tab, m, theta, th_ws, ld, M, loss, loss_ws, grad, grad_ws, ldg, ckpt, ck_ws); \
    }
#define SIRD_LG32_COST(SV, RV)                              \
    switch (m.cost) {                                       \
        case COST_MSE: SIRD_LG32(SV, COST_MSE, RV) break;   \
        case COST_MXSE: SIRD_LG32(SV, COST_MXSE, RV) break; \
        case COST_MAE: SIRD_LG32(SV, COST_MAE, RV) break;   \
        default: SIRD_LG32(SV, COST_MAPE, RV) break;        \
    }
    if (m.beta_form == BETA_RAMP) {
        SIRD_LG32_COST(0, true)
    } else {
        SIRD_LG32_COST(0, false)
    }
#undef SIRD_LG32_COST
#undef SIRD_LG32
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sird
