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
// and dL/dI0 = lambda_I(0) - lambda_S(0) (S0 = N - I0 - R0 - D0).
//
// The forward pass is the compensated FP32 integration of the evaluation kernels, operation for
// operation, so the loss equals the FP32 evaluation's bit for bit.  It stores the state at the
// start of every day (Sday, I, its low part, and the day's error e_d) in global scratch
// [day][4][M]; the reverse pass re-integrates one day at a time, staging each step's S, I and
// coefficient in shared memory, and sweeps the day backwards.  lambda_S and lambda_I carry
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

template <int SPD, int COST, bool RAMP>
__global__ void __launch_bounds__(64) loss_grad_f32_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                            const float* __restrict__ theta, int ld, int M,
                                                            float* __restrict__ loss, float* __restrict__ grad,
                                                            int ldg, float* __restrict__ grad_u0,
                                                            float* __restrict__ ckpt) {
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
    const int p = blockIdx.x * B + tid;
    const bool active = p < M;
    if (active)
        for (int d = 0; d < P; ++d) th_all[d * B + tid] = theta[(size_t)d * ld + p];
    __syncthreads();
    if (!active) return;
    const float* th = th_all + tid;

    const int L = n - 1, steps = L * spd, K = m.K;
    const int gi = RAMP ? 4 : K;
    const float gam = th[gi * B], mu = th[(gi + 1) * B];
    float I = m.fit_I0 ? th[(gi + 2) * B] : w.I0f;
    float Il = 0.f;
    const float gm = __fadd_rn(gam, mu);
    const float a = __fmaf_rn(gm, w.dt_h, __fmul_rn(gm, w.dt_l));
    const float dm = __fmaf_rn(mu, w.dt_h, __fmul_rn(mu, w.dt_l));
    RampF32 rp{};
    if (RAMP) {
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
    auto cb_of = [&](float beta) { return __fmaf_rn(beta, w.cbn_h, __fmul_rn(beta, w.cbn_l)); };

    // ---- forward: the FP32 evaluation's arithmetic, plus the day-start checkpoints
    DayStateF32 ds;
    ds.init(w, I, ys[0]);
    LossF32<COST> lossacc;
    float emax = 0.f, e_prev = 0.f;  // e_0 = y_0 - D_0 = 0
    int imax = 0;
    int seg = 0, next_b = (!RAMP && K > 1) ? segment_start(1, steps, K) : INT_MAX;
    float cb = RAMP ? 0.f : cb_of(th[0]);
    for (int day = 0; day < L; ++day) {
        const size_t base = (size_t)day * 4 * M + p;
        ckpt[base] = ds.Sday;
        ckpt[base + M] = I;
        ckpt[base + 2 * (size_t)M] = Il;
        ckpt[base + 3 * (size_t)M] = e_prev;
        float cday = 0.f, dday = 0.f;
        day_steps<SPD, RAMP, false>(day, spd, steps, K, th, B, rp, a, dm, w, ds.Sday, cday, dday, I, Il, seg, next_b,
                                    cb, nullptr, nullptr, nullptr);
        const float e = ds.close_day(w, cday, dday, ys[day + 1], I, Il);
        lossacc.add(e, COST == COST_MAPE ? invys[day + 1] : 0.f);
        if (COST == COST_MXSE) {
            const float e2 = __fmul_rn(e, e);
            if (e2 > emax) {
                emax = e2;
                imax = day + 1;
            }
        }
        e_prev = e;
    }
    const float Lval = lossacc.result(n, w.n_kept);

    // ---- reverse sweep, one day at a time
    double gacc[kMaxParams];
    for (int d = 0; d < P; ++d) gacc[d] = 0.0;
    float lS = 0.f, lI = 0.f, lSl = 0.f, lIl = 0.f;
    float lD = grad_D<COST>(e_prev, invys[L], n, w.n_kept, imax == L);
    int cur = RAMP ? 0 : seg_of_step(steps - 1, steps, K);
    int seg_lo = RAMP ? 0 : segment_start(cur, steps, K);
    // checkpoint of the day to re-integrate, loaded one day ahead
    size_t base = (size_t)(L - 1) * 4 * M + p;
    float nSday = ckpt[base], nI = ckpt[base + M], nIl = ckpt[base + 2 * (size_t)M], ne = ckpt[base + 3 * (size_t)M];
    for (int day = L - 1; day >= 0; --day) {
        const float Sday = nSday, e_d = ne;
        float Ir = nI, Ilr = nIl;
        if (day > 0) {
            base = (size_t)(day - 1) * 4 * M + p;
            nSday = ckpt[base];
            nI = ckpt[base + M];
            nIl = ckpt[base + 2 * (size_t)M];
            ne = ckpt[base + 3 * (size_t)M];
        }
        // re-integrate the day (the forward pass's coefficients), staging each step's S, I, cb
        {
            int sg = RAMP ? 0 : seg_of_step(day * spd, steps, K);
            int nb = (!RAMP && sg + 1 < K) ? segment_start(sg + 1, steps, K) : INT_MAX;
            float c = RAMP ? 0.f : cb_of(th[sg * B]);
            float cday = 0.f, dday = 0.f;
            day_steps<SPD, RAMP, true>(day, spd, steps, K, th, B, rp, a, dm, w, Sday, cday, dday, Ir, Ilr, sg, nb, c,
                                       stS, stI, stC);
        }
        float pb = 0.f, pg = 0.f, pm = 0.f, pr[4] = {0.f, 0.f, 0.f, 0.f};
        const float dmlD = __fmul_rn(dm, lD);  // lambda_D is constant within the day
#pragma unroll 4
        for (int s = spd - 1; s >= 0; --s) {
            const int k = day * spd + s;
            const float S = stS[s * B], Iv = stI[s * B], c = stC[s * B];
            if (!RAMP && k < seg_lo) {  // entering the previous segment (uniform across the warp)
                gacc[cur] += (double)pb;
                pb = 0.f;
                cur = seg_of_step(k, steps, K);
                seg_lo = segment_start(cur, steps, K);
            }
            const float q = __fsub_rn(lI, lS);
            const float SI = __fmul_rn(S, Iv);
            if (RAMP) {
                float db[4];
                rp.dbeta(k, db);
                const float r = __fmul_rn(SI, q);
#pragma unroll
                for (int j = 0; j < 4; ++j) pr[j] = __fmaf_rn(r, db[j], pr[j]);
            } else {
                pb = __fmaf_rn(SI, q, pb);
            }
            pg = __fmaf_rn(Iv, lI, pg);
            pm = __fmaf_rn(Iv, __fsub_rn(lD, lI), pm);
            // lambda_S and lambda_I change by small increments per step; as for I in the forward
            // pass, each sum's rounding error is kept (Fast2Sum) and folded in once a day
            const float dS = __fmul_rn(__fmul_rn(c, Iv), q);
            const float dI = __fmaf_rn(__fmul_rn(c, S), q, __fmaf_rn(-a, lI, dmlD));
            const float rS = __fadd_rn(lS, dS), rI = __fadd_rn(lI, dI);
            lSl = __fadd_rn(lSl, __fsub_rn(dS, __fsub_rn(rS, lS)));
            lIl = __fadd_rn(lIl, __fsub_rn(dI, __fsub_rn(rI, lI)));
            lS = rS;
            lI = rI;
        }
        {
            const float fs = __fadd_rn(lS, lSl), fi = __fadd_rn(lI, lIl);
            lSl = __fsub_rn(lSl, __fsub_rn(fs, lS));
            lIl = __fsub_rn(lIl, __fsub_rn(fi, lI));
            lS = fs;
            lI = fi;
        }
        lD = __fadd_rn(lD, grad_D<COST>(e_d, invys[day], n, w.n_kept, COST == COST_MXSE && imax == day));
        if (RAMP) {
#pragma unroll
            for (int j = 0; j < 4; ++j) gacc[j] += (double)pr[j];
        } else {
            gacc[cur] += (double)pb;
        }
        gacc[gi] += (double)pg;
        gacc[gi + 1] += (double)pm;
    }
    const double dtN = w.dt / w.N;
    const int nbeta = RAMP ? 4 : K;
    for (int d = 0; d < nbeta; ++d) grad[(size_t)d * ldg + p] = (float)(gacc[d] * dtN);
    grad[(size_t)gi * ldg + p] = (float)(-w.dt * gacc[gi]);
    grad[(size_t)(gi + 1) * ldg + p] = (float)(w.dt * gacc[gi + 1]);
    lS = __fadd_rn(lS, lSl);
    lI = __fadd_rn(lI, lIl);
    if (m.fit_I0) grad[(size_t)(gi + 2) * ldg + p] = __fsub_rn(lI, lS);
    loss[p] = Lval;
    if (grad_u0) {
        grad_u0[p] = lS;
        grad_u0[(size_t)ldg + p] = lI;
        grad_u0[2 * (size_t)ldg + p] = 0.f;
        grad_u0[3 * (size_t)ldg + p] = lD;
    }
}

}  // namespace

size_t adjoint_ckpt_bytes_f32(const WindowDev& w, int M) {
    return (size_t)(w.n_obs - 1) * 4 * (size_t)M * sizeof(float);
}

cudaError_t launch_loss_grad_f32(const WindowDev& w, const ModelDev& m, const ObsDev& o, const float* theta, int ld,
                                 int M, float* loss, float* grad, int ldg, float* grad_u0, float* ckpt,
                                 cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (m.spd < 1 || m.spd > kMaxSpdGeneric) return cudaErrorInvalidValue;
    // 64 threads per block: the work is one long serial chain per parameter vector, so a few
    // warps per SM on as many SMs as possible
    const int block = 64;
    const size_t sm = (2 * (size_t)((w.n_obs + 3) & ~3) + (size_t)m.P * block + 3 * (size_t)m.spd * block) * sizeof(float);
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
#define SIRD_LG32(SV, CV, RV)                                                                                 \
    {                                                                                                         \
        auto kern = loss_grad_f32_kernel<SV, CV, RV>;                                                         \
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
        switch (m.spd) {
            case 10: SIRD_LG32_COST(10, false) break;
            case 20: SIRD_LG32_COST(20, false) break;
            default: SIRD_LG32_COST(0, false) break;
        }
    }
#undef SIRD_LG32_COST
#undef SIRD_LG32
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sird
