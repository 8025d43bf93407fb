// adjoint.cu -- exact gradient of the discrete loss by the discrete adjoint of the Euler map.
//
// The paper calibrates with PSO because no gradient is at hand (Sec. 3.3).  The Euler-discretised
// loss does have one: with u_{k+1} = u_k + dt f(u_k, theta) (eq. (SIRD), f = (-bSI, bSI - (gamma
// + mu) I, gamma I, mu I), b = beta/N) and L = C(e_1..e_n), the adjoint runs backwards
//     lambda_k = lambda_{k+1} + dt (df/du)^T lambda_{k+1} + dL/du_k   (dL/dD at observation steps)
//     dL/dtheta += dt (df/dtheta)^T lambda_{k+1}
// and dL/du_0 = lambda_0; with S0 = N - I0 - R0 - D0, dL/dI0 = lambda_I(0) - lambda_S(0).
// R never feeds back into S, I or D and the F_D losses do not see it, so there lambda_R stays 0.
// F_IRD^C (Sec. 3.1) is the largest of the three series' costs; its gradient is that of the series
// attaining the maximum (the first of I, R, D on ties), each error divided by the series' range
// (MAPE unnormalised), injected into lambda_I, lambda_R or lambda_D on its observation days.
//
// One thread per parameter vector.  The forward pass stores (S, I, D), and R for F_IRD, every
// `ckpt` steps in global scratch ([checkpoint][3 or 4][M], coalesced); the backward pass recomputes each
// `ckpt`-step stretch from its checkpoint into thread-local memory and sweeps it in reverse.
// The FP64 version performs every operation in the order written above with no contraction,
// so loss and gradient are exactly those of the plain FP64 reference.
#include <climits>

#include "kernels.h"

namespace sird {

namespace {

constexpr int kMaxCkpt = 64;

__device__ __forceinline__ int seg_of(int k, int steps, int K) { return (int)(((long long)k * K) / steps); }

// One FP64 Euler step of (S, I, D) (R is not needed), paper operation order.
__device__ __forceinline__ void euler_f64(double bN, double gm, double mu, double dt, double& S, double& I,
                                          double& D) {
    const double fS = __dmul_rn(__dmul_rn(-bN, S), I);
    const double fI = __dsub_rn(__dmul_rn(__dmul_rn(bN, I), S), __dmul_rn(gm, I));
    const double fD = __dmul_rn(mu, I);
    S = __dadd_rn(S, __dmul_rn(dt, fS));
    I = __dadd_rn(I, __dmul_rn(dt, fI));
    D = __dadd_rn(D, __dmul_rn(dt, fD));
}

// The same step with R (F_IRD), in the paper's order: S, I, R, D.
__device__ __forceinline__ void euler_f64_r(double bN, double gam, double gm, double mu, double dt, double& S,
                                            double& I, double& R, double& D) {
    const double fS = __dmul_rn(__dmul_rn(-bN, S), I);
    const double fI = __dsub_rn(__dmul_rn(__dmul_rn(bN, I), S), __dmul_rn(gm, I));
    const double fR = __dmul_rn(gam, I);
    const double fD = __dmul_rn(mu, I);
    S = __dadd_rn(S, __dmul_rn(dt, fS));
    I = __dadd_rn(I, __dmul_rn(dt, fI));
    R = __dadd_rn(R, __dmul_rn(dt, fR));
    D = __dadd_rn(D, __dmul_rn(dt, fD));
}

struct RampF64 {
    double b1, b2, t1, t2;
    bool swapped;
};

__device__ __forceinline__ double ramp_beta(const RampF64& r, double t) {
    if (t < r.t1) return r.b1;
    if (t < r.t2) return __dadd_rn(r.b1, __dmul_rn(__ddiv_rn(__dsub_rn(r.b2, r.b1), __dsub_rn(r.t2, r.t1)), __dsub_rn(t, r.t1)));
    return r.b2;
}

// dC/dyhat_i of one series' cost over the errors e_i = (y_i - yhat_i) / scale, in the order of the
// plain reference: MSE -2 e_i / (n scale), MAE -sign(e_i) / (n scale), MXSE -2 e_i / scale on the
// first day with the largest e^2 (imax; none when every e is 0), MAPE -100 sign(e_i) / (|y_i| kept)
// on the days with y_i != 0 (scale 1).
template <int COST>
__device__ __forceinline__ double series_grad(double y, double yhat, double scale, int n, int kept, bool is_max) {
    const double e = __ddiv_rn(__dsub_rn(y, yhat), scale);
    const double sg = (double)((e > 0.0) - (e < 0.0));
    if (COST == COST_MSE) return __ddiv_rn(__dmul_rn(-2.0, e), __dmul_rn((double)n, scale));
    if (COST == COST_MAE) return __ddiv_rn(-sg, __dmul_rn((double)n, scale));
    if (COST == COST_MAPE) return (y != 0.0 && kept > 0) ? __ddiv_rn(__dmul_rn(-100.0, sg), __dmul_rn(fabs(y), (double)kept)) : 0.0;
    return is_max ? __ddiv_rn(__dmul_rn(-2.0, e), scale) : 0.0;
}

template <int COST, bool IRD>
__global__ void __launch_bounds__(128) loss_grad_f64_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                             const double* __restrict__ theta, int ld, int M,
                                                             double* __restrict__ loss, double* __restrict__ grad,
                                                             int ldg, double* __restrict__ grad_u0,
                                                             double* __restrict__ ckpt, int C) {
    extern __shared__ double dsm[];
    const int B = blockDim.x, tid = threadIdx.x, P = m.P;
    const int ps = obs_stride(w.n_obs), nys = IRD ? 3 * ps : w.n_obs;  // F_IRD: D | I | R stacked
    double* ys = dsm;
    double* th = dsm + nys;        // [P][B]
    double* g = th + P * B;        // [P][B] gradient accumulators
    for (int i = tid; i < nys; i += B) ys[i] = o.yd[i];
    const int p = blockIdx.x * B + tid;
    const bool active = p < M;
    if (active)
        for (int d = 0; d < P; ++d) {
            th[d * B + tid] = theta[(size_t)d * ld + p];
            g[d * B + tid] = 0.0;
        }
    __syncthreads();
    if (!active) return;
    const double* t_ = th + tid;
    double* g_ = g + tid;

    const int spd = m.spd, n = w.n_obs, L = n - 1, steps = L * spd, K = m.K;
    const bool ramp = m.beta_form == BETA_RAMP;
    const int gi = ramp ? 4 : K;
    const double gam = t_[gi * B], mu = t_[(gi + 1) * B];
    const double I0 = m.fit_I0 ? t_[(gi + 2) * B] : w.I0;
    const double gm = __dadd_rn(gam, mu), dt = w.dt, N = w.N;
    RampF64 rp{0, 0, 0, 0, false};
    if (ramp) {
        rp.b1 = t_[0];
        rp.b2 = t_[B];
        rp.swapped = t_[2 * B] > t_[3 * B];
        rp.t1 = rp.swapped ? t_[3 * B] : t_[2 * B];
        rp.t2 = rp.swapped ? t_[2 * B] : t_[3 * B];
    }
    auto beta_at = [&](int k) -> double {
        return ramp ? ramp_beta(rp, __ddiv_rn((double)k, (double)spd)) : t_[seg_of(k, steps, K) * B];
    };
    constexpr int NU = IRD ? 4 : 3;  // checkpointed state: S, I, D (F_D) or S, I, R, D (F_IRD)

    // ---- forward: loss (same order as the plain evaluation) and checkpoints
    double S = __dsub_rn(__dsub_rn(__dsub_rn(N, I0), w.R0), w.D0), I = I0, R = w.R0, D = w.D0;
    double acc = 0.0, emax = -1.0;
    int imax = 0;
    auto observe = [&](int i, double Dh) {
        const double e = __dsub_rn(ys[i], Dh);
        const double e2 = __dmul_rn(e, e);
        if (COST == COST_MSE) acc = __dadd_rn(acc, e2);
        else if (COST == COST_MXSE) { if (e2 > acc) acc = e2; }
        else if (COST == COST_MAE) acc = __dadd_rn(acc, fabs(e));
        else if (ys[i] != 0.0) acc = __dadd_rn(acc, fabs(__ddiv_rn(e, ys[i])));
        if (e2 > emax) {
            emax = e2;
            imax = i;
        }
    };
    // F_IRD: the three series' costs (the evaluation's SeriesCostF64) and, for MXSE, the first day
    // with each series' largest e^2 (-1: none above 0)
    const bool mape = COST == COST_MAPE;
    const double sI = mape ? 1.0 : w.rng_I, sR = mape ? 1.0 : w.rng_R, sD = mape ? 1.0 : w.rng_D;
    const double *yI = ys + ps, *yR = ys + 2 * ps;
    SeriesCostF64<COST> cI, cR, cD;
    int mxI = -1, mxR = -1, mxD = -1;
    auto observe3 = [&](int i) {
        if (COST == COST_MXSE) {
            const double eI = __ddiv_rn(__dsub_rn(yI[i], I), sI), eR = __ddiv_rn(__dsub_rn(yR[i], R), sR),
                         eD = __ddiv_rn(__dsub_rn(ys[i], D), sD);
            if (__dmul_rn(eI, eI) > cI.acc) mxI = i;
            if (__dmul_rn(eR, eR) > cR.acc) mxR = i;
            if (__dmul_rn(eD, eD) > cD.acc) mxD = i;
        }
        cI.add(yI[i], I, sI);
        cR.add(yR[i], R, sR);
        cD.add(ys[i], D, sD);
    };
    if (IRD) observe3(0);
    else observe(0, D);
    for (int k = 0; k < steps; ++k) {
        if (k % C == 0) {
            const size_t base = (size_t)(k / C) * NU * M + p;
            ckpt[base] = S;
            ckpt[base + M] = I;
            ckpt[base + 2 * (size_t)M] = D;
            if (IRD) ckpt[base + 3 * (size_t)M] = R;
        }
        if (IRD) {
            euler_f64_r(__ddiv_rn(beta_at(k), N), gam, gm, mu, dt, S, I, R, D);
            if ((k + 1) % spd == 0) observe3((k + 1) / spd);
        } else {
            euler_f64(__ddiv_rn(beta_at(k), N), gm, mu, dt, S, I, D);
            if ((k + 1) % spd == 0) observe((k + 1) / spd, D);
        }
    }
    double Lval;
    int which = 2;  // F_IRD: the series attaining the maximum (0: I, 1: R, 2: D; the first on ties)
    if (IRD) {
        const double a = cI.result(n), b = cR.result(n), c = cD.result(n);
        Lval = a;
        which = 0;
        if (b > Lval) { Lval = b; which = 1; }
        if (c > Lval) { Lval = c; which = 2; }
    } else if (COST == COST_MSE || COST == COST_MAE) Lval = __ddiv_rn(acc, (double)n);
    else if (COST == COST_MAPE) Lval = w.n_kept > 0 ? __ddiv_rn(__dmul_rn(100.0, acc), (double)w.n_kept) : 0.0;
    else Lval = acc;

    // dL/dDhat_i, as a function of day i and Dhat_i
    auto gD = [&](int i, double Dh) -> double {
        const double e = __dsub_rn(ys[i], Dh);
        const double sg = (double)((e > 0.0) - (e < 0.0));
        if (COST == COST_MSE) return __ddiv_rn(__dmul_rn(-2.0, e), (double)n);
        if (COST == COST_MAE) return __ddiv_rn(-sg, (double)n);
        if (COST == COST_MAPE)
            return (ys[i] != 0.0 && w.n_kept > 0) ? __ddiv_rn(__dmul_rn(-100.0, sg), __dmul_rn(fabs(ys[i]), (double)w.n_kept)) : 0.0;
        return i == imax ? __dmul_rn(-2.0, e) : 0.0;
    };
    // F_IRD: day i's cost gradients of the three series (zero but for the dominant one), added to
    // lambda_I, lambda_R and lambda_D as the plain reference adds them
    auto inject = [&](int i, double Ih, double Rh, double Dh, double& lI_, double& lR_, double& lD_) {
        if (!IRD) {
            lD_ = __dadd_rn(lD_, gD(i, Dh));
            return;
        }
        const double gI = which == 0 ? series_grad<COST>(yI[i], Ih, sI, n, w.n_kept_I, i == mxI) : 0.0;
        const double gR = which == 1 ? series_grad<COST>(yR[i], Rh, sR, n, w.n_kept_R, i == mxR) : 0.0;
        const double gDv = which == 2 ? series_grad<COST>(ys[i], Dh, sD, n, w.n_kept, i == mxD) : 0.0;
        lI_ = __dadd_rn(lI_, gI);
        lR_ = __dadd_rn(lR_, gR);
        lD_ = __dadd_rn(lD_, gDv);
    };

    // ---- backward over checkpointed stretches (lambda after the last step: the last day's gradients)
    double lS = 0.0, lI = 0.0, lR = 0.0, lD = 0.0;
    if (IRD) {
        lI = which == 0 ? series_grad<COST>(yI[n - 1], I, sI, n, w.n_kept_I, n - 1 == mxI) : 0.0;
        lR = which == 1 ? series_grad<COST>(yR[n - 1], R, sR, n, w.n_kept_R, n - 1 == mxR) : 0.0;
        lD = which == 2 ? series_grad<COST>(ys[n - 1], D, sD, n, w.n_kept, n - 1 == mxD) : 0.0;
    } else {
        lD = gD(n - 1, D);
    }
    double US[kMaxCkpt + 1], UI[kMaxCkpt + 1], UD[kMaxCkpt + 1], UR[IRD ? kMaxCkpt + 1 : 1];
    const int nck = (steps + C - 1) / C;
    for (int c = nck - 1; c >= 0; --c) {
        const int k0 = c * C, k1 = min(k0 + C, steps);
        const size_t base = (size_t)c * NU * M + p;
        double s = ckpt[base], i_ = ckpt[base + M], d_ = ckpt[base + 2 * (size_t)M];
        double r_ = IRD ? ckpt[base + 3 * (size_t)M] : 0.0;
        US[0] = s;
        UI[0] = i_;
        UD[0] = d_;
        if (IRD) UR[0] = r_;
        for (int k = k0; k < k1 - 1; ++k) {  // recompute states k0+1 .. k1-1 of this stretch
            if (IRD) euler_f64_r(__ddiv_rn(beta_at(k), N), gam, gm, mu, dt, s, i_, r_, d_);
            else euler_f64(__ddiv_rn(beta_at(k), N), gm, mu, dt, s, i_, d_);
            US[k - k0 + 1] = s;
            UI[k - k0 + 1] = i_;
            UD[k - k0 + 1] = d_;
            if (IRD) UR[k - k0 + 1] = r_;
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const double Sk = US[k - k0], Ik = UI[k - k0];
            const double beta = beta_at(k);
            const double b = __ddiv_rn(beta, N);
            const double dL_dbeta = __dmul_rn(__dmul_rn(dt, __ddiv_rn(__dmul_rn(Sk, Ik), N)), __dsub_rn(lI, lS));
            if (!ramp) {
                const int sg = seg_of(k, steps, K);
                g_[sg * B] = __dadd_rn(g_[sg * B], dL_dbeta);
            } else {
                const double t = __ddiv_rn((double)k, (double)spd);
                double d_b1 = 0, d_b2 = 0, d_t1 = 0, d_t2 = 0;
                if (t < rp.t1) {
                    d_b1 = 1.0;
                } else if (t < rp.t2) {
                    const double len = __dsub_rn(rp.t2, rp.t1), sr = __ddiv_rn(__dsub_rn(t, rp.t1), len);
                    d_b1 = __dsub_rn(1.0, sr);
                    d_b2 = sr;
                    d_t1 = __ddiv_rn(__dmul_rn(__dsub_rn(rp.b2, rp.b1), __dsub_rn(t, rp.t2)), __dmul_rn(len, len));
                    d_t2 = __ddiv_rn(__dmul_rn(-__dsub_rn(rp.b2, rp.b1), __dsub_rn(t, rp.t1)), __dmul_rn(len, len));
                } else {
                    d_b2 = 1.0;
                }
                const double db[4] = {d_b1, d_b2, rp.swapped ? d_t2 : d_t1, rp.swapped ? d_t1 : d_t2};
#pragma unroll
                for (int j = 0; j < 4; ++j) g_[j * B] = __dadd_rn(g_[j * B], __dmul_rn(dL_dbeta, db[j]));
            }
            g_[gi * B] = __dadd_rn(g_[gi * B], __dmul_rn(__dmul_rn(dt, Ik), __dsub_rn(lR, lI)));
            g_[(gi + 1) * B] = __dadd_rn(g_[(gi + 1) * B], __dmul_rn(__dmul_rn(dt, Ik), __dsub_rn(lD, lI)));
            const double nS = __dadd_rn(lS, __dmul_rn(dt, __dmul_rn(__dmul_rn(b, Ik), __dsub_rn(lI, lS))));
            const double inner = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(-b, Sk), lS),
                                                               __dmul_rn(__dsub_rn(__dsub_rn(__dmul_rn(b, Sk), gam), mu), lI)),
                                                     __dmul_rn(gam, lR)),
                                           __dmul_rn(mu, lD));
            const double nI = __dadd_rn(lI, __dmul_rn(dt, inner));
            lS = nS;
            lI = nI;
            if (k % spd == 0) inject(k / spd, UI[k - k0], IRD ? UR[k - k0] : 0.0, UD[k - k0], lI, lR, lD);
        }
    }
    if (m.fit_I0) g_[(gi + 2) * B] = __dsub_rn(lI, lS);
    loss[p] = Lval;
    for (int d = 0; d < P; ++d) grad[(size_t)d * ldg + p] = g_[d * B];
    if (grad_u0) {
        grad_u0[p] = lS;
        grad_u0[(size_t)ldg + p] = lI;
        grad_u0[2 * (size_t)ldg + p] = lR;
        grad_u0[3 * (size_t)ldg + p] = lD;
    }
}

}  // namespace

size_t adjoint_ckpt_bytes(const WindowDev& w, const ModelDev& m, int M, int C) {
    const long long steps = (long long)(w.n_obs - 1) * m.spd;
    return (size_t)((steps + C - 1) / C) * (m.ird ? 4 : 3) * (size_t)M * sizeof(double);
}

cudaError_t launch_loss_grad_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const double* theta, int ld,
                                 int M, double* loss, double* grad, int ldg, double* grad_u0, double* ckpt, int C,
                                 cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (C < 1 || C > kMaxCkpt) return cudaErrorInvalidValue;
    const int block = 128;
    const size_t nys = m.ird ? 3 * (size_t)obs_stride(w.n_obs) : (size_t)w.n_obs;
    const size_t sm = (nys + 2 * (size_t)m.P * block) * sizeof(double);
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
    switch (m.cost) {
#define SIRD_LG(CV)                                                                                         \
    {                                                                                                       \
        auto kern = m.ird ? loss_grad_f64_kernel<CV, true> : loss_grad_f64_kernel<CV, false>;               \
        if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e == cudaSuccess)                                                                               \
            kern<<<(M + block - 1) / block, block, sm, s>>>(w, m, o, theta, ld, M, loss, grad, ldg, grad_u0, ckpt, C); \
    }                                                                                                       \
    break;
        case COST_MSE: SIRD_LG(COST_MSE)
        case COST_MXSE: SIRD_LG(COST_MXSE)
        case COST_MAE: SIRD_LG(COST_MAE)
        default: SIRD_LG(COST_MAPE)
#undef SIRD_LG
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sird
