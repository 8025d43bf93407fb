// adjoint.cu -- exact gradient of the discrete loss by the discrete adjoint of the Euler map.
//
// The paper calibrates with PSO because no gradient is at hand (Sec. 3.3).  The Euler-discretised
// loss does have one: with u_{k+1} = u_k + dt f(u_k, theta) (eq. (SIRD), f = (-bSI, bSI - (gamma
// + mu) I, gamma I, mu I), b = beta/N) and L = C(e_1..e_n), the adjoint runs backwards
//     lambda_k = lambda_{k+1} + dt (df/du)^T lambda_{k+1} + dL/du_k   (dL/dD at observation steps)
//     dL/dtheta += dt (df/dtheta)^T lambda_{k+1}
// and dL/du_0 = lambda_0; with S0 = N - I0 - R0 - D0, dL/dI0 = lambda_I(0) - lambda_S(0).
// R never feeds back into S, I or D and the F_D losses do not see it, so lambda_R stays 0.
//
// One thread per parameter vector.  The forward pass stores (S, I, D) every `ckpt` steps in
// global scratch ([checkpoint][3][M], coalesced); the backward pass recomputes each
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

struct RampF64 {
    double b1, b2, t1, t2;
    bool swapped;
};

__device__ __forceinline__ double ramp_beta(const RampF64& r, double t) {
    if (t < r.t1) return r.b1;
    if (t < r.t2) return __dadd_rn(r.b1, __dmul_rn(__ddiv_rn(__dsub_rn(r.b2, r.b1), __dsub_rn(r.t2, r.t1)), __dsub_rn(t, r.t1)));
    return r.b2;
}

template <int COST>
__global__ void __launch_bounds__(128) loss_grad_f64_kernel(WindowDev w, ModelDev m, ObsDev o,
                                                             const double* __restrict__ theta, int ld, int M,
                                                             double* __restrict__ loss, double* __restrict__ grad,
                                                             int ldg, double* __restrict__ grad_u0,
                                                             double* __restrict__ ckpt, int C) {
    extern __shared__ double dsm[];
    const int B = blockDim.x, tid = threadIdx.x, P = m.P;
    double* ys = dsm;
    double* th = dsm + w.n_obs;    // [P][B]
    double* g = th + P * B;        // [P][B] gradient accumulators
    for (int i = tid; i < w.n_obs; i += B) ys[i] = o.yd[i];
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

    // ---- forward: loss (same order as the plain evaluation) and checkpoints
    double S = __dsub_rn(__dsub_rn(__dsub_rn(N, I0), w.R0), w.D0), I = I0, D = w.D0;
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
    observe(0, D);
    for (int k = 0; k < steps; ++k) {
        if (k % C == 0) {
            const size_t base = (size_t)(k / C) * 3 * M + p;
            ckpt[base] = S;
            ckpt[base + M] = I;
            ckpt[base + 2 * (size_t)M] = D;
        }
        euler_f64(__ddiv_rn(beta_at(k), N), gm, mu, dt, S, I, D);
        if ((k + 1) % spd == 0) observe((k + 1) / spd, D);
    }
    double Lval;
    if (COST == COST_MSE || COST == COST_MAE) Lval = __ddiv_rn(acc, (double)n);
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

    // ---- backward over checkpointed stretches
    double lS = 0.0, lI = 0.0, lR = 0.0, lD = gD(n - 1, D);
    double US[kMaxCkpt + 1], UI[kMaxCkpt + 1], UD[kMaxCkpt + 1];
    const int nck = (steps + C - 1) / C;
    for (int c = nck - 1; c >= 0; --c) {
        const int k0 = c * C, k1 = min(k0 + C, steps);
        const size_t base = (size_t)c * 3 * M + p;
        double s = ckpt[base], i_ = ckpt[base + M], d_ = ckpt[base + 2 * (size_t)M];
        US[0] = s;
        UI[0] = i_;
        UD[0] = d_;
        for (int k = k0; k < k1 - 1; ++k) {  // recompute states k0+1 .. k1-1 of this stretch
            euler_f64(__ddiv_rn(beta_at(k), N), gm, mu, dt, s, i_, d_);
            US[k - k0 + 1] = s;
            UI[k - k0 + 1] = i_;
            UD[k - k0 + 1] = d_;
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
            if (k % spd == 0) lD = __dadd_rn(lD, gD(k / spd, UD[k - k0]));
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
    return (size_t)((steps + C - 1) / C) * 3 * (size_t)M * sizeof(double);
}

cudaError_t launch_loss_grad_f64(const WindowDev& w, const ModelDev& m, const ObsDev& o, const double* theta, int ld,
                                 int M, double* loss, double* grad, int ldg, double* grad_u0, double* ckpt, int C,
                                 cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (C < 1 || C > kMaxCkpt) return cudaErrorInvalidValue;
    const int block = 128;
    const size_t sm = ((size_t)w.n_obs + 2 * (size_t)m.P * block) * sizeof(double);
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
    switch (m.cost) {
#define SIRD_LG(CV)                                                                                         \
    {                                                                                                       \
        auto kern = loss_grad_f64_kernel<CV>;                                                               \
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
