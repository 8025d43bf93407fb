// traj_f32.cuh -- the FP32 trajectory of eq. (SIRD) and its daily misfits, shared by every FP32
// kernel (evaluation, swarm, batch, adjoint forward pass, forecast).
//
// One template integrates one trajectory (T = float) or two in packed f32x2 pairs (T = F2):
// both run the same operations in the same order, so a pair's losses equal the single
// evaluations' bit for bit.
//
// The explicit Euler step of eq. (SIRD) with cb = dt beta/N, a = dt (gamma + mu), dm = dt mu,
//     S' = S - cb S I,  I' = I (1 + g),  g = cb S - a,  D' = D + dm I,  R' = R + dr I (dr = dt gamma),
// is carried in a form whose FP32 rounding stays near 1e-8 of I over thousands of steps:
//
//   * Q = S + I changes only by removals: over a day, Q_end = Q_start - a sum_k I_k.  Within a
//     day, S_k = Q_start - I_k - a isum_k (isum_k = sum_{j<k} I_j, exact in exact arithmetic), so
//         g_k = G - cb X_k,   X_k = I_k + a isum_k,   G = cb Q_start - a,
//     where G (the day's growth rate at I = 0) is a per-day constant held as a (hi, lo) pair and
//     cb X_k is a small term.  A step is then two FMAs for g and one FMA for I, with the rounding
//     error of the I update recovered exactly (fma(g, I, I - r)) into a low part Il.
//   * The day's sum of I is needed to ~1e-9: it is spd Is + W - A, where Is is the day's first I
//     (hi part), W = sum_k Il_k, and A = sum_k (spd - 1 - k) d_k with d_k = I_k - I_{k+1} (hi
//     parts) the exact per-step decrements.
//   * Day end: Il receives the growth the steps could not apply (G's low part and cb's low part
//     times the day's sum, and g times the low parts, G W) and is folded into I; G takes the
//     day's removals, G -= cb a (day's sum), as a pair; the deaths' misfit e = y - Dhat follows
//     e_i = e_{i-1} + (y_i - y_{i-1}) - dm sum_day I, with y_i - y_{i-1} - dmh Psh in one
//     rounding (it cancels at a good fit), which keeps e's rounding relative to e itself rather
//     than to D.  The observations arrive as y_i - y_0 in FP32 (exact differences for counts
//     below 2^24 over the window, whatever the level of y).
//   * Q itself is needed only where a transmission segment starts: there it is recovered from
//     the ending segment's G as Q = (G + a) / cb (a pair quotient).  Where that cb is 0, G says
//     nothing about Q, and Q is carried through the segment's days instead (Q -= a day's sum);
//     observers that read Q at day starts (the adjoint's checkpoints) get it carried every day.
//   * A transmission segment that starts inside a day switches (G, cb) at its step; the part of
//     the day run with the old constants is accounted for at the switch.
//   * The ramp of eq. (beta) changes beta every step: G_k and cb_k follow the ramp per step
//     (G1 + u_k HS between t1 and t2, G1 / G2 outside), from the pairs G1 = cb(beta1) Q - a,
//     G2 = cb(beta2) Q - a and HS = d cb/dt Q, set from the initial Q and then given each day's
//     removals like G; u_k = t_k - t1 is formed from the day (exact) and the step's offset.
//   * F_IRD carries the recovered series' misfit eR like e (dr = dt gamma) and compares I's
//     (hi, lo) pair with the reported I.
//
// Window and step conventions (Sec. 3.1): observations on days 0..L, Euler from D0 = y_0, the
// state after i*spd steps is compared with y_i; PWC segment j covers steps
// [ceil(j S/K), ceil((j+1) S/K)); beta at the left end of each step.
#pragma once

#include <climits>
#include <type_traits>

#include "device_common.cuh"

namespace sird {

// ---------------------------------------------------------------- lane-generic arithmetic
// Every operation is IEEE round-to-nearest; no contraction or reassociation.
__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float tadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float tsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float tmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float tneg(float a) { return __uint_as_float(__float_as_uint(a) ^ 0x80000000u); }
__device__ __forceinline__ F2 tfma(F2 a, F2 b, F2 c) { return fma2(a, b, c); }
__device__ __forceinline__ F2 tadd(F2 a, F2 b) { return add2(a, b); }
__device__ __forceinline__ F2 tsub(F2 a, F2 b) { return sub2(a, b); }
__device__ __forceinline__ F2 tmul(F2 a, F2 b) { return mul2(a, b); }
__device__ __forceinline__ F2 tneg(F2 a) { return F2{a.v ^ 0x8000000080000000ull}; }

template <class T>
__device__ __forceinline__ T tsplat(float x);
template <>
__device__ __forceinline__ float tsplat<float>(float x) { return x; }
template <>
__device__ __forceinline__ F2 tsplat<F2>(float x) { return f2(x); }

// per-lane select: c ? a : b with a lane mask (bit 0: lane 0, bit 1: lane 1)
__device__ __forceinline__ float tsel(unsigned c, float a, float b) { return (c & 1u) ? a : b; }
__device__ __forceinline__ F2 tsel(unsigned c, F2 a, F2 b) {
    return f2((c & 1u) ? f2lo(a) : f2lo(b), (c & 2u) ? f2hi(a) : f2hi(b));
}
// per-lane comparisons as lane masks
__device__ __forceinline__ unsigned tlt(float a, float b) { return a < b ? 1u : 0u; }
__device__ __forceinline__ unsigned tlt(F2 a, F2 b) {
    return (f2lo(a) < f2lo(b) ? 1u : 0u) | (f2hi(a) < f2hi(b) ? 2u : 0u);
}
__device__ __forceinline__ unsigned tge(float a, float b) { return a >= b ? 1u : 0u; }
__device__ __forceinline__ unsigned tge(F2 a, F2 b) {
    return (f2lo(a) >= f2lo(b) ? 1u : 0u) | (f2hi(a) >= f2hi(b) ? 2u : 0u);
}

// ---------------------------------------------------------------- error-free pieces
// a*b = h + l exactly
template <class T>
__device__ __forceinline__ void tprod(T a, T b, T& h, T& l) {
    h = tmul(a, b);
    l = tfma(a, b, tneg(h));
}
// renormalise (h, l) with |h| >= |l| (Fast2Sum)
template <class T>
__device__ __forceinline__ void tnorm(T& h, T& l) {
    const T s = tadd(h, l);
    l = tsub(l, tsub(s, h));
    h = s;
}
// a + b = s + e exactly (Knuth's TwoSum)
template <class T>
__device__ __forceinline__ void ttwo_sum(T a, T b, T& s, T& e) {
    s = tadd(a, b);
    const T bb = tsub(s, a);
    e = tadd(tsub(a, tsub(s, bb)), tsub(b, bb));
}
// (h, l) = c x with c = (ch, cl) a pair and x a float (exact product of the hi parts)
template <class T>
__device__ __forceinline__ void tmul_pair(T ch, T cl, T x, T& h, T& l) {
    tprod(ch, x, h, l);
    l = tfma(cl, x, l);
    tnorm(h, l);
}
// G = cb Q - a as a pair from the pairs cb, Q, a
template <class T>
__device__ __forceinline__ void growth_pair(T cbh, T cbl, T Qh, T Ql, T ah, T al, T& Gh, T& Gl) {
    T p, pe;
    tprod(cbh, Qh, p, pe);
    pe = tfma(cbh, Ql, tfma(cbl, Qh, pe));
    T s, er;
    ttwo_sum(p, tneg(ah), s, er);
    Gh = s;
    Gl = tadd(er, tsub(pe, al));
    tnorm(Gh, Gl);
}

// Q = (G + a) / cb from G = cb Q - a as a pair (cb != 0; the caller selects another Q where
// cb = 0).  The quotient's residual is formed exactly by the FMA, so the hardware's approximate
// reciprocal (a few ulp) serves: the pair still holds Q to ~2^-44.
__device__ __forceinline__ float trcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ F2 trcp(F2 x) { return f2(trcp(f2lo(x)), trcp(f2hi(x))); }
template <class T>
__device__ __forceinline__ void q_from_growth(T Gh, T Gl, T cbh, T cbl, T ah, T al, T& Qh, T& Ql) {
    T sh, se;
    ttwo_sum(Gh, ah, sh, se);
    se = tadd(se, tadd(Gl, al));
    const T rc = trcp(cbh);
    Qh = tmul(sh, rc);
    const T nq = tneg(Qh);
    Ql = tmul(tfma(nq, cbl, tadd(tfma(nq, cbh, sh), se)), rc);
}
// G -= c s for a coefficient pair c and the day's sum s = (Psh, Psl)
template <class T, bool NORM>
__device__ __forceinline__ void remove_pair(T ch, T cl, T Psh, T Psl, T& Gh, T& Gl) {
    const T dd = tfma(ch, Psh, tfma(ch, Psl, tmul(cl, Psh)));
    const T s = tsub(Gh, dd);
    const T er = tsub(tsub(Gh, s), dd);
    Gh = s;
    Gl = tadd(Gl, er);
    if (NORM) tnorm(Gh, Gl);
}
// (h, l) = x y for two pairs, to the pair's precision
template <class T>
__device__ __forceinline__ void tmul_pairs(T xh, T xl, T yh, T yl, T& h, T& l) {
    tprod(xh, yh, h, l);
    l = tfma(xh, yl, tfma(xl, yh, l));
}
__device__ __forceinline__ unsigned teq0(float a) { return a == 0.f ? 1u : 0u; }
__device__ __forceinline__ unsigned teq0(F2 a) { return (f2lo(a) == 0.f ? 1u : 0u) | (f2hi(a) == 0.f ? 2u : 0u); }

// An observer that reads Q = S + I at day starts declares kWantsQ = true; the others leave Q out.
template <class O, class = void>
struct obs_wants_q : std::false_type {};
template <class O>
struct obs_wants_q<O, std::void_t<decltype(O::kWantsQ)>> : std::integral_constant<bool, O::kWantsQ> {};
// An observer with kLeanRegs = true asks the trajectory to recompute per-segment masks where they
// are used instead of keeping them live (for kernels at their register bound); same arithmetic.
template <class O, class = void>
struct obs_lean : std::false_type {};
template <class O>
struct obs_lean<O, std::void_t<decltype(O::kLeanRegs)>> : std::integral_constant<bool, O::kLeanRegs> {};

// ---------------------------------------------------------------- Kahan sum of exact products
template <class T>
struct KahanT {
    T sum, comp;
    __device__ __forceinline__ void init() { sum = comp = tsplat<T>(0.f); }
    __device__ __forceinline__ void add(T x) {
        const T y = tsub(x, comp);
        const T t = tadd(sum, y);
        comp = tsub(tsub(t, sum), y);
        sum = t;
    }
    // adds the exact product a*b: y = fl(a*b - comp) in one rounding
    __device__ __forceinline__ void add_prod(T a, T b) {
        const T y = tfma(a, b, tneg(comp));
        const T t = tadd(sum, y);
        comp = tsub(tsub(t, sum), y);
        sum = t;
    }
};

__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ F2 tabs(F2 a) { return F2{a.v & 0x7FFFFFFF7FFFFFFFull}; }
__device__ __forceinline__ float tmaxsq(float m, float e) { return fmaxf(m, __fmul_rn(e, e)); }
__device__ __forceinline__ F2 tmaxsq(F2 m, F2 e) {
    const F2 e2 = mul2(e, e);
    return f2(fmaxf(f2lo(m), f2lo(e2)), fmaxf(f2hi(m), f2hi(e2)));
}

// One series' cost (Sec. 3.1) over the days e is reported for: MSE / MAE the mean over n, MXSE
// the largest e^2, MAPE 100 x the mean |e|/|y| over the nonzero y (invy = 0 where y == 0).
template <class T, int COST>
struct CostT {
    KahanT<T> k;
    T mx;
    __device__ __forceinline__ void init() {
        k.init();
        mx = tsplat<T>(0.f);
    }
    __device__ __forceinline__ void add(T e, float invy) {
        if (COST == 0) k.add_prod(e, e);
        else if (COST == 2) k.add(tabs(e));
        else if (COST == 3) k.add_prod(tabs(e), tsplat<T>(invy));
        else mx = tmaxsq(mx, e);
    }
    __device__ __forceinline__ float lane_result(float s, float m, int n, int n_kept) const {
        if (COST == 0 || COST == 2) return __fdiv_rn(s, (float)n);
        if (COST == 3) return n_kept > 0 ? __fdiv_rn(__fmul_rn(100.f, s), (float)n_kept) : 0.f;
        return m;
    }
    __device__ __forceinline__ void result(int n, int n_kept, float& fa, float& fb) const;
};
template <>
__device__ __forceinline__ void CostT<float, 0>::result(int n, int n_kept, float& fa, float& fb) const {
    fa = fb = lane_result(k.sum, mx, n, n_kept);
}
template <>
__device__ __forceinline__ void CostT<float, 1>::result(int n, int n_kept, float& fa, float& fb) const {
    fa = fb = lane_result(k.sum, mx, n, n_kept);
}
template <>
__device__ __forceinline__ void CostT<float, 2>::result(int n, int n_kept, float& fa, float& fb) const {
    fa = fb = lane_result(k.sum, mx, n, n_kept);
}
template <>
__device__ __forceinline__ void CostT<float, 3>::result(int n, int n_kept, float& fa, float& fb) const {
    fa = fb = lane_result(k.sum, mx, n, n_kept);
}
#define SIRD_COSTT_F2_RESULT(C)                                                                          \
    template <>                                                                                          \
    __device__ __forceinline__ void CostT<F2, C>::result(int n, int n_kept, float& fa, float& fb) const { \
        fa = lane_result(f2lo(k.sum), f2lo(mx), n, n_kept);                                              \
        fb = lane_result(f2hi(k.sum), f2hi(mx), n, n_kept);                                              \
    }
SIRD_COSTT_F2_RESULT(0)
SIRD_COSTT_F2_RESULT(1)
SIRD_COSTT_F2_RESULT(2)
SIRD_COSTT_F2_RESULT(3)
#undef SIRD_COSTT_F2_RESULT

// ---------------------------------------------------------------- parameter access
// theta_d of one vector at p[d * stride], or of two vectors packed lane by lane.
struct ThetaF1 {
    const float* p;
    int stride;
    __device__ __forceinline__ float operator()(int d) const { return p[d * stride]; }
};
struct ThetaF2 {
    const float *a, *b;
    int stride;
    __device__ __forceinline__ F2 operator()(int d) const { return f2(a[d * stride], b[d * stride]); }
};

// ---------------------------------------------------------------- the trajectory
// What a day end reports: e = y_D - Dhat (exact up to ~1e-8 of D), the infectious (Ih, Il),
// and for F_IRD eR = y_R - Rhat.  Observers implement
//     day_start(int day, T Qh, T Ql, T Ih, T Il, T e)     (before the day's first step)
//     day_end(int day, T e, T Ih, T Il, T eR)             (after its last)
// and see days 1..n_days (n_days may pass the window: then y stays at its last value, so e
// continues as y_L - Dhat).
// PWC segment j's first step: ceil(j*steps/K).
__device__ __forceinline__ int traj_segment_start(int j, int steps, int K) {
    return (int)(((long long)j * steps + K - 1) / K);
}

// Windows of more than this many steps run in the long-window mode (EXACTG), where rounding
// errors that otherwise add up with the square root of the steps or days are carried: the
// rounding of g each step (its error, recovered by one FMA, enters I's low part: three more
// operations a step), G renormalised after each day's update, and the misfits e and eR kept as
// (hi, lo) pairs with an exact TwoSum per day.
constexpr int kExactGrowthSteps = 1000;

template <class T, int SPD, bool RAMP, bool IRD, bool DTRACK = false, bool EXACTG = false, class Th, class Obs>
__device__ __forceinline__ void trajectory_f32(const WindowDev& w, const ModelDev& m, const float* __restrict__ ysD,
                                               const float* __restrict__ ysR, Th th, int n_days, Obs& obs) {
    const int spd = SPD > 0 ? SPD : m.spd;
    const int L = w.n_obs - 1, steps = L * spd;
    const T fspd = tsplat<T>((float)spd);
    const int gi = RAMP ? 4 : m.K;
    const T gam = th(gi), mu = th(gi + 1);
    T Ih = m.fit_I0 ? th(gi + 2) : tsplat<T>(w.I0f);
    T Il = tsplat<T>(m.fit_I0 ? 0.f : w.I0l);  // a given I0 enters as a pair
    const T dth = tsplat<T>(w.dt_h), dtl = tsplat<T>(w.dt_l);
    // a = dt (gamma + mu), dm = dt mu, dr = dt gamma as pairs, and spd times each
    T ah, al, dmh, dml, drh = tsplat<T>(0.f), drl = tsplat<T>(0.f);
    {
        T gs, ge;
        ttwo_sum(gam, mu, gs, ge);
        tprod(gs, dth, ah, al);
        al = tfma(gs, dtl, tfma(ge, dth, al));
        tnorm(ah, al);
        tprod(mu, dth, dmh, dml);
        dml = tfma(mu, dtl, dml);
        tnorm(dmh, dml);
        if (IRD) {
            tprod(gam, dth, drh, drl);
            drl = tfma(gam, dtl, drl);
            tnorm(drh, drl);
        }
    }
    const T ndmh = tneg(dmh), ndml = tneg(dml), ndrh = tneg(drh), ndrl = tneg(drl);
    const T cbnh = tsplat<T>(w.cbn_h), cbnl = tsplat<T>(w.cbn_l);
    auto cb_pair = [&](T beta, T& h, T& l) {  // cb = beta dt/N
        tprod(beta, cbnh, h, l);
        l = tfma(beta, cbnl, l);
        tnorm(h, l);
    };

    T Qh = tsplat<T>(w.Q0h), Ql = tsplat<T>(w.Q0l);
    // e_0 = y_0 - D0 = 0 (Euler starts from the first observation); eR_0 = y_R0 - R0.  ysD and
    // ysR hold y_i - y_0 (only their differences are used).  With DTRACK the observations are
    // ignored, ysD[0] holds D0 and e = -D (its rounding then relative to D).
    T e = tsplat<T>(DTRACK ? -ysD[0] : 0.f), eR = tsplat<T>(IRD ? w.eR0 : 0.f);
    T el = tsplat<T>(0.f), eRl = el;  // low parts of e, eR (long-window mode)
    float yprev = ysD[0], yRprev = IRD ? ysR[0] : 0.f;
    T isum = tsplat<T>(0.f), W = isum, A = isum, Is = Ih;
    obs.day_end(0, e, Ih, Il, eR);

    // day end: corrections, fold, removals into the growth rates (remove(Psh, Psl)) and Q,
    // misfits.  The day's sum of I is Psh + Psl with (Psh, Psl0) = spd Is exactly and Psl = Psl0
    // + W - A.  The removals come first: the next day's first step waits for them.
    constexpr bool kQ = obs_wants_q<Obs>::value;
    auto close_day = [&](int day, T Gh_, T Gl_, T ncbl_, bool trackQ, const auto& remove) {
        T Psh, Psl;
        tprod(fspd, Is, Psh, Psl);
        Psl = tadd(Psl, tsub(W, A));
        if (EXACTG) tnorm(Psh, Psl);  // short windows: Q's low part may grow, it is carried as is
        Il = tfma(Gh_, W, tfma(tfma(ncbl_, Is, Gl_), isum, Il));
        tnorm(Ih, Il);
        remove(Psh, Psl);
        if (kQ || trackQ) {   // Q -= a (day's sum)
            T qh, ql;
            tprod(ah, Psh, qh, ql);
            ql = tfma(ah, Psl, tfma(al, Psh, ql));
            const T s = tsub(Qh, qh);
            const T er = tsub(tsub(Qh, s), qh);
            Qh = s;
            Ql = tadd(Ql, tsub(er, ql));
        }
        {   // e += (y_day - y_{day-1}) - dm (day's sum)
            const float y = (day <= L && !DTRACK) ? ysD[day] : yprev;
            const T dy = tsplat<T>(__fsub_rn(y, yprev));
            yprev = y;
            if (EXACTG) {
                T dh, dl;
                tprod(dmh, Psh, dh, dl);
                dl = tfma(dmh, Psl, tfma(dml, Psh, dl));
                T s, er;
                ttwo_sum(e, tsub(dy, dh), s, er);
                e = s;
                el = tadd(el, tsub(er, dl));
            } else {  // dy - dmh Psh in one rounding (it cancels at a fit), then the low terms
                e = tadd(e, tfma(ndmh, Psl, tfma(ndml, Psh, tfma(ndmh, Psh, dy))));
            }
        }
        if (IRD) {  // eR += (yR_day - yR_{day-1}) - dr (day's sum)
            const float y = day <= L ? ysR[day] : yRprev;
            const T dy = tsplat<T>(__fsub_rn(y, yRprev));
            yRprev = y;
            if (EXACTG) {
                T rh, rl;
                tprod(drh, Psh, rh, rl);
                rl = tfma(drh, Psl, tfma(drl, Psh, rl));
                T s, er;
                ttwo_sum(eR, tsub(dy, rh), s, er);
                eR = s;
                eRl = tadd(eRl, tsub(er, rl));
            } else {
                eR = tadd(eR, tfma(ndrh, Psl, tfma(ndrl, Psh, tfma(ndrh, Psh, dy))));
            }
        }
        if (EXACTG) obs.day_end(day, tadd(e, el), Ih, Il, tadd(eR, eRl));
        else obs.day_end(day, e, Ih, Il, eR);
        isum = W = A = tsplat<T>(0.f);
        Is = Ih;
    };

    if (!RAMP) {
        // ---- piecewise-constant beta: segment-major, whole days unrolled
        const int K = m.K;
        T Gh = tsplat<T>(0.f), Gl = Gh, ncbh = Gh, ncbl = Gh, cbah = Gh, cbal = Gh;
        int k = 0, day = 0, in_day = 0;
        // lanes whose segment has cb = 0, where G does not determine Q
        constexpr bool kLean = obs_lean<Obs>::value;
        unsigned zero = 0u;
        auto cb_zero = [&]() { return kLean ? teq0(ncbh) : zero; };
        auto end_day = [&]() {
            close_day(day, Gh, Gl, ncbl, cb_zero() != 0u,
                      [&](T Psh, T Psl) { remove_pair<T, EXACTG>(cbah, cbal, Psh, Psl, Gh, Gl); });
        };
        // one step with weight spd-1-j for the day's sum (any j; the first step of a day finds
        // isum = W = A = 0)
        auto step = [&](T wj) {
            const T X = tfma(ah, isum, Ih);
            const T g = tfma(ncbh, X, Gh);
            isum = tadd(isum, Ih);
            W = tadd(W, Il);
            const T r = tfma(g, Ih, Ih);
            const T d = tsub(Ih, r);
            A = tfma(wj, d, A);
            if (EXACTG) Il = tfma(tfma(ncbh, X, tsub(Gh, g)), Ih, tadd(Il, tfma(g, Ih, d)));
            else Il = tadd(Il, tfma(g, Ih, d));
            Ih = r;
        };
        // the first step of a day: isum = W = A = 0
        auto step0 = [&](T wj) {
            const T g = tfma(ncbh, Ih, Gh);
            isum = Ih;
            W = Il;
            const T r = tfma(g, Ih, Ih);
            const T d = tsub(Ih, r);
            A = tmul(wj, d);
            if (EXACTG) Il = tfma(tfma(ncbh, Ih, tsub(Gh, g)), Ih, tadd(Il, tfma(g, Ih, d)));
            else Il = tadd(Il, tfma(g, Ih, d));
            Ih = r;
        };
        const int last_day = n_days;
        for (int seg = 0; seg < K; ++seg) {
            const T beta = th(seg);
            T cbh, cbl;
            cb_pair(beta, cbh, cbl);
            if (seg > 0) {  // the day-start Q from the ending segment's G where its cb is not 0
                T qh, ql;
                q_from_growth(Gh, Gl, tneg(ncbh), tneg(ncbl), ah, al, qh, ql);
                const unsigned z = cb_zero();
                Qh = tsel(z, Qh, qh);
                Ql = tsel(z, Ql, ql);
            }
            T cah, cal;
            tprod(cbh, ah, cah, cal);
            cal = tfma(cbh, al, tfma(cbl, ah, cal));
            T nGh, nGl;
            growth_pair(cbh, cbl, Qh, Ql, ah, al, nGh, nGl);  // Q is the day-start value
            if (in_day > 0) {
                // the day so far ran on the previous segment's constants: account for the
                // difference of the low-part corrections the day end will apply with the new ones
                const T ncbl_new = tneg(cbl);
                Il = tfma(tsub(Gh, nGh), W,
                          tfma(tsub(tfma(ncbl, Is, Gl), tfma(ncbl_new, Is, nGl)), isum, Il));
            }
            Gh = nGh;
            Gl = nGl;
            ncbh = tneg(cbh);
            ncbl = tneg(cbl);
            if (!kLean) zero = teq0(cbh);
            cbah = cah;
            cbal = cal;
            // the last segment runs on past the window (forecast)
            const int kend = seg + 1 < K ? traj_segment_start(seg + 1, steps, K) : INT_MAX;
            while (in_day != 0 && k < kend) {  // finish a day begun by the previous segment
                step(tsplat<T>((float)(spd - 1 - in_day)));
                ++k;
                if (++in_day == spd) {
                    ++day;
                    in_day = 0;
                    end_day();
                    if (day == last_day) return;
                }
            }
            while ((long long)k + spd <= (long long)kend) {  // whole days
                obs.day_start(day, Qh, Ql, Ih, Il, EXACTG ? tadd(e, el) : e);
                if (SPD > 0) {
                    step0(tsplat<T>((float)(SPD - 1)));
#pragma unroll
                    for (int s = 1; s < (SPD > 0 ? SPD : 1); ++s) step(tsplat<T>((float)(SPD - 1 - s)));
                } else {
                    step0(tsplat<T>((float)(spd - 1)));
                    for (int s = 1; s < spd; ++s) step(tsplat<T>((float)(spd - 1 - s)));
                }
                k += spd;
                ++day;
                end_day();
                if (day == last_day) return;
            }
            while (k < kend) {  // start a day the next segment finishes
                if (in_day == 0) obs.day_start(day, Qh, Ql, Ih, Il, EXACTG ? tadd(e, el) : e);
                step(tsplat<T>((float)(spd - 1 - in_day)));
                ++k;
                ++in_day;
            }
        }
        return;
    }

    // ---- ramp of eq. (beta): beta1 before t1, linear to beta2 on [t1, t2), beta2 after
    {
        const T b1 = th(0), b2 = th(1), ta = th(2), tb = th(3);
        T t1, t2;
        {
            const unsigned sw = tlt(tb, ta);
            t1 = tsel(sw, tb, ta);
            t2 = tsel(sw, ta, tb);
        }
        const T umax = tsub(t2, t1);
        // d cb / dt = (beta2 - beta1)/(t2 - t1) dt/N as a pair (0 for an empty ramp)
        T hh, hl;
        {
            const unsigned empty = tge(t1, t2);
            const T len = tsel(empty, tsplat<T>(1.f), umax);
            const T db = tsub(b2, b1);
            T sh;
            if constexpr (sizeof(T) == 4) sh = __fdiv_rn(db, len);
            else sh = f2(__fdiv_rn(f2lo(db), f2lo(len)), __fdiv_rn(f2hi(db), f2hi(len)));
            // residual of the quotient: (db - sh len) / len
            const T rr = tfma(tneg(sh), len, db);
            T sl;
            if constexpr (sizeof(T) == 4) sl = __fdiv_rn(rr, len);
            else sl = f2(__fdiv_rn(f2lo(rr), f2lo(len)), __fdiv_rn(f2hi(rr), f2hi(len)));
            sh = tsel(empty, tsplat<T>(0.f), sh);
            sl = tsel(empty, tsplat<T>(0.f), sl);
            tprod(sh, cbnh, hh, hl);
            hl = tfma(sh, cbnl, tfma(sl, cbnh, hl));
            tnorm(hh, hl);
        }
        T c1h, c1l, c2h, c2l;
        cb_pair(b1, c1h, c1l);
        cb_pair(b2, c2h, c2l);
        const T nc1h = tneg(c1h), nc2h = tneg(c2h), nhh = tneg(hh);
        const T dtf = tsplat<T>(__fadd_rn(w.dt_h, w.dt_l));
        // G1 = cb(beta1) Q - a, G2 = cb(beta2) Q - a and HS = d cb/dt Q from the initial Q, then
        // each day's removals a (day's sum) applied to them through the pairs cb(beta1) a, cb(beta2) a
        // and d cb/dt a
        T G1h, G1l, G2h, G2l, HSh, HSl;
        growth_pair(c1h, c1l, Qh, Ql, ah, al, G1h, G1l);
        growth_pair(c2h, c2l, Qh, Ql, ah, al, G2h, G2l);
        tprod(hh, Qh, HSh, HSl);
        HSl = tfma(hh, Ql, tfma(hl, Qh, HSl));
        tnorm(HSh, HSl);
        T c1ah, c1al, c2ah, c2al, hah, hal;
        tmul_pairs(c1h, c1l, ah, al, c1ah, c1al);
        tmul_pairs(c2h, c2l, ah, al, c2ah, c2al);
        tmul_pairs(hh, hl, ah, al, hah, hal);
        for (int day = 0; day < n_days; ++day) {
            const T us = tsub(tsplat<T>((float)day), t1);  // t at the day's start minus t1
            obs.day_start(day, Qh, Ql, Ih, Il, EXACTG ? tadd(e, el) : e);
            auto step = [&](int j, T wj) {
                const T u = tfma(tsplat<T>((float)j), dtf, us);
                const unsigned before = tlt(u, tsplat<T>(0.f)), after = tge(u, umax);
                const T Glin = tfma(u, HSh, G1h);
                const T nclin = tfma(u, nhh, nc1h);
                const T Gk = tsel(before, G1h, tsel(after, G2h, Glin));
                const T ncb = tsel(before, nc1h, tsel(after, nc2h, nclin));
                const T X = tfma(ah, isum, Ih);
                const T g = tfma(ncb, X, Gk);
                isum = tadd(isum, Ih);
                W = tadd(W, Il);
                const T r = tfma(g, Ih, Ih);
                const T d = tsub(Ih, r);
                A = tfma(wj, d, A);
                if (EXACTG) Il = tfma(tfma(ncb, X, tsub(Gk, g)), Ih, tadd(Il, tfma(g, Ih, d)));
                else Il = tadd(Il, tfma(g, Ih, d));
                Ih = r;
            };
            if (SPD > 0) {
#pragma unroll
                for (int s = 0; s < (SPD > 0 ? SPD : 1); ++s) step(s, tsplat<T>((float)(SPD - 1 - s)));
            } else {
                for (int s = 0; s < spd; ++s) step(s, tsplat<T>((float)(spd - 1 - s)));
            }
            // the day's low parts, taken in the regime of its middle step
            const T um = tfma(tsplat<T>(0.5f * (float)(spd - 1)), dtf, us);
            const unsigned before = tlt(um, tsplat<T>(0.f)), after = tge(um, umax);
            const T Glm = tsel(before, G1l, tsel(after, G2l, tfma(um, HSl, G1l)));
            const T Ghm = tsel(before, G1h, tsel(after, G2h, tfma(um, HSh, G1h)));
            const T ncl = tneg(tsel(before, c1l, tsel(after, c2l, tfma(um, hl, c1l))));
            close_day(day + 1, Ghm, Glm, ncl, false, [&](T Psh, T Psl) {
                remove_pair<T, EXACTG>(c1ah, c1al, Psh, Psl, G1h, G1l);
                remove_pair<T, EXACTG>(c2ah, c2al, Psh, Psl, G2h, G2l);
                remove_pair<T, EXACTG>(hah, hal, Psh, Psl, HSh, HSl);
            });
        }
    }
}

}  // namespace sird
