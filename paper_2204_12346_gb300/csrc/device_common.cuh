// device_common.cuh -- device helpers shared by the calibration kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sird {

constexpr int kMaxParams = 32;
constexpr int kMaxObs = 4096;

// Device error word bits (kernels OR them in; the host reads the word after a sync).
constexpr unsigned kErrNonFinite = 1u;   // a loss came out NaN (counted as +inf by the swarm)
constexpr unsigned kErrTimeout = 2u;     // a bounded wait ran out
constexpr unsigned kErrBounds = 4u;      // an index check failed (the access was skipped)

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two
// 32x32->64 multiplies with the published multipliers, key bumped by the published
// Weyl constants before every round after the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Uniform in [0,1): the top 24 bits of a word times 2^-24 (exact in float and double).
__device__ __forceinline__ float u01f(uint32_t r) { return __uint2float_rn(r >> 8) * 0x1p-24f; }
__device__ __forceinline__ double u01d(uint32_t r) { return (double)(r >> 8) * 0x1p-24; }

// ---------------------------------------------------------------- compensated sums
// Knuth's TwoSum: s + e == a + b exactly, with s = fl(a + b).  __fadd_rn / __fsub_rn keep
// the compiler from re-associating or contracting.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ---------------------------------------------------------------- packed pairs (f32x2)
// Two independent FP32 lanes in one 64-bit register: lane 0 in the low word.  Every operation
// is the IEEE round-to-nearest operation of each lane (the .f32x2 forms of add / sub / mul /
// fma), so a pair computes exactly what two scalar evaluations compute, with one instruction
// issued per operation instead of two.
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float a, float b) {
    return F2{((unsigned long long)__float_as_uint(b) << 32) | (unsigned long long)__float_as_uint(a)};
}
__device__ __forceinline__ F2 f2(float a) { return f2(a, a); }
__device__ __forceinline__ float f2lo(F2 x) { return __uint_as_float((uint32_t)x.v); }
__device__ __forceinline__ float f2hi(F2 x) { return __uint_as_float((uint32_t)(x.v >> 32)); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 abs2(F2 a) { return F2{a.v & 0x7FFFFFFF7FFFFFFFull}; }

__device__ __forceinline__ void two_sum2(F2 a, F2 b, F2& s, F2& e) {
    s = add2(a, b);
    const F2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

struct Kahan2 {
    F2 sum{0ull}, comp{0ull};
    __device__ __forceinline__ void add(F2 x) {
        const F2 y = sub2(x, comp);
        const F2 t = add2(sum, y);
        comp = sub2(sub2(t, sum), y);
        sum = t;
    }
    // adds the exact product a*b (the compensation is taken off before the single rounding);
    // products enter the sum only this way, so no product is rounded on its own and no
    // optimiser can fuse one into the subtraction in one form but not in the other
    __device__ __forceinline__ void add_prod(F2 a, F2 b) {
        const F2 y = fma2(a, b, F2{comp.v ^ 0x8000000080000000ull});
        const F2 t = add2(sum, y);
        comp = sub2(sub2(t, sum), y);
        sum = t;
    }
};

// Kahan summation step.
struct Kahan {
    float sum = 0.f, comp = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, comp);
        const float t = __fadd_rn(sum, y);
        comp = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
    }
    // adds the exact product a*b: y = fl(a*b - comp) in one rounding
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float y = __fmaf_rn(a, b, -comp);
        const float t = __fadd_rn(sum, y);
        comp = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
    }
};

// ---------------------------------------------------------------- argmin keys
// A float maps to a uint32 whose unsigned order is the float order; NaN maps above +inf.
__device__ __forceinline__ uint32_t ordered_bits(float f) {
    if (f != f) return 0xFFFFFFFFu;
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
// (value, index) packed so that the smallest key is the smallest value, lowest index on ties.
__device__ __forceinline__ unsigned long long argmin_key(float f, uint32_t idx) {
    return ((unsigned long long)ordered_bits(f) << 32) | idx;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Warp minimum of packed keys via two 32-bit warp reductions (value, then index among the
// lanes holding the minimum value); every lane gets the result.
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long key) {
    const uint32_t hi = (uint32_t)(key >> 32);
    const uint32_t mhi = __reduce_min_sync(0xFFFFFFFFu, hi);
    const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, hi == mhi ? (uint32_t)key : 0xFFFFFFFFu);
    return ((unsigned long long)mhi << 32) | lo;
}

// The same over the lanes in `mask` (every lane of the mask calls it with the same mask).
__device__ __forceinline__ unsigned long long masked_min_key(unsigned mask, unsigned long long key) {
    const uint32_t hi = (uint32_t)(key >> 32);
    const uint32_t mhi = __reduce_min_sync(mask, hi);
    const uint32_t lo = __reduce_min_sync(mask, hi == mhi ? (uint32_t)key : 0xFFFFFFFFu);
    return ((unsigned long long)mhi << 32) | lo;
}

// FP64 (value, index) pair with NaN as +inf and lowest index on ties.
struct MinPair64 {
    double f;
    int idx;
};
__device__ __forceinline__ bool pair_less(double fa, int ia, double fb, int ib) {
    const double a = (fa != fa) ? __longlong_as_double(0x7FF0000000000000LL) : fa;
    const double b = (fb != fb) ? __longlong_as_double(0x7FF0000000000000LL) : fb;
    return a < b || (a == b && ia < ib);
}
__device__ __forceinline__ void warp_min_pair(double& f, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double f2 = __shfl_xor_sync(0xFFFFFFFFu, f, o);
        const int i2 = __shfl_xor_sync(0xFFFFFFFFu, idx, o);
        if (pair_less(f2, i2, f, idx)) {
            f = f2;
            idx = i2;
        }
    }
}

}  // namespace sird
