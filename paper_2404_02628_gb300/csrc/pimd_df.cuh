// Double-float arithmetic with a wide exponent, for sm_103a.
//
// On GB300 an FP64 instruction issues once per 64 cycles per warp and has a
// 64-cycle dependent latency, while FP32 runs at 128 lanes/clk/SM with a
// 4.5-cycle latency.  The exchange part of the PIMD force field (arXiv
// 2404.02628, Sec. III) needs FP64-grade relative accuracy on every factor
// exp(-kappa |dr|^2), so its per-term arithmetic is carried out here on the
// FP32 pipe in double-float form: a value is hi + lo with |lo| <= ulp(hi)/2
// (about 48 significant bits), built from the error-free transformations
// TwoSum (Knuth) and TwoProduct via fused multiply-add.  A separate int32
// binary exponent ("Dfw") keeps sums of non-negative terms whose logarithms
// span thousands free of overflow and underflow.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pimd_device.cuh"

struct df {
    float h, l;
};

// a + b exactly as h + l (Knuth's TwoSum, no magnitude assumption)
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// a + b exactly for |a| >= |b| (Dekker's FastTwoSum)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

// a * b exactly as h + l
__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df{p, e};
}

// Double-float sum with error at most ~2^-47 (|a| + |b|); fine for any signs
// when absolute accuracy relative to |a| + |b| is what matters.
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b)
{
    df p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df df_scale(df a, float s) { return df{__fmul_rn(a.h, s), __fmul_rn(a.l, s)}; }

// FP64 <-> double-float (O(N) conversions only; these use the FP64 pipe)
__device__ __forceinline__ df df_from_double(double x)
{
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df{h, l};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

// 2^k as a float for k in [-126, 127]; 0 below -126.
__device__ __forceinline__ float pow2f(int k) { return (k < -126) ? 0.0f : __int_as_float((k + 127) << 23); }

// ---------------------------------------------------------------------------
// Wide-exponent double-float: value = (h + l) * 2^e with h in [1,2), or zero
// (h = l = 0, e = WEF_ZERO_E).

struct dfw {
    float h, l;
    int e;
};

__device__ __forceinline__ dfw dfw_zero() { return dfw{0.0f, 0.0f, WEF_ZERO_E}; }

// Normalise a non-negative double-float into [1,2) x 2^e.
__device__ __forceinline__ dfw dfw_norm(df v, int e)
{
    if (!(v.h > 0.0f)) {
        if (v.h == 0.0f) return dfw_zero();
        return dfw{v.h, v.l, e};  // NaN propagates
    }
    const int ex = ((__float_as_int(v.h) >> 23) & 0xFF) - 127;
    const float s = pow2f(-ex);
    const int en = e + ex;
    if (en < WEF_ZERO_E / 2) return dfw_zero();
    return dfw{__fmul_rn(v.h, s), __fmul_rn(v.l, s), en};
}

__device__ __forceinline__ dfw dfw_mul(dfw a, dfw b)
{
    return dfw_norm(df_mul(df{a.h, a.l}, df{b.h, b.l}), a.e + b.e);
}

__device__ __forceinline__ dfw dfw_add(dfw a, dfw b)
{
    const int E = max(a.e, b.e);
    const float sa = pow2f(a.e - E), sb = pow2f(b.e - E);
    df s = df_add(df_scale(df{a.h, a.l}, sa), df_scale(df{b.h, b.l}, sb));
    return dfw_norm(s, E);
}

// ln of a dfw (FP64 result; O(N) use only)
__device__ __forceinline__ double dfw_log(dfw a)
{
    if (a.h == 0.0f) return -INFINITY;
    const double ln2 = 0.6931471805599453;
    return log(df_to_double(df{a.h, a.l})) + (double)a.e * ln2;
}

__device__ __forceinline__ double dfw_to_double(dfw a)
{
    if (a.h == 0.0f) return 0.0;
    double m = df_to_double(df{a.h, a.l});
    if (a.e > 1023) return INFINITY;
    if (a.e >= -1022) return m * pow2i(a.e);
    if (a.e < -1100) return 0.0;
    return (m * pow2i(a.e + 64)) * pow2i(-64);
}

// ---------------------------------------------------------------------------
// e^x for a double-float x, as a dfw.  Table-driven reduction (Tang 1989):
// x = n ln2/256 + r with |r| <= ln2/512, e^x = 2^(n>>8) * 2^((n&255)/256) * e^r.
// e^r = 1 + r + r^2/2 in double-float plus r^3 (1/6 + r/24) in float; the
// truncation error is below 4e-17 relative.  tab[j] = 2^(j/256) as a
// double-float (computed on the host).

#define DF_LN2_256_H __int_as_float(0x3b317218)   // ln2/256, high part
#define DF_LN2_256_L __int_as_float(0xad02e308)   // ln2/256 - high part
#define DF_256_LN2 369.3299255371094f              // 256/ln2 (only steers n)

// Core for |x| <= 32768 (so |n| < 2^24 and n is exact in float).
__device__ __forceinline__ dfw dfw_exp_core(df x, const float2* tab)
{
    const float t = __fmul_rn(x.h, DF_256_LN2);
    const float nf = rintf(t);
    const int n = (int)nf;
    // r = x - n*C: n*C_h is split exactly by TwoProduct, x.h - p.h exactly by TwoSum
    const df p = two_prod(nf, DF_LN2_256_H);
    const df r0 = two_sum(x.h, -p.h);
    const float rl = __fadd_rn(r0.l, __fsub_rn(__fsub_rn(x.l, p.l), __fmul_rn(nf, DF_LN2_256_L)));
    const df r = two_sum(r0.h, rl);
    // e^r
    const df r2 = df_mul(r, r);
    const float tail = __fmul_rn(__fmul_rn(r2.h, r.h), __fmaf_rn(r.h, 1.0f / 24.0f, 1.0f / 6.0f));
    df s = two_sum(1.0f, r.h);
    s.l = __fadd_rn(s.l, r.l);
    s = fast_two_sum(s.h, s.l);
    s = df_add(s, df{__fmul_rn(r2.h, 0.5f), __fmaf_rn(r2.l, 0.5f, tail)});
    const int j = n & 255, m = n >> 8;
    const float2 tj = tab[j];
    return dfw_norm(df_mul(s, df{tj.x, tj.y}), m);
}

__device__ __forceinline__ dfw dfw_exp(df x, const float2* tab)
{
    if (!(x.h > -3.0e8f)) {
        if (x.h != x.h) return dfw{x.h, 0.0f, 0};
        return dfw_zero();
    }
    if (!(x.h < 3.0e8f)) return dfw{__int_as_float(0x7fc00000), 0.0f, 0};
    if (fabsf(x.h) <= 32768.0f) return dfw_exp_core(x, tab);
    // |x| > 32768: e^x = (e^(x/2^k))^(2^k), halvings exact
    int k = 0;
    while (fabsf(x.h) > 32768.0f) {
        x = df_scale(x, 0.5f);
        ++k;
    }
    dfw y = dfw_exp_core(x, tab);
    for (int i = 0; i < k; ++i) y = dfw_mul(y, y);
    return y;
}
