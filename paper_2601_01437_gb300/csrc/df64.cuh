// Double-float ("df64") arithmetic: a value is the unevaluated sum h + l of two
// FP32 numbers with |l| <= ulp(h)/2, giving a 48-bit significand. Built from
// error-free transformations: Dekker's FastTwoSum (Dekker 1971, "A
// floating-point technique for extending the available precision"), Knuth's
// TwoSum (TAOCP vol. 2, 4.2.2) and the FMA-based TwoProduct (Ogita, Rump &
// Oishi 2005, "Accurate sum and dot product"). Division is one Newton
// correction of an FP32 quotient (the double-single scheme of Bailey's DSFUN).
//
// On GB300 FP32 FMA throughput is 62x FP64's, so a df64 operation (5-12 FP32
// instructions) costs a fraction of an FP64 one while keeping the relative
// error near 2^-44. The __f*_rn intrinsics keep the compiler from fusing or
// reassociating the error-free steps.
#pragma once

#include <cuda_runtime.h>

struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float h, float l) {
    df r;
    r.h = h;
    r.l = l;
    return r;
}

// s + e = a + b exactly, assuming |a| >= |b| or a == 0 (FastTwoSum)
__device__ __forceinline__ df df_fts(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ df df_ts(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

__device__ __forceinline__ df df_from_double(double x) {
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return df_make(h, l);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.h, -a.l); }

__device__ __forceinline__ df df_add(df a, df b) {
    const df s = df_ts(a.h, b.h);
    const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return df_fts(s.h, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);  // exact error of the product of the heads
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_fts(p, e);
}

// a * b with the tail left unnormalised (|l| may reach a few ulp(h)): exact
// head product by FMA, cross terms gathered in the tail. For chains whose next
// step is itself error-free on the head (a product, a TwoSum) and renormalises
// at the end; the relative error stays near 2^-46.
__device__ __forceinline__ df df_mul_lazy(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_make(p, e);
}

// a / b: FP32 quotient q1, exact remainder a - b*q1 from TwoProduct, one correction
__device__ __forceinline__ df df_div(df a, df b) {
    const float rb = __frcp_rn(b.h);
    const float q1 = __fmul_rn(a.h, rb);
    const float p = __fmul_rn(b.h, q1);
    const float pe = __fmaf_rn(b.h, q1, -p);
    float r = __fsub_rn(a.h, p);
    r = __fsub_rn(r, pe);
    r = __fadd_rn(r, a.l);
    r = __fmaf_rn(-b.l, q1, r);
    const float q2 = __fmul_rn(r, rb);
    return df_fts(q1, q2);
}

// 1 / b
__device__ __forceinline__ df df_rcp(df b) { return df_div(df_make(1.0f, 0.0f), b); }

// a * b + c (TwoProduct of the heads, TwoSum with c's head, tails summed)
__device__ __forceinline__ df df_fma(df a, df b, df c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const df s = df_ts(p, c.h);
    return df_fts(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}

// The FP64 route of df_split_bits, out of line: inlined, the compiler may
// predicate it into the common path, where its conversions would issue for every
// value at the FP64 rate.
static __device__ __noinline__ df df_from_double_rare(double x) { return df_from_double(x); }

// Double-float split of an FP64 value by integer operations (no FP64
// instruction on the common path): the head is the value rounded to 24
// significant bits (the carry of the rounding increment runs into the
// exponent field), the tail is the remaining 29 fraction bits minus the
// rounding increment, converted once and scaled by 2^(e - 52). Exact head,
// tail within 2^-24 of itself: |x - h - l| <= 2^-48 |x|. Values outside
// [2^-70, 2^100] other than zero take the FP64 route.
__device__ __forceinline__ df df_split_bits(double x) {
    // the two 32-bit words directly (no 64-bit integer operations)
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    if (((hi << 1) | lo) == 0u) return df_make(__uint_as_float(hi & 0x80000000u), 0.f);  // +-0
    if (ex < 1023 - 70 || ex > 1023 + 100) return df_from_double_rare(x);
    const unsigned sign = hi & 0x80000000u;
    const unsigned up = (lo >> 28) & 1u;  // first dropped bit: round the head up
    const unsigned hb = (((unsigned)(ex - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)) + up;
    const int rt = (int)(lo & 0x1fffffffu) - (int)(up << 29);  // tail in units of 2^(ex - 1075)
    const float scale = __uint_as_float((unsigned)(ex - 948) << 23);  // 2^(ex - 1075)
    // rt as FP32 without an integer-to-float conversion (those issue at the FP64
    // rate on this part): rt = th 2^14 + tl with |th| < 2^15, 0 <= tl < 2^14, each
    // exact in FP32 by adding it into the mantissa of 1.5 * 2^23 and subtracting
    // that again; one FMA then rounds th 2^14 + tl to nearest, as a conversion would.
    const int th = rt >> 14, tl = rt & 0x3fff;
    const float fh = __fsub_rn(__int_as_float(0x4B400000 + th), 12582912.0f);
    const float fl = __fsub_rn(__int_as_float(0x4B400000 + tl), 12582912.0f);
    const float l = __fmul_rn(__fmaf_rn(fh, 16384.0f, fl), scale);
    return df_make(__uint_as_float(sign | hb), sign ? -l : l);
}

// 1 / b for b.h >= 1: the hardware's approximate FP32 reciprocal, one FP32
// Newton step (relative error ~2^-24), then the double-float correction
// q = r0 + r0 (1 - b r0) with the remainder 1 - b r0 formed exactly, which
// squares the FP32 error (~2^-47 relative).
__device__ __forceinline__ df df_rcp_ge1(df b) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(b.h));
    r0 = __fmaf_rn(r0, __fmaf_rn(-b.h, r0, 1.0f), r0);
    const float p = __fmul_rn(b.h, r0);
    const float pe = __fmaf_rn(b.h, r0, -p);  // b.h r0 = p + pe exactly
    float r = __fsub_rn(1.0f, p);             // exact: p is within 2^-22 of 1
    r = __fsub_rn(r, pe);
    r = __fmaf_rn(-b.l, r0, r);
    return df_fts(r0, __fmul_rn(r, r0));
}

// 1 / sqrt(s) for s > 0: the approximate FP32 reciprocal square root y0, then
// one Newton step y0 + y0 (1 - s y0^2) / 2 with s y0^2 formed in double-float
// (y0^2 exactly by TwoProduct), which squares y0's error (~2^-46 relative).
__device__ __forceinline__ df df_rsqrt(df s) {
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(s.h));
    const float q = __fmul_rn(y0, y0);
    const df t = df_mul(s, df_make(q, __fmaf_rn(y0, y0, -q)));  // s y0^2, close to 1
    const float r = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);       // 1 - t.h is exact
    return df_fts(y0, __fmul_rn(__fmul_rn(0.5f, y0), r));
}


// Multiply by 2^e exactly (as long as the result stays in the FP32 normal range)
__device__ __forceinline__ df df_ldexp(df a, int e) { return df_make(ldexpf(a.h, e), ldexpf(a.l, e)); }
