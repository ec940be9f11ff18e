// gwam_df.cuh -- FP64-free building blocks for GB300, whose FP64 rate is 1/72 of its FP32 rate:
// exact float <-> double conversions by integer operations and double-float ("DF") arithmetic,
// hi + lo pairs of FP32 values carrying about 48 significant bits on the FP32 pipes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gwam {

// Exact float -> double with integer operations only (on GB300 the conversion instruction runs at
// the FP64 rate): sign kept, exponent re-biased from 127 to 1023, the 23 mantissa bits moved to the
// top of the 52-bit field; subnormal floats are normalised first; infinities and NaNs keep their
// class.
__device__ __forceinline__ double widen(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint32_t sign = u & 0x80000000u;
    uint32_t ex = (u >> 23) & 0xFFu, man = u & 0x7FFFFFu;
    if (ex == 0xFFu) return __hiloint2double((int)(sign | 0x7FF00000u | (man >> 3)), (int)(man << 29));
    if (ex == 0u) {
        if (man == 0u) return __hiloint2double((int)sign, 0);
        const int sh = __clz((int)man) - 8;   // moves the leading one to bit 23
        man = (man << sh) & 0x7FFFFFu;
        ex = 1u - (uint32_t)sh;               // wraps below zero; the re-bias brings it back
    }
    return __hiloint2double((int)(sign | ((ex + 896u) << 20) | (man >> 3)), (int)(man << 29));
}

// double -> float, round to nearest even, with integer operations only (the conversion instruction
// runs at the FP64 rate on GB300).  The 53-bit significand is shifted right to 24 bits (fewer for
// a float subnormal) and rounded on the dropped bits; a carry out of the significand moves into
// the exponent, an exponent beyond the float range gives infinity, infinities and NaNs keep their
// class.
__device__ __forceinline__ float narrow_general(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u | (uint32_t)(m >> 29) : 0u));
    const int E = e - 896;                       // float biased exponent (1023 - 127)
    if (E >= 255) return __uint_as_float(sign | 0x7F800000u);
    const int shift = E > 0 ? 29 : 30 - E;       // significand bits dropped
    if (shift > 60) return __uint_as_float(sign);
    const unsigned long long mm = m | (e ? (1ull << 52) : 0ull);
    const unsigned long long keep = mm >> shift;
    const unsigned long long rem = mm & ((1ull << shift) - 1ull);
    const unsigned long long half = 1ull << (shift - 1);
    const unsigned long long q = keep + ((rem > half || (rem == half && (keep & 1ull))) ? 1ull : 0ull);
    uint32_t r = E > 0 ? ((uint32_t)E << 23) + (uint32_t)(q - (1ull << 23)) : (uint32_t)q;
    if (r > 0x7F800000u) r = 0x7F800000u;
    return __uint_as_float(sign | r);
}

// Fast path of narrow for the usual cases -- the result is a normal float or rounds up to infinity,
// or x has a zero exponent field (zeros and FP64 subnormals, far below the float range: a signed
// zero) -- with 32-bit operations on the two words of the double and no branch between them;
// everything else takes narrow_general.  The zeros are folded in because projected fields are
// mostly empty cells: a warp mixing zeros and nonzeros would otherwise run both paths.
__device__ __forceinline__ float narrow(double x)
{
    const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
    const uint32_t e = (hw >> 20) & 0x7FFu;
    uint32_t r = (((hw & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lw >> 29);
    const uint32_t rem = lw & 0x1FFFFFFFu;      // the 29 dropped bits
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
    const bool normal = e - 897u < 254u;        // float exponent 1 .. 254
    if (normal || e == 0u) return __uint_as_float((hw & 0x80000000u) | (normal ? r : 0u));
    return narrow_general(x);
}

// Double-float values hi + lo on the FP32 pipes, about 48 significant bits: products by TwoProduct
// (an FMA gives the exact rounding error), sums by TwoSum (Dekker 1971, Knuth); every operation is
// an explicitly rounded intrinsic, never contracted or reordered.  Sums are renormalised
// (FastTwoSum); products return the unevaluated pair they form -- the rounded product and the sum of
// its rounding error and cross terms, |lo| at most a few ulp(hi) -- without renormalising: the next
// operation takes both parts, so this costs a few units of 2^-48 and saves three of a product's seven
// instructions (the ray-step kernel: 0.77 -> 0.67 ms per step on the sphere together with the
// double-float increment sums of rk3).  A sum must stay renormalised: after a cancellation its
// unrenormalised pair can have |lo| near |hi|, and a product that drops lo x lo then keeps only FP32
// precision (measured: errors up to 5e-8 of the flux scales).  floor, ceil and comparisons
// renormalise first (df_norm).
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ DF df_mul(DF x, float b)
{
    const float p = __fmul_rn(x.hi, b);
    const float e = __fmaf_rn(x.lo, b, __fmaf_rn(x.hi, b, -p));
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb)), __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

// a - b exactly as a double-float
__device__ __forceinline__ DF df_diff(float a, float b)
{
    const float s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb))};
}

// hi + lo as a double (exact: the two parts span far fewer than 53 bits); a value that is one float
// needs no FP64 add
__device__ __forceinline__ double df_to_double(DF x)
{
    return x.lo == 0.0f ? widen(x.hi) : widen(x.hi) + widen(x.lo);
}

// Segmented inclusive sum over runs of equal keys in a warp, in double-float: the FP32 pipes do the
// additions, the last lane of each run holds the run's sum (a scan by key at distances 1, 2, 4, ...).
// Returns true on the last lane of a run.  All 32 lanes must call it; every lane its own run returns
// at once.
template <int NV>
__device__ __forceinline__ bool warp_segment_reduce_df(int key, DF (&v)[NV])
{
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    if (heads == 0xffffffffu) return true;
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    // the warp's longest run: the steps at distances beyond it would add nothing (no lane has a run
    // partner that far back), so they are skipped -- the same sums, bit for bit
    const unsigned longest = __reduce_max_sync(0xffffffffu, (unsigned)(lane - start + 1));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if ((unsigned)d >= longest) break;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            DF o;
            o.hi = __shfl_up_sync(0xffffffffu, v[q].hi, d);
            o.lo = __shfl_up_sync(0xffffffffu, v[q].lo, d);
            if (lane - d >= start) v[q] = df_add(v[q], o);
        }
    }
    return lane == 31 || next != key;
}


__device__ __forceinline__ DF df_mul2(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return {p, e};
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
// multiplication by a power of two (exact)
__device__ __forceinline__ DF df_pow2(DF a, float s) { return {a.hi * s, a.lo * s}; }
__device__ __forceinline__ DF df_f(float a) { return {a, 0.0f}; }

// renormalise an unevaluated sum s + c into a DF pair (TwoSum)
__device__ __forceinline__ DF df_norm(float s, float c)
{
    const float h = __fadd_rn(s, c);
    const float bb = __fsub_rn(h, s);
    return {h, __fadd_rn(__fsub_rn(s, __fsub_rn(h, bb)), __fsub_rn(c, bb))};
}

// 1 / x: the FP32 hardware approximation (about 23 correct bits) refined by one Newton step
// y <- y + y (1 - x y) in DF, which squares the relative error to about 2^-45
__device__ __forceinline__ DF df_rcp(DF x)
{
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x.hi));
    const DF e = df_sub(df_f(1.0f), df_mul(x, r0));
    return df_add(df_f(r0), df_mul(e, r0));
}

// 1 / sqrt(x): the FP32 hardware approximation refined by one Newton step
// y <- y + y (1 - x y^2) / 2 in DF (relative error about 2^-45, as df_rcp)
__device__ __forceinline__ DF df_rsqrt(DF x)
{
    float r0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x.hi));
    const DF e = df_sub(df_f(1.0f), df_mul2(x, df_prod(r0, r0)));
    return df_add(df_f(r0), df_pow2(df_mul(e, r0), 0.5f));
}

// floor and ceil of hi + lo (renormalised first, so that lo only matters when hi is an integer)
__device__ __forceinline__ float df_floor(DF x)
{
    x = df_norm(x.hi, x.lo);
    const float f = floorf(x.hi);
    return (f == x.hi && x.lo < 0.0f) ? f - 1.0f : f;
}
__device__ __forceinline__ float df_ceil(DF x)
{
    x = df_norm(x.hi, x.lo);
    const float f = ceilf(x.hi);
    return (f == x.hi && x.lo > 0.0f) ? f + 1.0f : f;
}
// a < b (both renormalised first)
__device__ __forceinline__ bool df_less(DF a, DF b) { a = df_norm(a.hi, a.lo); b = df_norm(b.hi, b.lo); return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// x = hi + lo to about 48 bits: hi = x rounded to FP32, lo = (x - hi) rounded to FP32.  For
// 2^-74 <= |x| < 2^127 (hi a finite normal float, lo normal or zero) with integer operations and one
// int -> float conversion, no FP64 instruction: x - hi is the 29 bits narrow dropped, less 2^29 when
// it rounded up, in units of 2^(e - 1075); that integer rounded to FP32 and scaled by the power of
// two is RN(x - hi) exactly.  Zeros and FP64 subnormals (e = 0; the empty cells of a projected
// field) round to hi = +-0 and lo = x rounded, +-0 likewise (+0 for a zero x).  Other x:
// narrow(x - widen(hi)) (one FP64 subtraction), the same values.
__device__ __forceinline__ DF df_split(double x)
{
    const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
    const uint32_t e = (hw >> 20) & 0x7FFu;
    if (e == 0u) {
        const uint32_t sign = hw & 0x80000000u;
        return {__uint_as_float(sign), __uint_as_float(((hw & 0xFFFFFu) | lw) ? sign : 0u)};
    }
    if (e - 949u < 201u) {
        uint32_t r = (((hw & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lw >> 29);
        const uint32_t rem = lw & 0x1FFFFFFFu;   // the 29 dropped bits
        const bool up = rem > 0x10000000u || (rem == 0x10000000u && (r & 1u));
        r += up ? 1u : 0u;
        const uint32_t sign = hw & 0x80000000u;
        int res = up ? (int)rem - (1 << 29) : (int)rem;   // |res| <= 2^28
        if (sign) res = -res;
        const float scale = __uint_as_float((e - 948u) << 23);   // 2^(e - 1075), a normal float
        return {__uint_as_float(sign | r), __fmul_rn(__int2float_rn(res), scale)};
    }
    const float hi = narrow(x);
    return {hi, narrow(x - widen(hi))};
}

// ln(a / b) for positive normal doubles, in double-float on the FP32 pipes.  a = 2^ea ma and
// b = 2^eb mb with ma, mb in [1, 2) (exponent fields set by integer operations); mb is doubled when
// ma / mb >= sqrt(2) and ma when ma / mb < sqrt(1/2), so that ma / mb lies in [sqrt(1/2), sqrt(2))
// and a / b = 2^e ma / mb.
// Then ln(ma / mb) = 2 atanh(s), s = (ma - mb) / (ma + mb), |s| < 0.172 (the difference is exact
// in FP64: ma and mb lie within a factor of two), from the series
// ln = 2 s (1 + s^2/3 + s^4/5 + ...) (Abramowitz & Stegun 4.1.27): the terms to s^8/9 in DF,
// s^10/11 ... s^20/21 in FP32 (each below 2e-9 of the sum), truncated after s^20/21 (the next term is
// below 1e-18); e ln 2 with ln 2 as a DF constant.  Relative error about 2^-45: logarithms of
// ratios near one keep their relative precision.
__device__ __forceinline__ DF df_log_ratio(double a, double b)
{
    const int ha = __double2hiint(a), hb = __double2hiint(b);
    int e = ((ha >> 20) & 0x7FF) - ((hb >> 20) & 0x7FF);
    double ma = __hiloint2double((ha & 0x800FFFFF) | 0x3FF00000, __double2loint(a));
    double mb = __hiloint2double((hb & 0x800FFFFF) | 0x3FF00000, __double2loint(b));
    // ma / mb in (1/2, 2): the leading mantissa bits decide (either side of a boundary is accurate)
    const float fa = __int_as_float(((ha & 0x000FFFFF) << 3) | 0x3F800000);
    const float fb = __int_as_float(((hb & 0x000FFFFF) << 3) | 0x3F800000);
    if (fa >= 1.41421356f * fb) {
        mb = __hiloint2double(__double2hiint(mb) + 0x00100000, __double2loint(mb));   // 2 mb
        e += 1;
    } else if (fa * 1.41421356f < fb) {
        ma = __hiloint2double(__double2hiint(ma) + 0x00100000, __double2loint(ma));   // 2 ma
        e -= 1;
    }
    const DF num = df_split(ma - mb), den = df_split(ma + mb);
    float d0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(d0) : "f"(den.hi));
    const DF id1 = df_add(df_f(d0), df_mul(df_sub(df_f(1.0f), df_mul(den, d0)), d0));
    const DF id = df_add(id1, df_mul2(df_sub(df_f(1.0f), df_mul2(den, id1)), id1));
    const DF t = df_mul2(num, id);
    const DF t2 = df_mul2(t, t);
    const float z = t2.hi;
    const float tail = 1.0f / 11.0f + z * (1.0f / 13.0f + z * (1.0f / 15.0f + z * (1.0f / 17.0f + z * (1.0f / 19.0f + z * (1.0f / 21.0f)))));
    constexpr DF c3{1.0f / 3.0f, (float)(1.0 / 3.0 - (double)(1.0f / 3.0f))};
    constexpr DF c5{1.0f / 5.0f, (float)(1.0 / 5.0 - (double)(1.0f / 5.0f))};
    constexpr DF c7{1.0f / 7.0f, (float)(1.0 / 7.0 - (double)(1.0f / 7.0f))};
    constexpr DF c9{1.0f / 9.0f, (float)(1.0 / 9.0 - (double)(1.0f / 9.0f))};
    constexpr DF ln2{0.693147182f, (float)(0.69314718055994530942 - (double)0.693147182f)};
    DF p = df_add(c9, df_mul(t2, tail));
    p = df_add(c7, df_mul2(t2, p));
    p = df_add(c5, df_mul2(t2, p));
    p = df_add(c3, df_mul2(t2, p));
    p = df_add(df_f(1.0f), df_mul2(t2, p));
    const DF lnm = df_mul2(df_pow2(t, 2.0f), p);
    return df_add(df_mul(ln2, (float)e), lnm);
}

}  // namespace gwam
