// dfloat.cuh -- double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi), about 48 significant bits. Used by the FP64-accurate
// residual b - A x of iterative refinement, which then runs on the FP32 pipes (on GB300 the FP64
// pipe has 1/62 of the FP32 rate).
//
// The error-free transformations are the classical ones: the exact product a*b = p + e with
// e = fma(a, b, -p) (one rounding of the fused multiply-add), and Knuth's two-sum
// s + e = a + b (six additions, no ordering requirement). Sums are left unnormalised (hi is the
// rounded leading sum, lo collects the exact errors and may exceed half an ulp of hi): over the
// few dozen taps of one output lo stays a few ulps of the largest partial sum, which costs no
// accuracy (its own rounding is 2^-24 of that) and saves the three-operation renormalisation per
// tap. Every operation uses the explicitly rounded intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn)
// so that the compiler cannot contract a multiply and an add into one fused operation, which
// would break the transformations.
#pragma once

#include <cstdint>

namespace bsk {

struct __align__(8) dfl {
    float hi, lo;   // value hi + lo (not necessarily normalised)
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}   // exact for |v| < 2^24
    // host-side split of a double (kernel coefficients): hi = round(v), lo = round(v - hi)
    __host__ static dfl from_double_host(double v)
    {
        const float h = (float)v;
        return dfl(h, (float)(v - (double)h));
    }
};

struct __align__(16) dfl2 {
    dfl x, y;
};

// (s, e) with s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// c + a * b (a.lo * b.lo, below 2^-48 of the product, is dropped)
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, se;
    two_sum(c.hi, p, s, se);
    return dfl(s, __fadd_rn(se, __fadd_rn(pe, c.lo)));
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return dfl(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl(-a.hi, -a.lo); }

// Split of a double into hi + lo without the FP64 pipe: hi keeps the leading 24 significant bits
// (truncated), lo the next ones (the 29 remaining bits rounded to 24), so hi + lo equals d to
// about 2^-47 relative. Zero and subnormal inputs give 0; magnitudes below 2^-74 or beyond the
// float range fall back to a plain conversion (hi only).
__device__ __forceinline__ dfl df_from_double(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned top = (unsigned)(u >> 32);
    const int e = (int)((top >> 20) & 0x7ffu);
    if (e == 0) return dfl(0.f, 0.f);
    if (e < 949 || e > 1023 + 127) return dfl(__double2float_rn(d), 0.f);
    const unsigned sign = top & 0x80000000u;
    const unsigned long long mant = u & 0xfffffffffffffull;
    const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(mant >> 29));
    const float scale = __uint_as_float((unsigned)(e - 1023 - 52 + 127) << 23);   // 2^(e - 1075)
    float lo = __fmul_rn(__uint2float_rn((unsigned)(mant & 0x1fffffffull)), scale);
    if (sign) lo = -lo;
    return dfl(hi, lo);
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

}  // namespace bsk
