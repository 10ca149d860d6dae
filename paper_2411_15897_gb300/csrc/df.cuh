// Double-FP32 ("double-float") arithmetic for the Krylov vectors.
//
// A real number is stored as an unevaluated sum hi + lo of two FP32 values
// (48 significant bits); a complex entry is a float4 (re.hi, re.lo, im.hi,
// im.lo), 16 bytes like an FP64 complex.  Products use the error-free FMA
// product (Dekker/Kahan: p = a*b, e = fma(a, b, -p) exactly), sums use Knuth's
// two-sum; both are exact transformations, so a double-float dot product is
// accurate to about 2^-47 relative to the sum of magnitudes.  Conversion from
// FP64 splits the bit pattern with integer operations (no FP64 arithmetic):
// hi keeps the leading 24 significand bits, lo the next 24 (truncation), so
// hi + lo equals the double to 2^-47 relative.  Values below the FP32 normal
// range (|x| < 1.2e-38) are flushed to zero.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bah {

struct dfl { float hi, lo; };

__device__ __forceinline__ dfl df_from_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const int fe = e - 1023 + 127;
    dfl r;
    if (e == 0 || fe <= 0) { r.hi = 0.f; r.lo = 0.f; return r; }
    if (fe >= 255) { r.hi = __int_as_float((int)(sign | 0x7F800000u)); r.lo = 0.f; return r; }   // overflow: inf
    r.hi = __int_as_float((int)(sign | ((unsigned int)fe << 23) | (unsigned int)(m >> 29)));
    const unsigned long long rest = m & 0x1FFFFFFFull;          // 29 remaining bits, weight 2^(e-1075)
    if (rest == 0) { r.lo = 0.f; return r; }
    const int nb = 64 - __clzll((long long)rest);               // significant bits of rest (1..29)
    const unsigned int mant = nb > 24 ? (unsigned int)(rest >> (nb - 24)) : (unsigned int)(rest << (24 - nb));
    const int le = nb + e - 949;                                 // biased FP32 exponent of lo
    if (le <= 0) { r.lo = 0.f; return r; }
    r.lo = __int_as_float((int)(sign | ((unsigned int)le << 23) | (mant & 0x7FFFFFu)));
    return r;
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// exact sum of two floats: s + e = a + b
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ dfl df_renorm(float hi, float lo) {
    dfl r;
    r.hi = hi + lo;
    r.lo = lo - (r.hi - hi);
    return r;
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return df_renorm(s, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) { dfl r; r.hi = -a.hi; r.lo = -a.lo; return r; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_renorm(p, e);
}

// a (double-float) times a float, to about 2^-47 relative
__device__ __forceinline__ dfl df_mul_f(dfl a, float x) {
    const float p = a.hi * x;
    float e = fmaf(a.hi, x, -p);
    e = fmaf(a.lo, x, e);
    return df_renorm(p, e);
}
// a - b for two floats, exactly, as a double-float
__device__ __forceinline__ dfl df_diff_f(float a, float b) {
    dfl r;
    two_sum(a, -b, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ dfl df_of(const float2& v) { dfl r; r.hi = v.x; r.lo = v.y; return r; }

// accumulator for long sums: acc += a*b, renormalised on every step
struct dfacc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(dfl a, dfl b) {
        const float p = a.hi * b.hi;
        float pe = fmaf(a.hi, b.hi, -p);
        pe = fmaf(a.hi, b.lo, pe);
        pe = fmaf(a.lo, b.hi, pe);
        float s, e;
        two_sum(hi, p, s, e);
        e += lo + pe;
        hi = s + e;
        lo = e - (hi - s);
    }
    __device__ __forceinline__ void add(dfl a) {
        float s, e;
        two_sum(hi, a.hi, s, e);
        e += lo + a.lo;
        hi = s + e;
        lo = e - (hi - s);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// complex double-float stored as float4 (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ dfl re_of(const float4& v) { dfl r; r.hi = v.x; r.lo = v.y; return r; }
__device__ __forceinline__ dfl im_of(const float4& v) { dfl r; r.hi = v.z; r.lo = v.w; return r; }
__device__ __forceinline__ float4 cdf_make(dfl re, dfl im) { return make_float4(re.hi, re.lo, im.hi, im.lo); }
__device__ __forceinline__ float4 cdf_from_double2(double2 z) { return cdf_make(df_from_double(z.x), df_from_double(z.y)); }
__device__ __forceinline__ double2 cdf_to_double2(const float4& v) {
    return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

}  // namespace bah
