// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits (internal).
//
// On this GPU the FP32 pipe issues about sixty times the FP64 pipe's rate,
// so an FFT whose butterflies run in double-float (a few FP32 operations per
// FP64 one) is several times faster than the same FFT in FP64, at a rounding
// error about 30 times FP64's and 2^24 times below FP32's.  The building
// blocks are the error-free transformations of Knuth (TwoSum), Dekker
// (FastTwoSum) and the FMA form of TwoProduct; the sum below is the
// "sloppy" double-float addition (error bounded relative to |a| + |b|, which
// is the bound an FFT's error analysis uses).  Every operation is written
// with round-to-nearest intrinsics so that no contraction or reassociation
// changes it.
#pragma once
#include "common.cuh"

struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (hi is d rounded to float, lo the rest
    // rounded); constant-folded where d is a compile-time constant
    __host__ __device__ constexpr dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

struct dfc {
    dfl x, y;
};

template <> struct cplx<dfl> { using type = dfc; };

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));   // TwoSum(a.hi, b.hi)
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);                                                  // FastTwoSum(s, e)
    return dfl(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);                                             // TwoProduct(a.hi, b.hi)
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return dfl(h, __fsub_rn(e, __fsub_rn(h, p)));
}

__device__ __forceinline__ dfc operator+(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc operator-(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc operator*(dfc a, dfc b) { return dfc{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ dfc operator*(dfc a, dfl s) { return dfc{a.x * s, a.y * s}; }
