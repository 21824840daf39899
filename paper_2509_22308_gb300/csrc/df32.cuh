// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2 (about 48 significant bits, the FP32 exponent range).  On GB300 the
// FP32 pipe issues 64 times as many operations per clock as the FP64 pipe, so a
// double-float step is bound by HBM (8 bytes per value, as FP64) instead of by the FP64
// pipe, at an accuracy close to FP64's.
//
// The operations are the published error-free transformations and double-word algorithms:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971), TwoProd by FMA;
//   sum of two double-words: AccurateDWPlusDW, product: DWTimesDW (Joldes, Muller and
//   Popescu, "Tight and rigorous error bounds for basic building blocks of double-word
//   arithmetic", ACM TOMS 44 (2017)), whose relative errors are a few u^2 (u = 2^-24).
// Every FP32 operation is an explicitly rounded intrinsic, so nothing is contracted or
// reassociated.
#pragma once

#include <cuda_runtime.h>

namespace lbmem {

struct alignas(8) df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // nearest double-float to a double (hi = x rounded, lo = the rest rounded)
    __host__ __device__ explicit df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit df(int x) : df((double)x) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator+(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
    const float ch = __fmul_rn(a.hi, b.hi);
    const float cl1 = __fmaf_rn(a.hi, b.hi, -ch);
    const float cl2 = __fadd_rn(cl1, __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.lo)));
    return fast_two_sum(ch, cl2);
}

__device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }

// a * b + c as a product and a sum (no fused double-word form is used)
__device__ __forceinline__ df fmat(df a, df b, df c) { return a * b + c; }

// The runaway test of common.cuh (exponent field >= thr, the FP32 threshold): the leading
// word decides
__device__ __forceinline__ bool field_runaway(df e3, unsigned thr) {
    return (__float_as_uint(e3.hi) & 0x7f800000u) >= thr;
}

}  // namespace lbmem
