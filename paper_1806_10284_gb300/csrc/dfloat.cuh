// Double-float real and complex types for the complex128 transforms on the FP32 units.
//
// A value is the unevaluated sum h + l of two floats (about 48 significant bits,
// relative rounding near 2^-47 per operation against 2^-53 for FP64).  GB300 runs
// FP64 at 1/64 of its FP32 rate, so an FFT pass whose FP64 arithmetic is the limit
// runs several times faster in this form.  Sums use Knuth's two-sum of the leading
// parts plus the trailing parts, renormalised (the "sloppy" double-float add: its
// error is relative to the larger operand, which is what an FFT butterfly needs);
// products use the exact FMA split of h_a h_b (Dekker's two-product) plus the cross
// terms.  Conversions from and to double work on the bit patterns (df64.cuh), so no
// FP64 instruction is needed except one add per value written back as a double.
//
// The types plug into the radix building blocks of fft2.cuh and the range-basis
// code of phases.cuh: dfr has the arithmetic operators those use, dfc the members
// x, y of a complex value.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"

struct dfr {
    float h, l;
    dfr() = default;
    __host__ __device__ constexpr dfr(float a, float b) : h(a), l(b) {}
    __host__ __device__ constexpr dfr(int i) : h((float)i), l(0.0f) {}
    // from a double constant (folded at compile time where the argument is constant)
    __host__ __device__ constexpr dfr(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
};

struct dfc {
    dfr x, y;
};

namespace dfl {
__device__ __forceinline__ dfr quick_two_sum(float a, float b) {
    const float s = a + b;
    return dfr(s, b - (s - a));
}
__device__ __forceinline__ dfr two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return dfr(s, (a - (s - bb)) + (b - bb));
}
}  // namespace dfl

__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
    const dfr s = dfl::two_sum(a.h, b.h);
    return dfl::quick_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ dfr operator-(dfr a) { return dfr(-a.h, -a.l); }
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return dfl::quick_two_sum(p, e);
}
__device__ __forceinline__ bool operator>(dfr a, dfr b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

// 1 / sqrt(x), x > 0 in the float range: the hardware estimate refined by two Newton
// steps y <- y + y (1 - x y^2) / 2 in double-float arithmetic (each step doubles the
// correct bits: about 2^-22 -> 2^-44 -> the format's own precision)
__device__ __forceinline__ dfr rsq(dfr x) {
    dfr y(rsqrtf(x.h), 0.0f);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const dfr r = dfr(1) - x * (y * y);
        y = y + y * (r * dfr(0.5f, 0.0f));
    }
    return y;
}
__device__ __forceinline__ dfr root(dfr x) { return x * rsq(x); }

__device__ __forceinline__ dfc mk(dfr a, dfr b) { return dfc{a, b}; }
__device__ __forceinline__ dfc operator+(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc operator-(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc operator*(dfr s, dfc a) { return dfc{s * a.x, s * a.y}; }
__device__ __forceinline__ dfc badd(dfc a, dfc b) { return a + b; }
__device__ __forceinline__ dfc bsub(dfc a, dfc b) { return a - b; }

// storage conversions: complex128 in memory <-> double-float in registers
__device__ __forceinline__ dfr to_df(double v) {
    const df64::Split s = df64::split(v);
    return dfr(s.h, s.l);
}
__device__ __forceinline__ dfc to_df(double2 v) { return dfc{to_df(v.x), to_df(v.y)}; }
__device__ __forceinline__ double to_double(dfr v) { return df64::widen(v.h) + df64::widen(v.l); }
__device__ __forceinline__ double2 to_double(dfc v) { return make_double2(to_double(v.x), to_double(v.y)); }
