// Double-float arithmetic for FP64-accurate sums of products at FP32 rate.
//
// A double x is carried as the unevaluated sum h + l of two floats: h holds the
// leading 24 significant bits of x (truncated) and l the remaining 29 bits
// rounded to 24, so h + l equals x to about 2^-48 relative.  Products use the
// exact FMA split of h_a h_b (Dekker's two-product, with the hardware FMA) plus
// the cross terms h_a l_b + l_a h_b; sums use Knuth's two-sum, so a running sum
// S + E keeps about 2^-47 relative accuracy.  The double <-> float conversions
// are done on the bit patterns with integer instructions.
#pragma once

#include <cuda_runtime.h>

namespace df64 {

struct Split { float h, l; };

// x = h + l (exact for |x| in [2^-74, 2^127]; below 2^-125 both parts are 0,
// a relative loss far below what the callers resolve)
__device__ __forceinline__ Split split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    Split r;
    if (e < -125) {
        r.h = 0.0f;
        r.l = 0.0f;
        return r;
    }
    if (e > 127) {                       // out of float range: not met by the callers' data
        r.h = (float)x;
        r.l = 0.0f;
        return r;
    }
    r.h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    const unsigned ml = lo & 0x1fffffffu;             // the low 29 mantissa bits, weight 2^(e-52)
    const float low = (e >= -74 && ml) ? __uint2float_rn(ml) * __uint_as_float((unsigned)(e + 75) << 23) : 0.0f;
    r.l = sign ? -low : low;
    return r;
}

// x rounded to a float (h + l in one single-precision add), without an FP64 conversion
__device__ __forceinline__ float narrow(double x) {
    const Split s = split(x);
    return s.h + s.l;
}

// exact float -> double
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xffu;
    if (ef == 0u || ef == 0xffu) return (double)f;    // zero, subnormal, inf, nan
    const unsigned hi = (u & 0x80000000u) | ((ef + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    const unsigned lo = (u & 0x7u) << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// (S, E) += (ah + al)(bh + bl), dropping al bl
__device__ __forceinline__ void mac(float& S, float& E, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);                       // ah bh = p + e exactly
    e = fmaf(ah, bl, fmaf(al, bh, e));
    const float s = S + p;                            // two-sum: S + p = s + err exactly
    const float bb = s - S;
    const float err = (S - (s - bb)) + (p - bb);
    S = s;
    E += err + e;
}

}  // namespace df64
